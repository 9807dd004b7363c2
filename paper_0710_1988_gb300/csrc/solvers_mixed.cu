// Mixed-precision BiCGStab with FP64 reliable updates, batched over
// right-hand sides (the "precision" growth line of the workload; the paper
// itself is silent on precision).
//
// The Krylov vectors r, r_hat, p, v, t and the solution increment xs live in
// FP32 ([rhs][6][V] float4) and the iteration runs in the FP32 kernels of
// mixed.cu, with the same device-resident FP64 scalars and per-system status
// words as the FP64 solver.  Every `reliable_every` iterations, and whenever
// a recursive FP32 residual reaches the tolerance, the FP64 state is
// refreshed: x += xs, r = b - A x with the FP64 operator, r_fp32 = r.  A
// system is done only when that FP64 residual is below the tolerance.  Each
// chunk of iterations between host status reads is captured once as a CUDA
// graph and replayed.
//
// With FP16 storage (h->mixed_bits = 16) the three vectors the operator
// reads or writes, p, v and t, are half vectors with a per-site norm and the
// links are FP16; r, r_hat and xs stay FP32 so that the recursive residual
// and the dots it feeds keep FP32 accuracy between reliable updates.
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "mixed.h"
#include "solvers.h"
#include "wd_internal.h"

namespace wd {

namespace {

#define RET_IF(call)              \
  do {                            \
    int rc_ = (call);             \
    if (rc_ != WD_OK) return rc_; \
  } while (0)

int ok(cudaError_t e, const char *what) { return e == cudaSuccess ? WD_OK : cuda_fail(e, what); }

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  ~GraphGuard() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

}  // namespace

int ensure_links32(wd_context *h, cudaStream_t s) {
  if (h->V >= (1LL << 31)) {
    set_error("the FP32/FP16 kernels index sites with 32 bits: fewer than 2^31 sites");
    return WD_BAD_ARG;
  }
  if (h->links32 != nullptr) return WD_OK;
  WD_CK(cudaMalloc(&h->links32, sizeof(float4) * 12 * h->V));
  WD_CK(launch_links_to_f32(h, h->links32, s));
  return WD_OK;
}

int ensure_links16(wd_context *h, cudaStream_t s) {
  if (h->V >= (1LL << 31)) {
    set_error("the FP32/FP16 kernels index sites with 32 bits: fewer than 2^31 sites");
    return WD_BAD_ARG;
  }
  if (h->eo) {
    set_error("the FP16 kernels act on the full operator: switch the handle back with wd_set_operator(h, 0)");
    return WD_BAD_ARG;
  }
  if (h->links16 != nullptr) return WD_OK;
  WD_CK(cudaMalloc(&h->links16, sizeof(uint2) * 20 * h->V));   // 4 links x 5 uint2
  WD_CK(launch_links_to_f16(h, h->links16, s));
  return WD_OK;
}

int bicgstab_mixed_batched(wd_context *h, const double2 *B, double2 *X, const double2 *R0,
                           int nrhs, double tol, int max_iter, int reliable_every,
                           wd_stats *stats, cudaStream_t s, Arena &ar) {
  const bool half = h->mixed_bits == 16;
  const bool eo = h->eo != 0;  // FP32 only: the Schur operator on even half vectors
  if (eo && half) {
    set_error("FP16 storage acts on the full operator: use FP32 storage with even-odd");
    return WD_BAD_ARG;
  }
  RET_IF(half ? ensure_links16(h, s) : ensure_links32(h, s));
  const long long V = eo ? h->V / 2 : h->V, n = op_n(h), n4 = 6 * V;
  const size_t v32 = (size_t)nrhs * n4, nv = (size_t)nrhs * V;
  float4 *r = ar.take<float4>(v32), *rhat = ar.take<float4>(v32), *xs = ar.take<float4>(v32);
  float4 *p = nullptr, *v = nullptr, *t = nullptr;
  Half16 p16{}, v16{}, t16{};
  if (half) {
    p16 = Half16{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
    v16 = Half16{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
    t16 = Half16{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
  } else {
    p = ar.take<float4>(v32);
    v = ar.take<float4>(v32);
    t = ar.take<float4>(v32);
  }
  double2 *r64 = ar.take<double2>((size_t)nrhs * n), *tmp64 = ar.take<double2>((size_t)nrhs * n);
  float4 *tmp_o = eo ? ar.take<float4>(v32) : nullptr;  // odd half vectors of the Schur operator
  {  // pick the Wilson kernel's launch shape for this nrhs once per handle
    const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
    if (!half && !eo && h->tune_R[key] == 0 && !ar.failed) {
      WD_CK(cudaMemsetAsync(r, 0, sizeof(float4) * v32, s));
      WD_CK(tune_wilson_f32(h, h->links32, nrhs, r, v, s));
    }
    if (half && h->tune16_R[key] == 0 && !ar.failed) {
      WD_CK(cudaMemsetAsync(p16.v, 0, sizeof(uint4) * 3 * nv, s));
      WD_CK(cudaMemsetAsync(p16.n, 0, sizeof(float) * nv, s));
      WD_CK(tune_wilson_f16(h, h->links16, nrhs, p16, v16, s));
    }
  }
  const int nbw = eo ? schur32_blocks(h) : half ? wilson16_blocks(h, nrhs) : wilson32_blocks(h, nrhs);
  const int nbs = half ? stream16_blocks(V) : stream32_blocks(n4), nbc = conv_blocks_count(V);
  const int nb64 = stream_blocks(n);
  double *part_w = ar.take<double>((size_t)nrhs * nbw * 3);
  double *part_s = ar.take<double>((size_t)nrhs * nbs * 3);
  double *part_c = ar.take<double>((size_t)nrhs * nbc * 3);
  double *part_b = ar.take<double>((size_t)nrhs * nb64 * 3);
  BicgScalars *sc = ar.take<BicgScalars>(nrhs);
  int *status = ar.take<int>(nrhs);
  if (ar.failed) return WD_OUT_OF_MEMORY;
  const Mixed32 m{h, h->links32};

  std::vector<BicgScalars> hsc(nrhs);
  const bool restart = h->mixed_delta > 0.0;
  for (auto &q : hsc) {
    std::memset(&q, 0, sizeof(q));
    q.tol = tol;
    q.tol_outer = tol;
    q.delta = h->mixed_delta;
    q.max_iter = max_iter;
    q.max_restarts = 0;
  }
  WD_CK(cudaMemcpyAsync(sc, hsc.data(), sizeof(BicgScalars) * nrhs, cudaMemcpyHostToDevice, s));
  WD_CK(cudaMemsetAsync(status, 0, sizeof(int) * nrhs, s));
  WD_CK(cudaMemsetAsync(xs, 0, sizeof(float4) * v32, s));
  WD_CK(cudaMemcpyAsync(r64, R0, sizeof(double2) * nrhs * n, cudaMemcpyDeviceToDevice, s));
  RET_IF(ok(launch_norms(B, r64, part_b, n, nrhs, s), "norms"));
  RET_IF(ok(launch_bicg_finalize(FIN_INIT, part_b, nb64, sc, status, nullptr, 0, nrhs, s), "fin_init"));
  // r32 = r64 for every system, r_hat = r, p = v = 0
  RET_IF(ok(launch_f64_to_f32(r64, r, V, nrhs, nullptr, nullptr, nullptr, M_ALL, s), "to_f32"));
  const unsigned M_LIVE = M_RESTART | M_RECURSIVE;
  if (half)
    RET_IF(ok(launch_bicg16_restart(rhat, r, p16, v16, status, M_LIVE, V, nrhs, s), "restart16"));
  else
    RET_IF(ok(launch_bicg32_restart(rhat, r, p, v, status, M_LIVE, n4, nrhs, s), "restart32"));
  // a system whose initial residual already meets tol is checked like any other
  RET_IF(ok(launch_f64_to_f32(r64, r, V, nrhs, rhat, part_c, status, M_RECURSIVE, s), "to_f32"));
  RET_IF(ok(launch_reliable_finalize(part_c, nbc, sc, status, M_RECURSIVE, nrhs, s), "reliable0"));
  RET_IF(ok(launch_bicg_finalize(FIN_ACTIVATE, nullptr, 0, sc, status, nullptr, 0, nrhs, s), "activate"));
  if (restart) RET_IF(ok(launch_mixed_inner_tol(sc, status, nrhs, s), "inner_tol"));

  // restarted refinement checks every `reliable_every` iterations whether a
  // system reached its inner target and forces a restart after mixed_inner_max
  const int every = restart ? h->mixed_inner_max : reliable_every;
  const int chunk = reliable_every < 10 ? (reliable_every < 1 ? 1 : reliable_every) : 10;
  auto enqueue_chunk = [&]() -> int {
    for (int it = 0; it < chunk; ++it) {
      if (half) {
        RET_IF(ok(launch_bicg16_update_p(p16, r, v16, sc, status, V, nrhs, s), "update_p16"));
        RET_IF(ok(launch_wilson_f16(h, h->links16, p16, nullptr, v16, nrhs, 0, EPI_DOT, sc, rhat, part_w, status, M_ACTIVE, s), "w16_dot"));
      } else {
        RET_IF(ok(launch_bicg32_update_p(p, r, v, sc, status, n4, nrhs, s), "update_p32"));
        if (eo)
          RET_IF(ok(launch_schur_f32(m, p, nullptr, v, tmp_o, nrhs, 0, EPI_DOT, sc, rhat, part_w, status, M_ACTIVE, s), "s32_dot"));
        else
          RET_IF(ok(launch_wilson_f32(m, p, nullptr, v, nrhs, 0, EPI_DOT, sc, rhat, part_w, status, M_ACTIVE, s), "w32_dot"));
      }
      RET_IF(ok(launch_bicg_finalize(FIN_ALPHA, part_w, nbw, sc, status, nullptr, 0, nrhs, s), "fin_alpha"));
      if (half)
        RET_IF(ok(launch_wilson_f16(h, h->links16, v16, r, t16, nrhs, 0, EPI_TSTT, sc, nullptr, part_w, status, M_ACTIVE, s), "w16_tstt"));
      else if (eo)
        RET_IF(ok(launch_schur_f32(m, r, v, t, tmp_o, nrhs, 0, EPI_TSTT, sc, nullptr, part_w, status, M_ACTIVE, s), "s32_tstt"));
      else
        RET_IF(ok(launch_wilson_f32(m, r, v, t, nrhs, 0, EPI_TSTT, sc, nullptr, part_w, status, M_ACTIVE, s), "w32_tstt"));
      RET_IF(ok(launch_bicg_finalize(FIN_OMEGA, part_w, nbw, sc, status, nullptr, 0, nrhs, s), "fin_omega"));
      if (half)
        RET_IF(ok(launch_bicg16_update_xr(xs, r, p16, v16, t16, rhat, sc, status, part_s, V, nrhs, s), "update_xr16"));
      else
        RET_IF(ok(launch_bicg32_update_xr(xs, r, p, v, t, rhat, sc, status, part_s, n4, nrhs, s), "update_xr32"));
      RET_IF(ok(launch_bicg_finalize(FIN_RHO, part_s, nbs, sc, status, nullptr, 0, nrhs, s), "fin_rho"));
    }
    return WD_OK;
  };
  // graphs are skipped while kernel timing is on (events cannot be replayed)
  Profiler *prof = current_profiler();
  // and on the legacy default stream, which cannot be captured
  const bool use_graph = (prof == nullptr || prof->mask == 0) && s != nullptr;
  GraphGuard graph;
  if (use_graph) {
    WD_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_chunk();
    cudaError_t e = cudaStreamEndCapture(s, &graph.g);
    if (rc != WD_OK) return rc;
    WD_CK(e);
    WD_CK(cudaGraphInstantiate(&graph.x, graph.g, 0));
  }

  std::vector<int> hst(nrhs);
  const unsigned M_RU = M_ACTIVE | M_RECURSIVE;
  int since = 0;
  long long guard = 0;
  for (;;) {
    if (++guard > (long long)max_iter / chunk + 64) break;
    if (use_graph) {
      WD_CK(cudaGraphLaunch(graph.x, s));
    } else {
      RET_IF(enqueue_chunk());
    }
    since += chunk;
    WD_CK(cudaMemcpyAsync(hst.data(), status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    WD_CK(cudaStreamSynchronize(s));
    bool active = false, recursive = false;
    for (int q : hst) {
      active |= q == ST_ACTIVE;
      recursive |= q == ST_RECURSIVE;
    }
    if (!active && !recursive) break;
    const bool due = since >= every;
    if (recursive || !active || due) {
      // reliable update: x += xs, r = b - A x in FP64, r32 = r
      RET_IF(ok(launch_add_f32_to_f64(X, xs, V, nrhs, status, M_RU, s), "x += xs"));
      RET_IF(ok(launch_wilson_f64_epi(h, X, tmp64, nrhs, 0, EPI_NONE, nullptr, nullptr, status, s, M_RU), "w64"));
      RET_IF(ok(launch_sub_norm(r64, B, tmp64, status, M_RU, part_b, n, nrhs, s), "r64"));
      RET_IF(ok(launch_f64_to_f32(r64, r, V, nrhs, rhat, part_c, status, M_RU, s), "r32"));
      RET_IF(ok(launch_reliable_finalize(part_c, nbc, sc, status, M_RU, nrhs, s, restart && due ? 1 : 0), "reliable"));
      if (!restart || due) since = 0;
      WD_CK(cudaMemcpyAsync(hst.data(), status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
      WD_CK(cudaStreamSynchronize(s));
      bool left = false, restarted = false;
      for (int q : hst) {
        left |= q == ST_ACTIVE || q == ST_RESTART;
        restarted |= q == ST_RESTART;
      }
      if (restarted) {  // restarted refinement: r_hat = r, p = v = 0, then active again
        if (half)
          RET_IF(ok(launch_bicg16_restart(rhat, r, p16, v16, status, M_RESTART, V, nrhs, s), "restart16"));
        else
          RET_IF(ok(launch_bicg32_restart(rhat, r, p, v, status, M_RESTART, n4, nrhs, s), "restart32"));
        RET_IF(ok(launch_bicg_finalize(FIN_ACTIVATE, nullptr, 0, sc, status, nullptr, 0, nrhs, s), "activate"));
      }
      if (!left) break;
    }
  }
  // systems stopped by breakdown or the iteration cap: fold in xs, record the residual
  const unsigned M_FINAL = (1u << ST_BREAKDOWN) | (1u << ST_MAXITER);
  RET_IF(ok(launch_add_f32_to_f64(X, xs, V, nrhs, status, M_FINAL, s), "x += xs"));
  RET_IF(ok(launch_wilson_f64_epi(h, X, tmp64, nrhs, 0, EPI_NONE, nullptr, nullptr, status, s, M_FINAL), "w64"));
  RET_IF(ok(launch_sub_norm(r64, B, tmp64, status, M_FINAL, part_b, n, nrhs, s), "r64"));
  RET_IF(ok(launch_f64_to_f32(r64, r, V, nrhs, rhat, part_c, status, M_FINAL, s), "r32"));
  RET_IF(ok(launch_reliable_finalize(part_c, nbc, sc, status, M_FINAL, nrhs, s), "reliable"));

  WD_CK(cudaMemcpyAsync(hsc.data(), sc, sizeof(BicgScalars) * nrhs, cudaMemcpyDeviceToHost, s));
  WD_CK(cudaMemcpyAsync(hst.data(), status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  int rc = WD_OK;
  for (int q = 0; q < nrhs; ++q) {
    const BicgScalars &S = hsc[q];
    if (stats) {
      wd_stats &o = stats[q];
      o.mvp = S.mvp;
      o.mvp_extra += S.mvp_extra;
      o.iters = S.iters;
      o.restarts = S.restarts;
      o.converged = hst[q] == ST_DONE ? 1 : 0;
      o.breakdown = hst[q] == ST_BREAKDOWN ? 1 : 0;
      o.rel_res = S.bnorm > 0 ? S.rnorm / S.bnorm : 0.0;
      o.true_rel_res = S.true_rel;
    }
    if (hst[q] == ST_BREAKDOWN) rc = rc == WD_OK ? WD_BREAKDOWN : rc;
    else if (hst[q] != ST_DONE && rc == WD_OK) rc = WD_NOT_CONVERGED;
  }
  if (rc == WD_BREAKDOWN) set_error("mixed BiCGStab breakdown");
  if (rc == WD_NOT_CONVERGED) set_error("mixed BiCGStab did not reach the tolerance within max_iter");
  return rc;
}

}  // namespace wd
