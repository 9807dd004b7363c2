// Host-side drivers of the FP64 solvers.  Every vector operation, reduction
// and small dense step runs in the kernels of dslash.cu, blas.cu and
// dense.cu; the host only sequences launches on one stream and reads a
// status word every few iterations (BiCGStab) or once per cycle (GMRES-DR).
//
//  bicgstab_batched   BiCGStab for nrhs systems in lockstep, each with its
//                     own device-resident scalars and convergence status.
//  deflation_build    W = A V, G = U^dagger A V, LU(G)         (Sec. 2)
//  deflate_batched    y = G^{-1} U^dagger r0, x0 += V y, r0 -= W y (Sec. 2)
//  gmresdr_run        GMRES-DR(m,k)                        (Sec. 1, Sec. 3)
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "solvers.h"
#include "wd_internal.h"

namespace wd {

namespace {

constexpr int CHUNK = 8;  // BiCGStab iterations between host status checks

#define RET_IF(call)                   \
  do {                                 \
    int rc_ = (call);                  \
    if (rc_ != WD_OK) return rc_;      \
  } while (0)

int launch_ok(cudaError_t e, const char *what) {
  if (e != cudaSuccess) return cuda_fail(e, what);
  return WD_OK;
}

}  // namespace

// --------------------------------------------------------------------- BiCGStab

int bicgstab_batched(wd_context *h, const double2 *B, double2 *X, const double2 *R0,
                     int nrhs, double tol, int max_iter, wd_stats *stats, cudaStream_t s,
                     double *hist_host, int hist_len, Arena &ar) {
  const long long n = op_n(h);
  const int nbs = stream_blocks(n), nbw = wilson_blocks(h);
  const size_t vec = (size_t)nrhs * n;
  double2 *r = ar.take<double2>(vec), *rhat = ar.take<double2>(vec);
  double2 *p = ar.take<double2>(vec), *v = ar.take<double2>(vec);
  double2 *sv = ar.take<double2>(vec), *t = ar.take<double2>(vec);
  double *part_s = ar.take<double>((size_t)nrhs * nbs * 3);
  double *part_w = ar.take<double>((size_t)nrhs * nbw * 3);
  BicgScalars *sc = ar.take<BicgScalars>(nrhs);
  int *status = ar.take<int>(nrhs);
  double *hist = hist_len > 0 ? ar.take<double>((size_t)nrhs * hist_len) : nullptr;
  if (ar.failed) return WD_OUT_OF_MEMORY;

  std::vector<BicgScalars> hsc(nrhs);
  for (auto &q : hsc) {
    std::memset(&q, 0, sizeof(q));
    q.tol = tol;
    q.max_iter = max_iter;
    q.max_restarts = 3;
  }
  WD_CK(cudaMemcpyAsync(sc, hsc.data(), sizeof(BicgScalars) * nrhs, cudaMemcpyHostToDevice, s));
  if (hist) WD_CK(cudaMemsetAsync(hist, 0, sizeof(double) * nrhs * hist_len, s));

  // r0 and the norms ||b||, ||r0||
  if (R0 != nullptr) {
    WD_CK(cudaMemcpyAsync(r, R0, sizeof(double2) * vec, cudaMemcpyDeviceToDevice, s));
  } else {
    RET_IF(launch_ok(launch_wilson_f64_epi(h, X, t, nrhs, 0, EPI_NONE, nullptr, nullptr, nullptr, s, M_ALL), "wilson"));
    RET_IF(launch_ok(launch_sub_norm(r, B, t, nullptr, M_ALL, part_s, n, nrhs, s), "sub_norm"));
  }
  RET_IF(launch_ok(launch_norms(B, r, part_s, n, nrhs, s), "norms"));
  WD_CK(cudaMemsetAsync(status, 0, sizeof(int) * nrhs, s));
  RET_IF(launch_ok(launch_bicg_finalize(FIN_INIT, part_s, nbs, sc, status, hist, hist_len, nrhs, s), "fin_init"));
  RET_IF(launch_ok(launch_bicg_restart_vectors(rhat, r, p, v, status, M_RESTART, n, nrhs, s), "restart"));
  RET_IF(launch_ok(launch_bicg_finalize(FIN_ACTIVATE, nullptr, 0, sc, status, nullptr, 0, nrhs, s), "activate"));

  std::vector<int> hst(nrhs);
  const unsigned M_FINAL_CHECK = (1u << ST_BREAKDOWN) | (1u << ST_MAXITER);
  long long guard = 0;
  for (;;) {
    if (++guard > (long long)max_iter + 64) break;  // every pass does >= 1 iteration
    for (int it = 0; it < CHUNK; ++it) {
      RET_IF(launch_ok(launch_bicg_update_p(p, r, v, sc, status, n, nrhs, s), "update_p"));
      RET_IF(launch_ok(launch_wilson_f64_epi(h, p, v, nrhs, 0, EPI_DOT, rhat, part_w, status, s, M_ACTIVE), "wilson_dot"));
      RET_IF(launch_ok(launch_bicg_finalize(FIN_ALPHA, part_w, nbw, sc, status, hist, hist_len, nrhs, s), "fin_alpha"));
      RET_IF(launch_ok(launch_bicg_update_s(sv, r, v, sc, status, n, nrhs, s), "update_s"));
      RET_IF(launch_ok(launch_wilson_f64_epi(h, sv, t, nrhs, 0, EPI_TSTT, nullptr, part_w, status, s, M_ACTIVE), "wilson_tstt"));
      RET_IF(launch_ok(launch_bicg_finalize(FIN_OMEGA, part_w, nbw, sc, status, hist, hist_len, nrhs, s), "fin_omega"));
      RET_IF(launch_ok(launch_bicg_update_xr(X, r, p, sv, t, rhat, sc, status, part_s, n, nrhs, s), "update_xr"));
      RET_IF(launch_ok(launch_bicg_finalize(FIN_RHO, part_s, nbs, sc, status, hist, hist_len, nrhs, s), "fin_rho"));
    }
    WD_CK(cudaMemcpyAsync(hst.data(), status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    WD_CK(cudaStreamSynchronize(s));
    bool active = false, recursive = false;
    for (int q : hst) {
      active |= q == ST_ACTIVE;
      recursive |= q == ST_RECURSIVE;
    }
    if (active) continue;
    if (!recursive) break;
    // true residual r = b - A x for the systems whose recursive residual converged
    RET_IF(launch_ok(launch_wilson_f64_epi(h, X, t, nrhs, 0, EPI_NONE, nullptr, nullptr, status, s, M_RECURSIVE), "wilson_true"));
    RET_IF(launch_ok(launch_sub_norm(r, B, t, status, M_RECURSIVE, part_s, n, nrhs, s), "sub_norm_true"));
    RET_IF(launch_ok(launch_bicg_finalize(FIN_TRUE, part_s, nbs, sc, status, hist, hist_len, nrhs, s), "fin_true"));
    RET_IF(launch_ok(launch_bicg_restart_vectors(rhat, r, p, v, status, M_RESTART, n, nrhs, s), "restart"));
    RET_IF(launch_ok(launch_bicg_finalize(FIN_ACTIVATE, nullptr, 0, sc, status, nullptr, 0, nrhs, s), "activate"));
  }
  // true residual of systems that stopped on breakdown or the iteration cap
  RET_IF(launch_ok(launch_wilson_f64_epi(h, X, t, nrhs, 0, EPI_NONE, nullptr, nullptr, status, s, M_FINAL_CHECK), "wilson_final"));
  RET_IF(launch_ok(launch_sub_norm(sv, B, t, status, M_FINAL_CHECK, part_s, n, nrhs, s), "sub_norm_final"));
  RET_IF(launch_ok(launch_bicg_finalize(FIN_TRUE, part_s, nbs, sc, status, hist, hist_len, nrhs, s), "fin_final"));

  WD_CK(cudaMemcpyAsync(hsc.data(), sc, sizeof(BicgScalars) * nrhs, cudaMemcpyDeviceToHost, s));
  WD_CK(cudaMemcpyAsync(hst.data(), status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
  if (hist_host && hist) WD_CK(cudaMemcpyAsync(hist_host, hist, sizeof(double) * nrhs * hist_len, cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  int rc = WD_OK;
  for (int q = 0; q < nrhs; ++q) {
    const BicgScalars &S = hsc[q];
    const int st = hst[q];
    if (stats) {
      wd_stats &o = stats[q];
      o.mvp = S.mvp;
      o.mvp_extra += S.mvp_extra;
      o.iters = S.iters;
      o.restarts = S.restarts;
      o.converged = st == ST_DONE ? 1 : 0;
      o.breakdown = st == ST_BREAKDOWN ? 1 : 0;
      o.rel_res = S.bnorm > 0 ? S.rnorm / S.bnorm : 0.0;
      o.true_rel_res = S.true_rel;
    }
    if (st == ST_BREAKDOWN) rc = rc == WD_OK ? WD_BREAKDOWN : rc;
    else if (st != ST_DONE && rc == WD_OK) rc = WD_NOT_CONVERGED;
  }
  if (rc == WD_BREAKDOWN) set_error("BiCGStab breakdown: <r_hat, r> or <r_hat, v> vanished");
  if (rc == WD_NOT_CONVERGED) set_error("BiCGStab did not reach the tolerance within max_iter / 3 restarts");
  return rc;
}

// --------------------------------------------------------------------- deflation (Sec. 2)

int deflation_build(wd_deflation_space *d, cudaStream_t s, Arena &ar) {
  wd_context *h = d->h;
  const long long n = op_n(h);
  const int k = d->k;
  // W = A V: k MVPs, batched as k right-hand sides
  RET_IF(launch_ok(launch_wilson_f64(h, d->V, d->W, k, 0, s), "wilson(V)"));
  // G = U^dagger W, in column groups of 16
  const double2 *Uop = d->U ? d->U : d->V;
  const int g5 = d->U ? 0 : 1;
  double2 *part = ar.take<double2>(ts_dot_partial_count(n, k, 16));
  double *info = ar.take<double>(2);
  if (ar.failed) return WD_OUT_OF_MEMORY;
  for (int j0 = 0; j0 < k; j0 += 16) {
    const int nc = k - j0 < 16 ? k - j0 : 16;
    RET_IF(launch_ok(launch_ts_dot(Uop, k, d->W + (size_t)j0 * n, nc, g5, n, part, nullptr, s), "ts_dot(G)"));
    RET_IF(launch_ok(launch_ts_dot_finalize(part, n, k, nc, d->LU + j0, k, nullptr, 0, nullptr, s), "ts_fin(G)"));
  }
  RET_IF(launch_ok(launch_lu_factor(d->LU, k, d->piv, info, s), "lu_factor"));
  double hinfo[2];
  WD_CK(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  if (hinfo[0] != 0.0 || hinfo[1] > 1e14) {
    set_error("projected matrix U^dagger A V is numerically singular (pivot ratio " +
              std::to_string(hinfo[1]) + ")");
    return WD_SINGULAR_PROJECTION;
  }
  return WD_OK;
}

// OUT = (beta_one ? IN : 0) + sign V Y: on the tensor cores (exact-split
// emulation) when the handle allows it and the product is wide (ncol >= 8),
// else by FP64 FMAs.  scratch (ts_update_tc_scratch_bytes) and err (device
// int, set on a tensor-core wait that gave up) may be NULL for the FP64 form.
static cudaError_t wide_update(const wd_context *h, const double2 *V, int kv, const double2 *Y,
                               int ldy, int ncol, const double2 *IN, double2 *OUT, int beta_one,
                               double sign, long long n, void *scratch, int *err, cudaStream_t s) {
  if (h->tc_contract && scratch != nullptr && err != nullptr && ncol >= 8 &&
      ts_update_tc_supported(kv, ncol))
    return launch_ts_update_tc(V, kv, Y, ldy, ncol, IN, OUT, beta_one, sign, n, scratch, err, s);
  return launch_ts_update(V, kv, Y, ldy, ncol, IN, OUT, beta_one, sign, n, nullptr, s);
}

static int tc_error_check(int *err, cudaStream_t s) {
  int herr = 0;
  WD_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  if (herr != 0) {
    set_error("tensor-core contraction: a wait in the kernel gave up");
    return WD_TIMEOUT;
  }
  return WD_OK;
}

int deflate_batched(wd_deflation_space *d, double2 *X, double2 *R0, int nrhs, cudaStream_t s,
                    Arena &ar) {
  const long long n = op_n(d->h);
  const int k = d->k;
  const double2 *Uop = d->U ? d->U : d->V;
  const int g5 = d->U ? 0 : 1;
  int *tc_err = ar.take<int>(1);
  if (ar.failed) return WD_OUT_OF_MEMORY;
  WD_CK(cudaMemsetAsync(tc_err, 0, sizeof(int), s));
  bool used_tc = false;
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int nc = nrhs - r0 < 16 ? nrhs - r0 : 16;
    double2 *part = ar.take<double2>(ts_dot_partial_count(n, k, nc));
    double2 *C = ar.take<double2>((size_t)k * nc);
    unsigned char *tcs = d->h->tc_contract && nc >= 8 && ts_update_tc_supported(k, nc)
                             ? ar.take<unsigned char>(ts_update_tc_scratch_bytes(k, nc, n))
                             : nullptr;
    used_tc |= tcs != nullptr;
    if (ar.failed) return WD_OUT_OF_MEMORY;
    double2 *Xg = X + (size_t)r0 * n, *Rg = R0 + (size_t)r0 * n;
    // c = U^dagger r0 (= V^dagger gamma5 r0 when U = gamma5 V)
    RET_IF(launch_ok(launch_ts_dot(Uop, k, Rg, nc, g5, n, part, nullptr, s), "ts_dot(c)"));
    RET_IF(launch_ok(launch_ts_dot_finalize(part, n, k, nc, C, nc, nullptr, 0, nullptr, s), "ts_fin(c)"));
    // y = G^{-1} c
    RET_IF(launch_ok(launch_lu_solve(d->LU, d->piv, k, C, nc, s), "lu_solve"));
    // x0 += V y ; r0 -= W y  (W = A V, so r0 = b - A x0 stays exact)
    RET_IF(launch_ok(wide_update(d->h, d->V, k, C, nc, nc, Xg, Xg, 1, 1.0, n, tcs, tc_err, s), "update(x)"));
    RET_IF(launch_ok(wide_update(d->h, d->W, k, C, nc, nc, Rg, Rg, 1, -1.0, n, tcs, tc_err, s), "update(r)"));
  }
  return used_tc ? tc_error_check(tc_err, s) : WD_OK;
}

// --------------------------------------------------------------------- GMRES-DR

int gmresdr_run(wd_context *h, const double2 *b, double2 *x, int m, int k, double tol,
                int max_mv, double2 *V_out, double2 *Hbar_host, double2 *theta_host,
                wd_stats *stats, cudaStream_t s, double *hist_host, int hist_len, Arena &ar) {
  h->gmresdr_hist.clear();
  const long long n = op_n(h);
  const int nbs = stream_blocks(n), nbw = wilson_blocks(h);
  double2 *Va = ar.take<double2>((size_t)(m + 1) * n);
  double2 *Vb = ar.take<double2>((size_t)(m + 1) * n);
  double2 *w = ar.take<double2>(n);
  double2 *r = ar.take<double2>(n);
  size_t npart = 0;
  for (int j = 1; j <= m + 1; ++j) npart = std::max(npart, ts_dot_partial_count(n, j, 1));
  double2 *part_t = ar.take<double2>(npart);
  // the basis as FP32 pairs (high and low planes) for the double-float dot
  // and the FP32 correction
  float2 *Vsh = ar.take<float2>((size_t)2 * (m + 1) * n);
  float2 *Vsl = Vsh == nullptr ? nullptr : Vsh + (size_t)(m + 1) * n;
  double *part_w = ar.take<double>((size_t)nbw * 3);
  double *part_n = ar.take<double>((size_t)nbs * 2);
  double2 *H = ar.take<double2>((size_t)(m + 1) * m);
  double2 *c = ar.take<double2>(m + 1);
  double2 *h2 = ar.take<double2>(m + 1);
  double2 *d = ar.take<double2>(m);
  double2 *rho = ar.take<double2>(m + 1);
  double *res = ar.take<double>(1);
  double2 *P = ar.take<double2>((size_t)(m + 1) * (k + 1));
  double2 *Hk = ar.take<double2>((size_t)(k + 1) * (k > 0 ? k : 1));
  double2 *ck = ar.take<double2>(k + 1);
  double2 *theta = ar.take<double2>(k > 0 ? k : 1);
  double2 *scal = ar.take<double2>(2);
  int *flags = ar.take<int>(3);
  int *status = ar.take<int>(1);
  int *m_eff = ar.take<int>(1);
  double2 *work = ar.take<double2>((size_t)2 * (m + 1) * (m + 1) + (size_t)2 * m * m + 4 * m + 2);
  // WD_TRACE_DENSE=1 prints the SM-clock split of every cycle-end kernel
  const bool trace_dense = std::getenv("WD_TRACE_DENSE") != nullptr;
  long long *clk = trace_dense ? ar.take<long long>(13) : nullptr;
  const bool tc_restart = h->tc_contract && k + 1 >= 8 && ts_update_tc_supported(m + 1, k + 1);
  unsigned char *tc_scratch =
      tc_restart ? ar.take<unsigned char>(ts_update_tc_scratch_bytes(m + 1, k + 1, n)) : nullptr;
  int *tc_err = ar.take<int>(1);
  if (ar.failed) return WD_OUT_OF_MEMORY;
  WD_CK(cudaMemsetAsync(tc_err, 0, sizeof(int), s));

  long long mvp = 0, mvp_extra = 0;
  // initial residual (x0 = 0 needs no product)
  RET_IF(launch_ok(launch_norms(x, nullptr, part_n, n, 1, s), "norms(x)"));
  RET_IF(launch_ok(launch_norm_finalize(part_n, nbs, 2, scal, s), "norm(x)"));
  double2 hx;
  WD_CK(cudaMemcpyAsync(&hx, scal, sizeof(hx), cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  if (hx.x == 0.0) {
    WD_CK(cudaMemcpyAsync(r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    RET_IF(launch_ok(launch_wilson_f64(h, x, w, 1, 0, s), "wilson(x0)"));
    RET_IF(launch_ok(launch_sub_norm(r, b, w, nullptr, M_ALL, part_n, n, 1, s), "r0"));
    mvp_extra += 1;
  }
  RET_IF(launch_ok(launch_norms(r, nullptr, part_n, n, 1, s), "norms(r0)"));
  WD_CK(cudaMemsetAsync(c, 0, sizeof(double2) * (m + 1), s));
  RET_IF(launch_ok(launch_norm_finalize(part_n, nbs, 2, c, s), "beta"));
  double2 hb;
  WD_CK(cudaMemcpyAsync(&hb, c, sizeof(hb), cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  const double bnorm0 = hb.x;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (bnorm0 == 0.0) {
    if (stats) stats->converged = 1;
    if (V_out && k > 0) WD_CK(cudaMemsetAsync(V_out, 0, sizeof(double2) * k * n, s));
    WD_CK(cudaStreamSynchronize(s));
    return WD_OK;
  }
  WD_CK(cudaMemsetAsync(H, 0, sizeof(double2) * (m + 1) * m, s));
  RET_IF(launch_ok(launch_scale_by_inverse_entry(Va, r, c, 0, n, nullptr, s), "v1"));
  RET_IF(launch_ok(launch_split_df(Va, Vsh, Vsl, n, nullptr, s), "v1 split"));

  double2 *V = Va, *Vn = Vb;
  int j0 = 0, cycles = 0, rc = WD_NOT_CONVERGED;
  const int zero = 0;
  double last_rel = 1.0;
  std::vector<double> hist;
  for (;;) {
    WD_CK(cudaMemcpyAsync(status, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    WD_CK(cudaMemcpyAsync(m_eff, &m, sizeof(int), cudaMemcpyHostToDevice, s));
    for (int j = j0; j < m; ++j) {
      double2 *vj = V + (size_t)j * n;
      // w = A v_j, with ||w||^2 fused (lucky-breakdown reference)
      RET_IF(launch_ok(launch_wilson_f64_epi(h, vj, w, 1, 0, EPI_TSTT, nullptr, part_w, status, s, M_ACTIVE), "arnoldi wilson"));
      // classical Gram-Schmidt, applied twice: the first pass's coefficients
      // in double-float (~48 bits, FP32 pipe), the second pass's in FP64 (it
      // removes what the first left, so H = h1 + h2 is exact to FP64
      // rounding), its update in FP32 when h2 is at rounding level
      RET_IF(launch_ok(launch_ts_dot_df(Vsh, Vsl, j + 1, w, n, part_t, status, s), "cgs dot1"));
      RET_IF(launch_ok(launch_ts_dot_df_finalize(part_t, n, j + 1, H + j, m, status, s), "cgs fin1"));
      RET_IF(launch_ok(launch_ts_update(V, j + 1, H + j, m, 1, w, w, 1, -1.0, n, status, s), "cgs upd1"));
      RET_IF(launch_ok(launch_ts_dot(V, j + 1, w, 1, 0, n, part_t, status, s), "cgs dot2"));
      RET_IF(launch_ok(launch_ts_dot_finalize(part_t, n, j + 1, 1, h2, 1, H + j, m, status, s), "cgs fin2"));
      RET_IF(launch_ok(launch_ts_update_correction(V, Vsh, j + 1, h2, H + j, m, part_w, nbw, w, n, status, s), "cgs upd2"));
      // h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
      RET_IF(launch_ok(launch_norms(w, nullptr, part_n, n, 1, s), "norm w"));
      RET_IF(launch_ok(launch_arnoldi_normalize_finalize(part_n, nbs, part_w, nbw, H, m, j, 1e-14, status, m_eff, s), "arnoldi fin"));
      RET_IF(launch_ok(launch_scale_by_inverse_entry(V + (size_t)(j + 1) * n, w, H, (j + 1) * m + j, n, status, s), "arnoldi scale"));
      RET_IF(launch_ok(launch_split_df(V + (size_t)(j + 1) * n, Vsh + (size_t)(j + 1) * n, Vsl + (size_t)(j + 1) * n, n, status, s), "arnoldi split"));
    }
    cycles += 1;
    CycleEndArgs a;
    a.H = H; a.c = c; a.m = m; a.k = k; a.m_eff = m_eff; a.d = d; a.rho = rho; a.res = res;
    a.P = P; a.Hk = Hk; a.ck = ck; a.theta = theta; a.flags = flags; a.work = work;
    a.do_restart = 1;
    a.eig32 = h->eig32;
    a.clk = clk;
    RET_IF(launch_ok(launch_gmresdr_cycle_end(a, s), "cycle_end"));
    if (clk) {
      long long hc[13] = {0};
      WD_CK(cudaMemcpyAsync(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost, s));
      WD_CK(cudaStreamSynchronize(s));
      std::fprintf(stderr,
                   "cycle_end clk: lsq %lld f %lld hessenberg32 %lld qr32 %lld refine %lld "
                   "qr(P) %lld products %lld | qr32 sweeps %lld rotations %lld fp64 fallback %lld\n",
                   hc[1] - hc[0], hc[2] - hc[1], hc[7] - hc[2], hc[3] - hc[7], hc[4] - hc[3],
                   hc[5] - hc[4], hc[6] - hc[5], hc[8], hc[9], hc[12]);
    }
    int hflags[2], hme;
    double hres;
    WD_CK(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    WD_CK(cudaMemcpyAsync(&hme, m_eff, sizeof(int), cudaMemcpyDeviceToHost, s));
    WD_CK(cudaMemcpyAsync(&hres, res, sizeof(double), cudaMemcpyDeviceToHost, s));
    WD_CK(cudaStreamSynchronize(s));
    mvp += hme - j0;
    // x += V_m d
    RET_IF(launch_ok(launch_ts_update(V, hme, d, 1, 1, x, x, 1, 1.0, n, nullptr, s), "x update"));
    last_rel = hres / bnorm0;
    hist.push_back(last_rel);
    if (hflags[0] != 0) {
      set_error("GMRES-DR restart: harmonic Ritz eigenproblem failed (flag " +
                std::to_string(hflags[0]) + ")");
      rc = WD_BREAKDOWN;
      break;
    }
    const bool lucky = hflags[1] != 0;
    const bool done = lucky || last_rel <= tol;
    if (!lucky) {
      // V_{k+1} = V_{m+1} P_{k+1} (also after the last cycle, to emit V)
      RET_IF(launch_ok(wide_update(h, V, m + 1, P, k + 1, k + 1, nullptr, Vn, 0, 1.0, n, tc_scratch, tc_err, s), "restart combine"));
      std::swap(V, Vn);
    }
    if (done) {
      rc = WD_OK;
      break;
    }
    if (mvp + (m - k) > max_mv) {
      set_error("GMRES-DR: MVP budget exhausted before the tolerance was met");
      rc = WD_NOT_CONVERGED;
      break;
    }
    // Hbar <- [Hbar_k; 0], c <- [P^dagger rho; 0]
    WD_CK(cudaMemsetAsync(H, 0, sizeof(double2) * (m + 1) * m, s));
    WD_CK(cudaMemsetAsync(c, 0, sizeof(double2) * (m + 1), s));
    if (k > 0)
      WD_CK(cudaMemcpy2DAsync(H, sizeof(double2) * m, Hk, sizeof(double2) * k, sizeof(double2) * k,
                              k + 1, cudaMemcpyDeviceToDevice, s));
    WD_CK(cudaMemcpyAsync(c, ck, sizeof(double2) * (k + 1), cudaMemcpyDeviceToDevice, s));
    if (k > 0) {
      // re-orthogonalise v_{k+1} against v_1..v_k
      double2 *vk = V + (size_t)k * n;
      RET_IF(launch_ok(launch_ts_dot(V, k, vk, 1, 0, n, part_t, nullptr, s), "reorth dot"));
      RET_IF(launch_ok(launch_ts_dot_finalize(part_t, n, k, 1, h2, 1, nullptr, 0, nullptr, s), "reorth fin"));
      RET_IF(launch_ok(launch_ts_update(V, k, h2, 1, 1, vk, vk, 1, -1.0, n, nullptr, s), "reorth upd"));
      RET_IF(launch_ok(launch_norms(vk, nullptr, part_n, n, 1, s), "reorth norm"));
      RET_IF(launch_ok(launch_norm_finalize(part_n, nbs, 2, scal, s), "reorth nrm"));
      RET_IF(launch_ok(launch_scale_by_inverse_entry(vk, vk, scal, 0, n, nullptr, s), "reorth scale"));
    }
    // the restarted basis v_1 .. v_{k+1} in split form
    RET_IF(launch_ok(launch_split_df(V, Vsh, Vsl, (long long)(k + 1) * n, nullptr, s), "restart split"));
    j0 = k;
  }
  // outputs
  if (V_out && k > 0) WD_CK(cudaMemcpyAsync(V_out, V, sizeof(double2) * k * n, cudaMemcpyDeviceToDevice, s));
  if (Hbar_host && k > 0) WD_CK(cudaMemcpyAsync(Hbar_host, Hk, sizeof(double2) * (k + 1) * k, cudaMemcpyDeviceToHost, s));
  if (theta_host && k > 0) WD_CK(cudaMemcpyAsync(theta_host, theta, sizeof(double2) * k, cudaMemcpyDeviceToHost, s));
  // true residual
  RET_IF(launch_ok(launch_wilson_f64(h, x, w, 1, 0, s), "wilson(x)"));
  RET_IF(launch_ok(launch_sub_norm(r, b, w, nullptr, M_ALL, part_n, n, 1, s), "true r"));
  RET_IF(launch_ok(launch_norm_finalize(part_n, nbs, 1, scal, s), "true norm"));
  double2 htr;
  WD_CK(cudaMemcpyAsync(&htr, scal, sizeof(htr), cudaMemcpyDeviceToHost, s));
  WD_CK(cudaStreamSynchronize(s));
  mvp_extra += 1;
  if (stats) {
    stats->mvp = mvp;
    stats->mvp_extra = mvp_extra;
    stats->cycles = cycles;
    stats->rel_res = last_rel;
    stats->true_rel_res = htr.x / bnorm0;
    stats->converged = rc == WD_OK ? 1 : 0;
  }
  if (hist_host) {
    for (int i = 0; i < hist_len && i < (int)hist.size(); ++i) hist_host[i] = hist[i];
  }
  h->gmresdr_hist = hist;
  if (tc_restart && (rc == WD_OK || rc == WD_NOT_CONVERGED)) {
    const int trc = tc_error_check(tc_err, s);
    if (trc != WD_OK) return trc;
  }
  return rc;
}

// --------------------------------------------------------------------- Sec. 4 shifts

// Twisted-mass systems A(mu_i) x_i = b solved one shift after another
// (Sec. 4).  Before shift i, every right-hand side is projected over its own
// solutions of shifts 0..i-1: with Q = [x_0 .. x_{i-1}], solve
// Q^dagger A_i^dagger A_i Q d = Q^dagger A_i^dagger b and start from Q d.
//
// One shift: B (nrhs vectors of the handle's operator) and X, the solutions
// of all shifts ([shift][rhs][n]); shift i's slot is written.
namespace {
struct ShiftWork {
  double2 *R0, *Qc, *AQ, *part, *M, *c;
  int *piv;
  double *info;
};
}  // namespace

static int shift_step(wd_context *h, const double2 *B, double2 *X, int i, int nrhs, double tol,
                      int max_iter, int project, int mixed, wd_stats *st, cudaStream_t s,
                      Arena &ar, const ShiftWork &w) {
  const long long n = op_n(h);
  double2 *R0 = w.R0, *Qc = w.Qc, *AQ = w.AQ, *part = w.part, *M = w.M, *c = w.c;
  double2 *Xi = X + (size_t)i * nrhs * n;
  WD_CK(cudaMemcpyAsync(R0, B, sizeof(double2) * nrhs * n, cudaMemcpyDeviceToDevice, s));
  WD_CK(cudaMemsetAsync(Xi, 0, sizeof(double2) * nrhs * n, s));
  if (st) std::memset(st, 0, sizeof(wd_stats) * nrhs);
  if (project && i > 0) {
    for (int r = 0; r < nrhs; ++r) {
      for (int j = 0; j < i; ++j)
        WD_CK(cudaMemcpyAsync(Qc + (size_t)j * n, X + ((size_t)j * nrhs + r) * n,
                              sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
      RET_IF(launch_ok(launch_wilson_f64(h, Qc, AQ, i, 0, s), "A Q"));
      RET_IF(launch_ok(launch_ts_dot(AQ, i, AQ, i, 0, n, part, nullptr, s), "Q^H A^H A Q"));
      RET_IF(launch_ok(launch_ts_dot_finalize(part, n, i, i, M, i, nullptr, 0, nullptr, s), "fin M"));
      RET_IF(launch_ok(launch_ts_dot(AQ, i, B + (size_t)r * n, 1, 0, n, part, nullptr, s), "Q^H A^H b"));
      RET_IF(launch_ok(launch_ts_dot_finalize(part, n, i, 1, c, 1, nullptr, 0, nullptr, s), "fin c"));
      RET_IF(launch_ok(launch_lu_factor(M, i, w.piv, w.info, s), "lu"));
      double hinfo[2];
      WD_CK(cudaMemcpyAsync(hinfo, w.info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
      WD_CK(cudaStreamSynchronize(s));
      if (st) st[r].mvp_extra += i;
      if (hinfo[0] != 0.0 || hinfo[1] > 1e14) continue;  // degenerate Q: start from 0
      RET_IF(launch_ok(launch_lu_solve(M, w.piv, i, c, 1, s), "lu solve"));
      RET_IF(launch_ok(launch_ts_update(Qc, i, c, 1, 1, nullptr, Xi + (size_t)r * n, 0, 1.0, n, nullptr, s), "x0 = Q d"));
      RET_IF(launch_ok(launch_ts_update(AQ, i, c, 1, 1, B + (size_t)r * n, R0 + (size_t)r * n, 1, -1.0, n, nullptr, s), "r0 = b - A Q d"));
    }
  }
  return mixed ? bicgstab_mixed_batched(h, B, Xi, R0, nrhs, tol, max_iter, 50, st, s, ar)
               : bicgstab_batched(h, B, Xi, R0, nrhs, tol, max_iter, st, s, nullptr, 0, ar);
}

// In even-odd mode B and X are full-lattice vectors: each shift's source is
// prepared with that shift's mu, the Schur system is solved (projected over
// the earlier shifts' even-site solutions) and x_i is reconstructed.
int tm_shifts_run(wd_context *h, const double2 *B, double2 *X, int nrhs, const double *mus,
                  int nshift, double tol, int max_iter, int project, int mixed,
                  wd_stats *stats, cudaStream_t s, Arena &ar) {
  const long long n = op_n(h);
  const double mu_saved = h->mu;
  const int kmax = nshift > 1 ? nshift - 1 : 1;
  ShiftWork w;
  w.R0 = ar.take<double2>((size_t)nrhs * n);
  w.Qc = ar.take<double2>((size_t)kmax * n);
  w.AQ = ar.take<double2>((size_t)kmax * n);
  w.part = ar.take<double2>(ts_dot_partial_count(n, kmax, kmax));
  w.M = ar.take<double2>((size_t)kmax * kmax);
  w.c = ar.take<double2>(kmax);
  w.piv = ar.take<int>(kmax);
  w.info = ar.take<double>(2);
  const bool eo = h->eo != 0;
  double2 *Bh = eo ? ar.take<double2>((size_t)nrhs * n) : nullptr;          // b_hat of the shift
  double2 *Xh = eo ? ar.take<double2>((size_t)nshift * nrhs * n) : nullptr; // even solutions
  double2 *be = eo ? ar.take<double2>((size_t)nrhs * n) : nullptr;
  double2 *bo = eo ? ar.take<double2>((size_t)nrhs * n) : nullptr;
  if (ar.failed) return WD_OUT_OF_MEMORY;
  int rc = WD_OK;
  for (int i = 0; i < nshift && rc != WD_CUDA_ERROR && rc != WD_OUT_OF_MEMORY; ++i) {
    h->mu = mus[i];
    wd_stats *st = stats ? stats + (size_t)i * nrhs : nullptr;
    int rci;
    if (eo) {
      RET_IF(launch_ok(launch_eo_prepare(h, B, Bh, be, bo, nrhs, s), "prepare"));
      rci = shift_step(h, Bh, Xh, i, nrhs, tol, max_iter, project, mixed, st, s, ar, w);
      if (rci != WD_CUDA_ERROR && rci != WD_OUT_OF_MEMORY && rci != WD_BAD_ARG)
        RET_IF(launch_ok(launch_eo_reconstruct(h, B, Xh + (size_t)i * nrhs * n,
                                               X + (size_t)i * nrhs * h->n, be, bo, nrhs, s),
                         "reconstruct"));
    } else {
      rci = shift_step(h, B, X, i, nrhs, tol, max_iter, project, mixed, st, s, ar, w);
    }
    if (rci == WD_CUDA_ERROR || rci == WD_OUT_OF_MEMORY || rci == WD_BAD_ARG) rc = rci;
    else if (rci != WD_OK && rc == WD_OK) rc = rci;
  }
  h->mu = mu_saved;
  return rc;
}

}  // namespace wd
