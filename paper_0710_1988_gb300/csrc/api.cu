// C ABI of libwd.so (declared in include/wd.h): argument checks, host-pointer
// staging, handle and deflation-space lifetime, error reporting.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "mixed.h"
#include "solvers.h"
#include "wd_internal.h"

namespace wd {

static thread_local std::string g_last_error;

int bad_alloc();

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? WD_OUT_OF_MEMORY : WD_CUDA_ERROR;
}

bool is_device_pointer(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static thread_local Profiler *g_prof = nullptr;
Profiler *current_profiler() { return g_prof; }
void set_current_profiler(Profiler *p) { g_prof = p; }

cudaEvent_t Profiler::take() {
  if (!spare.empty()) {
    cudaEvent_t e = spare.back();
    spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Profiler::flush() {
  for (const Rec &r : pending) {
    float t = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&t, r.a, r.b);
    launches[r.cat] += 1;
    ms[r.cat] += t;
    spare.push_back(r.a);
    spare.push_back(r.b);
  }
  pending.clear();
}

void Profiler::reset() {
  flush();
  for (int c = 0; c < PC_COUNT; ++c) {
    launches[c] = 0;
    ms[c] = 0.0;
  }
  if (d_sites) cudaMemset(d_sites, 0, 2 * sizeof(unsigned long long));
}

void Profiler::destroy() {
  flush();
  for (cudaEvent_t e : spare) cudaEventDestroy(e);
  spare.clear();
  if (d_sites) cudaFree(d_sites);
  d_sites = nullptr;
}

static int bad(const std::string &msg) {
  set_error(msg);
  return WD_BAD_ARG;
}

// A device view of a "device or host" vector argument.
struct Staged {
  double2 *dev = nullptr;
  const void *user = nullptr;
  bool host = false;
  size_t bytes = 0;
};

static int stage_in(const void *user, size_t bytes, bool copy, Staged &st, Arena &ar,
                    cudaStream_t s) {
  st.user = user;
  st.bytes = bytes;
  st.host = !is_device_pointer(user);
  if (!st.host) {
    st.dev = const_cast<double2 *>(static_cast<const double2 *>(user));
    return WD_OK;
  }
  st.dev = ar.take<double2>(bytes / sizeof(double2));
  if (ar.failed) return bad_alloc();
  if (copy) WD_CK(cudaMemcpyAsync(st.dev, user, bytes, cudaMemcpyHostToDevice, s));
  return WD_OK;
}

}  // namespace wd

namespace wd {
int bad_alloc() {
  set_error("out of device memory for solver scratch");
  return WD_OUT_OF_MEMORY;
}
}  // namespace wd

using namespace wd;

// ------------------------------------------------------------------ handles

extern "C" int wd_create(const int lat[4], const void *links, double kappa, double mu,
                         wd_handle *out) {
  if (out == nullptr) return bad("wd_create: out is NULL");
  *out = nullptr;
  if (lat == nullptr || links == nullptr) return bad("wd_create: lat or links is NULL");
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (lat[i] < 1 || lat[i] > 4096) return bad("wd_create: lattice extents must be in [1, 4096]");
    V *= lat[i];
  }
  if (V * 12 >= (1LL << 40)) return bad("wd_create: lattice too large");
  wd_context *h = new wd_context();
  h->prof.d_sites = nullptr;
  h->links32 = nullptr;
  h->links16 = nullptr;
  h->mixed_bits = 32;
  h->mixed_delta = 0.0;
  h->mixed_inner_max = 300;
  h->side = nullptr;
  h->ev_in = h->ev_out = nullptr;
  h->eo = 0;
  for (int i = 0; i < WD_TUNE_SLOTS; ++i) {
    h->tune_R[i] = h->tune_T[i] = 0;
    h->tune_ms[i] = 0.f;
    h->tune16_R[i] = h->tune16_T[i] = 0;
    h->tune16_ms[i] = 0.f;
  }
  h->eo_tmp = nullptr;
  h->eo_tmp_cap = 0;
  h->tc_contract = 1;
  h->eig32 = 1;
  for (int i = 0; i < 4; ++i) h->dims[i] = lat[i];
  h->V = V;
  h->n = 12 * V;
  h->kappa = kappa;
  h->mu = mu;
  h->links = nullptr;
  h->pool = nullptr;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->links, sizeof(double2) * 36 * V);
  if (e == cudaSuccess) e = cudaMalloc(&h->prof.d_sites, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(h->prof.d_sites, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(h->links, links, sizeof(double2) * 36 * V, cudaMemcpyDefault);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = h->device;
    e = cudaMemPoolCreate(&h->pool, &props);
    if (e == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      e = cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "wd_create");
    if (h->links) cudaFree(h->links);
    if (h->pool) cudaMemPoolDestroy(h->pool);
    h->prof.destroy();
    delete h;
    return rc;
  }
  *out = h;
  return WD_OK;
}

extern "C" int wd_set_operator(wd_handle h, int even_odd) {
  if (h == nullptr) return bad("wd_set_operator: NULL handle");
  if (even_odd && (h->dims[0] % 2 != 0)) return bad("wd_set_operator: even-odd needs an even Lx");
  if (even_odd && (h->dims[1] % 2 || h->dims[2] % 2 || h->dims[3] % 2))
    return bad("wd_set_operator: even-odd needs even extents (periodic parity)");
  h->eo = even_odd ? 1 : 0;
  return WD_OK;
}

extern "C" int wd_eo_prepare(wd_handle h, const void *B, void *Bhat, int nrhs, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr || B == nullptr || Bhat == nullptr) return bad("wd_eo_prepare: NULL argument");
  if (!h->eo) return bad("wd_eo_prepare: the handle is not in even-odd mode");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_eo_prepare: nrhs must be in [1, 65535]");
  if (!is_device_pointer(B) || !is_device_pointer(Bhat)) return bad("wd_eo_prepare: device pointers required");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const size_t half = (size_t)nrhs * (h->n / 2);
  double2 *be = ar.take<double2>(half), *bo = ar.take<double2>(half);
  if (ar.failed) return bad_alloc();
  cudaError_t e = launch_eo_prepare(h, static_cast<const double2 *>(B), static_cast<double2 *>(Bhat),
                                    be, bo, nrhs, s);
  ar.release();
  return e == cudaSuccess ? WD_OK : cuda_fail(e, "wd_eo_prepare");
}

extern "C" int wd_eo_reconstruct(wd_handle h, const void *B, const void *Xe, void *X, int nrhs,
                                 wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr || B == nullptr || Xe == nullptr || X == nullptr) return bad("wd_eo_reconstruct: NULL argument");
  if (!h->eo) return bad("wd_eo_reconstruct: the handle is not in even-odd mode");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_eo_reconstruct: nrhs must be in [1, 65535]");
  if (!is_device_pointer(B) || !is_device_pointer(Xe) || !is_device_pointer(X))
    return bad("wd_eo_reconstruct: device pointers required");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const size_t half = (size_t)nrhs * (h->n / 2);
  double2 *be = ar.take<double2>(half), *bo = ar.take<double2>(half);
  if (ar.failed) return bad_alloc();
  cudaError_t e = launch_eo_reconstruct(h, static_cast<const double2 *>(B), static_cast<const double2 *>(Xe),
                                        static_cast<double2 *>(X), be, bo, nrhs, s);
  ar.release();
  return e == cudaSuccess ? WD_OK : cuda_fail(e, "wd_eo_reconstruct");
}

extern "C" int wd_set_params(wd_handle h, double kappa, double mu) {
  if (h == nullptr) return bad("wd_set_params: NULL handle");
  h->kappa = kappa;
  h->mu = mu;
  return WD_OK;
}

extern "C" void wd_destroy(wd_handle h) {
  if (h == nullptr) return;
  cudaDeviceSynchronize();
  h->prof.destroy();
  if (h->links32) cudaFree(h->links32);
  if (h->links16) cudaFree(h->links16);
  if (h->eo_tmp) cudaFree(h->eo_tmp);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->links) cudaFree(h->links);
  if (h->pool) cudaMemPoolDestroy(h->pool);
  delete h;
}

extern "C" int wd_profile_enable(wd_handle h, unsigned mask) {
  if (h == nullptr) return bad("wd_profile_enable: NULL handle");
  h->prof.reset();
  h->prof.mask = mask & ((1u << PC_COUNT) - 1);
  return WD_OK;
}

extern "C" int wd_profile_read(wd_handle h, wd_profile *out) {
  if (h == nullptr || out == nullptr) return bad("wd_profile_read: NULL argument");
  h->prof.flush();
  for (int c = 0; c < PC_COUNT; ++c) {
    out->launches[c] = h->prof.launches[c];
    out->ms[c] = h->prof.ms[c];
  }
  unsigned long long sites[2] = {0, 0};
  cudaError_t e = cudaMemcpy(sites, h->prof.d_sites, sizeof(sites), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "wd_profile_read");
  out->dslash_site_updates = (long long)sites[0];
  out->dslash_low_site_updates = (long long)sites[1];
  return WD_OK;
}

extern "C" int wd_apply(wd_handle h, const void *in, void *out, int nrhs, int dagger,
                        wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("wd_apply: NULL handle");
  if (in == nullptr || out == nullptr) return bad("wd_apply: NULL vector");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_apply: nrhs must be in [1, 65535]");
  if (in == out) return bad("wd_apply: in and out must not alias");
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return bad("wd_apply: in and out must be device pointers");
  const char *a = static_cast<const char *>(in);
  const char *b = static_cast<const char *>(out);
  const size_t bytes = sizeof(double2) * (size_t)op_n(h) * nrhs;
  if (a < b + bytes && b < a + bytes) return bad("wd_apply: in and out overlap");
  cudaError_t e = launch_wilson_f64(h, static_cast<const double2 *>(in),
                                    static_cast<double2 *>(out), nrhs, dagger ? 1 : 0,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "wd_apply");
  return WD_OK;
}

// ------------------------------------------------------------------ GMRES-DR

extern "C" int gmresdr_history(wd_handle h, double *out, int len) {
  if (h == nullptr || len < 0 || (len > 0 && out == nullptr)) {
    set_error("gmresdr_history: NULL handle, negative len or NULL out");
    return -WD_BAD_ARG;
  }
  const int c = (int)h->gmresdr_hist.size();
  for (int i = 0; i < len && i < c; ++i) out[i] = h->gmresdr_hist[i];
  return c;
}

extern "C" int gmresdr_solve(wd_handle h, const void *b, void *x, int m, int k, double tol,
                             int max_mv, void *V_out, void *Hbar_out, void *theta_out,
                             wd_stats *stats, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("gmresdr_solve: NULL handle");
  if (b == nullptr || x == nullptr) return bad("gmresdr_solve: NULL b or x");
  if (m < 1 || m > 80) return bad("gmresdr_solve: m must be in [1, 80]");
  if (k < 0 || k >= m) return bad("gmresdr_solve: k must satisfy 0 <= k < m");
  if ((long long)m > op_n(h)) return bad("gmresdr_solve: m exceeds the vector length");
  if (!(tol > 0.0)) return bad("gmresdr_solve: tol must be positive");
  if (max_mv < m) return bad("gmresdr_solve: max_mv must be >= m");
  if (V_out != nullptr && !is_device_pointer(V_out)) return bad("gmresdr_solve: V_out must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const size_t bytes = sizeof(double2) * (size_t)op_n(h);
  Staged sb, sx;
  int rc = stage_in(b, bytes, true, sb, ar, s);
  if (rc == WD_OK) rc = stage_in(x, bytes, true, sx, ar, s);
  wd_stats local;
  std::memset(&local, 0, sizeof(local));
  if (rc == WD_OK)
    rc = gmresdr_run(h, sb.dev, sx.dev, m, k, tol, max_mv, static_cast<double2 *>(V_out),
                     static_cast<double2 *>(Hbar_out), static_cast<double2 *>(theta_out),
                     &local, s, nullptr, 0, ar);
  if ((rc == WD_OK || rc == WD_NOT_CONVERGED) && sx.host) {
    cudaError_t e = cudaMemcpyAsync(x, sx.dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "gmresdr_solve: copy x");
  }
  cudaEventRecord(e1, s);
  ar.release();
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && (rc == WD_OK || rc == WD_NOT_CONVERGED)) rc = cuda_fail(e, "gmresdr_solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  local.ms = ms;
  if (stats) *stats = local;
  return rc;
}

// ------------------------------------------------------------------ deflation

extern "C" int wd_deflation_create(wd_handle h, const void *V, const void *U, int k,
                                   wd_deflation *out, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (out == nullptr) return bad("wd_deflation_create: out is NULL");
  *out = nullptr;
  if (h == nullptr || V == nullptr) return bad("wd_deflation_create: NULL handle or V");
  if (k < 1 || k > 128) return bad("wd_deflation_create: k must be in [1, 128]");
  if (!is_device_pointer(V) || (U != nullptr && !is_device_pointer(U)))
    return bad("wd_deflation_create: V and U must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vb = sizeof(double2) * (size_t)op_n(h) * k;
  wd_deflation_space *d = new wd_deflation_space();
  std::memset(d, 0, sizeof(*d));
  d->h = h;
  d->k = k;
  d->kappa = h->kappa;
  d->mu = h->mu;
  cudaError_t e = cudaMalloc(&d->V, vb);
  if (e == cudaSuccess && U) e = cudaMalloc(&d->U, vb);
  if (e == cudaSuccess) e = cudaMalloc(&d->W, vb);
  if (e == cudaSuccess) e = cudaMalloc(&d->LU, sizeof(double2) * k * k);
  if (e == cudaSuccess) e = cudaMalloc(&d->piv, sizeof(int) * k);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d->V, V, vb, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && U) e = cudaMemcpyAsync(d->U, U, vb, cudaMemcpyDeviceToDevice, s);
  int rc = e == cudaSuccess ? WD_OK : cuda_fail(e, "wd_deflation_create");
  if (rc == WD_OK) {
    Arena ar;
    ar.pool = h->pool;
    ar.stream = s;
    rc = deflation_build(d, s, ar);
    ar.release();
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc == WD_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "wd_deflation_create");
  }
  if (rc != WD_OK) {
    wd_deflation_destroy(d);
    return rc;
  }
  *out = d;
  return WD_OK;
}

extern "C" void wd_deflation_destroy(wd_deflation d) {
  if (d == nullptr) return;
  cudaDeviceSynchronize();
  cudaFree(d->V);
  cudaFree(d->U);
  cudaFree(d->W);
  cudaFree(d->LU);
  cudaFree(d->piv);
  delete d;
}

// ------------------------------------------------------------------ D-BiCGStab

extern "C" int dbicgstab_solve_deflated(wd_handle h, wd_deflation d, const void *B, void *X,
                                        int nrhs, double tol, int max_iter, wd_stats *stats,
                                        wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("dbicgstab_solve: NULL handle");
  if (B == nullptr || X == nullptr) return bad("dbicgstab_solve: NULL B or X");
  if (nrhs < 1 || nrhs > 65535) return bad("dbicgstab_solve: nrhs must be in [1, 65535]");
  if (!(tol > 0.0)) return bad("dbicgstab_solve: tol must be positive");
  if (max_iter < 1) return bad("dbicgstab_solve: max_iter must be >= 1");
  if (d != nullptr && d->h != h) return bad("dbicgstab_solve: deflation space built for another handle");
  if (d != nullptr && (d->kappa != h->kappa || d->mu != h->mu))
    return bad("dbicgstab_solve: kappa/mu changed since the deflation space was built");
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = op_n(h);
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const size_t bytes = sizeof(double2) * (size_t)n * nrhs;
  Staged sb, sx;
  std::vector<wd_stats> local(nrhs);
  std::memset(local.data(), 0, sizeof(wd_stats) * nrhs);
  int rc = stage_in(B, bytes, true, sb, ar, s);
  if (rc == WD_OK) rc = stage_in(X, bytes, true, sx, ar, s);
  double2 *R0 = rc == WD_OK ? ar.take<double2>((size_t)n * nrhs) : nullptr;
  double *part = rc == WD_OK ? ar.take<double>((size_t)stream_blocks(n) * 2 * nrhs) : nullptr;
  if (rc == WD_OK && ar.failed) rc = bad_alloc();
  if (rc == WD_OK) {
    // r0 = B - A X0, skipping the product when every X0 is zero (the usual x0 = 0)
    std::vector<double> hp((size_t)stream_blocks(n) * 2 * nrhs);
    cudaError_t e = launch_norms(sx.dev, nullptr, part, n, nrhs, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve: ||x0||");
    bool zero = true;
    for (size_t i = 0; i < hp.size(); i += 2) zero &= hp[i] == 0.0;
    if (rc == WD_OK) {
      if (zero) {
        e = cudaMemcpyAsync(R0, sb.dev, bytes, cudaMemcpyDeviceToDevice, s);
      } else {
        e = launch_wilson_f64(h, sx.dev, R0, nrhs, 0, s);
        if (e == cudaSuccess) e = launch_sub_norm(R0, sb.dev, R0, nullptr, M_ALL, part, n, nrhs, s);
        for (auto &q : local) q.mvp_extra += 1;
      }
      if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve: r0");
    }
  }
  if (rc == WD_OK && d != nullptr) rc = deflate_batched(d, sx.dev, R0, nrhs, s, ar);
  if (rc == WD_OK)
    rc = bicgstab_batched(h, sb.dev, sx.dev, R0, nrhs, tol, max_iter, local.data(), s, nullptr,
                          0, ar);
  if ((rc == WD_OK || rc == WD_NOT_CONVERGED || rc == WD_BREAKDOWN) && sx.host) {
    cudaError_t e = cudaMemcpyAsync(X, sx.dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve: copy X");
  }
  cudaEventRecord(e1, s);
  ar.release();
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && rc != WD_CUDA_ERROR) rc = cuda_fail(e, "dbicgstab_solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    for (int q = 0; q < nrhs; ++q) {
      local[q].ms = ms;
      stats[q] = local[q];
    }
  }
  return rc;
}

extern "C" int dbicgstab_solve(wd_handle h, const void *B, void *X, int nrhs, const void *V,
                               const void *U, int k, double tol, int max_iter, wd_stats *stats,
                               wd_stream stream) {
  if (h == nullptr) return bad("dbicgstab_solve: NULL handle");
  if (k < 0) return bad("dbicgstab_solve: k must be >= 0");
  if (k > 0 && V == nullptr) return bad("dbicgstab_solve: V is NULL with k > 0");
  wd_deflation d = nullptr;
  if (k > 0) {
    int rc = wd_deflation_create(h, V, U, k, &d, stream);
    if (rc != WD_OK) return rc;
  }
  int rc = dbicgstab_solve_deflated(h, d, B, X, nrhs, tol, max_iter, stats, stream);
  if (d) wd_deflation_destroy(d);
  return rc;
}

// ------------------------------------------------------------------ Sec. 4 shifts

extern "C" int tm_multishift_solve(wd_handle h, const void *B, void *X, int nrhs,
                                   const double *mus, int nshift, double tol, int max_iter,
                                   int project, int mixed, wd_stats *stats, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("tm_multishift_solve: NULL handle");
  if (B == nullptr || X == nullptr || mus == nullptr) return bad("tm_multishift_solve: NULL argument");
  if (nrhs < 1 || nrhs > 65535) return bad("tm_multishift_solve: nrhs must be in [1, 65535]");
  if (nshift < 1 || nshift > 64) return bad("tm_multishift_solve: nshift must be in [1, 64]");
  if (!(tol > 0.0) || max_iter < 1) return bad("tm_multishift_solve: tol > 0 and max_iter >= 1 required");
  if (!is_device_pointer(B) || !is_device_pointer(X)) return bad("tm_multishift_solve: B and X must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  int rc = tm_shifts_run(h, static_cast<const double2 *>(B), static_cast<double2 *>(X), nrhs, mus,
                         nshift, tol, max_iter, project, mixed, stats, s, ar);
  ar.release();
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && rc != WD_CUDA_ERROR) rc = cuda_fail(e, "tm_multishift_solve");
  return rc;
}

// ------------------------------------------------------------------ differentiation

// LAM = gamma5 A(-mu)^{-1} gamma5 G with the FP64 (mixed = false) or the
// mixed-precision solver.
static int adjoint_solve(wd_handle h, wd_deflation d, const void *G, void *LAM, int nrhs,
                         double tol, int max_iter, int mixed, int reliable_every,
                         wd_stats *stats, wd_stream stream) {
  if (h == nullptr || G == nullptr || LAM == nullptr) return bad("dbicgstab_solve_adjoint: NULL argument");
  if (nrhs < 1 || nrhs > 65535) return bad("dbicgstab_solve_adjoint: nrhs must be in [1, 65535]");
  if (!is_device_pointer(G) || !is_device_pointer(LAM)) return bad("dbicgstab_solve_adjoint: G and LAM must be device memory");
  if (G == LAM) return bad("dbicgstab_solve_adjoint: G and LAM must not alias");
  cudaStream_t s = (cudaStream_t)stream;
  const long long nn = op_n(h) * nrhs;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  double2 *t = ar.take<double2>((size_t)nn);
  if (ar.failed) return bad_alloc();
  cudaError_t e = launch_gamma5(static_cast<const double2 *>(G), t, nn, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(LAM, 0, sizeof(double2) * nn, s);
  if (e != cudaSuccess) {
    ar.release();
    return cuda_fail(e, "dbicgstab_solve_adjoint");
  }
  const double mu = h->mu;
  h->mu = -mu;
  int rc = mixed ? dbicgstab_solve_mixed(h, d, t, LAM, nrhs, tol, max_iter, reliable_every, stats, stream)
                 : dbicgstab_solve_deflated(h, d, t, LAM, nrhs, tol, max_iter, stats, stream);
  h->mu = mu;
  if (rc == WD_OK || rc == WD_NOT_CONVERGED || rc == WD_BREAKDOWN) {
    e = cudaMemcpyAsync(t, LAM, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_gamma5(t, static_cast<double2 *>(LAM), nn, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve_adjoint");
  }
  ar.release();
  cudaStreamSynchronize(s);
  return rc;
}

extern "C" int dbicgstab_solve_adjoint(wd_handle h, wd_deflation d, const void *G, void *LAM,
                                       int nrhs, double tol, int max_iter, wd_stats *stats,
                                       wd_stream stream) {
  return adjoint_solve(h, d, G, LAM, nrhs, tol, max_iter, 0, 0, stats, stream);
}

extern "C" int dbicgstab_solve_adjoint_mixed(wd_handle h, wd_deflation d, const void *G, void *LAM,
                                             int nrhs, double tol, int max_iter, int reliable_every,
                                             wd_stats *stats, wd_stream stream) {
  return adjoint_solve(h, d, G, LAM, nrhs, tol, max_iter, 1, reliable_every, stats, stream);
}

extern "C" int wd_gradients(wd_handle h, const void *lam, const void *x, void *force,
                            double *dkappa, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr || lam == nullptr || x == nullptr) return bad("wd_gradients: NULL argument");
  if (h->eo) return bad("wd_gradients: defined for the full operator (wd_set_operator(h, 0))");
  if (!is_device_pointer(lam) || !is_device_pointer(x) || (force && !is_device_pointer(force)))
    return bad("wd_gradients: lam, x and force must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (force) e = launch_link_force(h, static_cast<const double2 *>(lam), static_cast<const double2 *>(x),
                                   static_cast<double *>(force), s);
  if (e != cudaSuccess) return cuda_fail(e, "wd_gradients: force");
  if (dkappa) {
    if (h->kappa == 0.0) return bad("wd_gradients: dL/dkappa needs kappa != 0");
    const long long n = h->n;
    Arena ar;
    ar.pool = h->pool;
    ar.stream = s;
    double2 *ax = ar.take<double2>((size_t)n);
    double *part = ar.take<double>((size_t)stream_blocks(n));
    if (ar.failed) return bad_alloc();
    e = launch_wilson_f64(h, static_cast<const double2 *>(x), ax, 1, 0, s);
    if (e == cudaSuccess)
      e = launch_dkappa(static_cast<const double2 *>(lam), static_cast<const double2 *>(x), ax, h->mu,
                        n, part, s);
    std::vector<double> hp(stream_blocks(n));
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
    ar.release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "wd_gradients: dkappa");
    double acc = 0.0;
    for (double v : hp) acc += v;
    *dkappa = acc / h->kappa;
  }
  return WD_OK;
}

// ------------------------------------------------------------------ mixed precision

extern "C" int dbicgstab_solve_mixed(wd_handle h, wd_deflation d, const void *B, void *X,
                                     int nrhs, double tol, int max_iter, int reliable_every,
                                     wd_stats *stats, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("dbicgstab_solve_mixed: NULL handle");
  if (h->eo && h->mixed_bits != 32)
    return bad("dbicgstab_solve_mixed: with even-odd only FP32 storage is available");
  if (B == nullptr || X == nullptr) return bad("dbicgstab_solve_mixed: NULL B or X");
  if (nrhs < 1 || nrhs > 65535) return bad("dbicgstab_solve_mixed: nrhs must be in [1, 65535]");
  if (!(tol > 0.0)) return bad("dbicgstab_solve_mixed: tol must be positive");
  if (max_iter < 1 || reliable_every < 1) return bad("dbicgstab_solve_mixed: max_iter, reliable_every >= 1");
  if (d != nullptr && d->h != h) return bad("dbicgstab_solve_mixed: deflation space built for another handle");
  if (d != nullptr && (d->kappa != h->kappa || d->mu != h->mu))
    return bad("dbicgstab_solve_mixed: kappa/mu changed since the deflation space was built");
  cudaStream_t caller = (cudaStream_t)stream;
  // CUDA graphs cannot be captured on the legacy default stream: work on the
  // handle's side stream, ordered after and before the caller's stream
  cudaStream_t s = caller;
  if (caller == nullptr) {
    if (h->side == nullptr) {
      cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "dbicgstab_solve_mixed: side stream");
    }
    s = h->side;
    cudaEventRecord(h->ev_in, caller);
    cudaStreamWaitEvent(s, h->ev_in, 0);
  }
  const long long n = op_n(h);
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const size_t bytes = sizeof(double2) * (size_t)n * nrhs;
  Staged sb, sx;
  std::vector<wd_stats> local(nrhs);
  std::memset(local.data(), 0, sizeof(wd_stats) * nrhs);
  int rc = stage_in(B, bytes, true, sb, ar, s);
  if (rc == WD_OK) rc = stage_in(X, bytes, true, sx, ar, s);
  double2 *R0 = rc == WD_OK ? ar.take<double2>((size_t)n * nrhs) : nullptr;
  double *part = rc == WD_OK ? ar.take<double>((size_t)stream_blocks(n) * 2 * nrhs) : nullptr;
  if (rc == WD_OK && ar.failed) rc = bad_alloc();
  if (rc == WD_OK) {
    std::vector<double> hp((size_t)stream_blocks(n) * 2 * nrhs);
    cudaError_t e = launch_norms(sx.dev, nullptr, part, n, nrhs, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve_mixed: ||x0||");
    bool zero = true;
    for (size_t i = 0; i < hp.size(); i += 2) zero &= hp[i] == 0.0;
    if (rc == WD_OK) {
      if (zero) {
        e = cudaMemcpyAsync(R0, sb.dev, bytes, cudaMemcpyDeviceToDevice, s);
      } else {
        e = launch_wilson_f64(h, sx.dev, R0, nrhs, 0, s);
        if (e == cudaSuccess) e = launch_sub_norm(R0, sb.dev, R0, nullptr, M_ALL, part, n, nrhs, s);
        for (auto &q : local) q.mvp_extra += 1;
      }
      if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve_mixed: r0");
    }
  }
  if (rc == WD_OK && d != nullptr) rc = deflate_batched(d, sx.dev, R0, nrhs, s, ar);
  if (rc == WD_OK)
    rc = bicgstab_mixed_batched(h, sb.dev, sx.dev, R0, nrhs, tol, max_iter, reliable_every,
                                local.data(), s, ar);
  if ((rc == WD_OK || rc == WD_NOT_CONVERGED || rc == WD_BREAKDOWN) && sx.host) {
    cudaError_t e = cudaMemcpyAsync(X, sx.dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "dbicgstab_solve_mixed: copy X");
  }
  cudaEventRecord(e1, s);
  ar.release();
  if (s != caller) {
    cudaEventRecord(h->ev_out, s);
    cudaStreamWaitEvent(caller, h->ev_out, 0);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && rc != WD_CUDA_ERROR) rc = cuda_fail(e, "dbicgstab_solve_mixed");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    for (int q = 0; q < nrhs; ++q) {
      local[q].ms = ms;
      stats[q] = local[q];
    }
  }
  return rc;
}

extern "C" int wd_apply_f32(wd_handle h, const void *in, void *out, int nrhs, int dagger,
                            wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("wd_apply_f32: NULL handle");
  if (in == nullptr || out == nullptr) return bad("wd_apply_f32: NULL vector");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_apply_f32: nrhs must be in [1, 65535]");
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return bad("wd_apply_f32: in and out must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_links32(h, s);
  if (rc != WD_OK) return rc;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const long long Vop = h->eo ? h->V / 2 : h->V;  // even half vectors in even-odd mode
  const size_t v32 = (size_t)nrhs * 6 * Vop;
  float4 *a = ar.take<float4>(v32), *b = ar.take<float4>(v32);
  float4 *tmp = h->eo ? ar.take<float4>(v32) : nullptr;
  if (ar.failed) return bad_alloc();
  const Mixed32 m{h, h->links32};
  cudaError_t e = launch_f64_to_f32(static_cast<const double2 *>(in), a, Vop, nrhs, nullptr,
                                    nullptr, nullptr, M_ALL, s);
  if (e == cudaSuccess)
    e = h->eo ? launch_schur_f32(m, a, nullptr, b, tmp, nrhs, dagger ? 1 : 0, EPI_NONE, nullptr,
                                 nullptr, nullptr, nullptr, M_ALL, s)
              : launch_wilson_f32(m, a, nullptr, b, nrhs, dagger ? 1 : 0, EPI_NONE, nullptr,
                                  nullptr, nullptr, nullptr, M_ALL, s);
  if (e == cudaSuccess) e = launch_f32_to_f64(b, static_cast<double2 *>(out), Vop, nrhs, s);
  ar.release();
  if (e != cudaSuccess) return cuda_fail(e, "wd_apply_f32");
  return WD_OK;
}

extern "C" int wd_apply_f16(wd_handle h, const void *in, void *out, int nrhs, int dagger,
                            wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr) return bad("wd_apply_f16: NULL handle");
  if (h->eo) return bad("wd_apply_f16: the FP16 kernel acts on the full operator");
  if (in == nullptr || out == nullptr) return bad("wd_apply_f16: NULL vector");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_apply_f16: nrhs must be in [1, 65535]");
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return bad("wd_apply_f16: in and out must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_links16(h, s);
  if (rc != WD_OK) return rc;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const size_t nv = (size_t)nrhs * h->V;
  Half16 a{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
  Half16 b{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
  if (ar.failed) return bad_alloc();
  cudaError_t e = launch_f64_to_f16(static_cast<const double2 *>(in), a, h->V, nrhs, s);
  if (e == cudaSuccess)
    e = launch_wilson_f16(h, h->links16, a, nullptr, b, nrhs, dagger ? 1 : 0, EPI_NONE, nullptr,
                          nullptr, nullptr, nullptr, M_ALL, s);
  if (e == cudaSuccess) e = launch_f16_to_f64(b, static_cast<double2 *>(out), h->V, nrhs, s);
  ar.release();
  if (e != cudaSuccess) return cuda_fail(e, "wd_apply_f16");
  return WD_OK;
}

extern "C" int wd_autotune_f16(wd_handle h, int nrhs, int *R, int *threads, float *ms,
                               wd_stream stream) {
  if (h == nullptr) return bad("wd_autotune_f16: NULL handle");
  if (h->eo) return bad("wd_autotune_f16: the FP16 kernel acts on the full operator");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_autotune_f16: nrhs must be in [1, 65535]");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_links16(h, s);
  if (rc != WD_OK) return rc;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const size_t nv = (size_t)nrhs * h->V;
  Half16 a{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
  Half16 b{ar.take<uint4>(3 * nv), ar.take<float>(nv)};
  if (ar.failed) return bad_alloc();
  cudaError_t e = cudaMemsetAsync(a.v, 0, sizeof(uint4) * 3 * nv, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.n, 0, sizeof(float) * nv, s);
  if (e == cudaSuccess) e = tune_wilson_f16(h, h->links16, nrhs, a, b, s);
  ar.release();
  if (e != cudaSuccess) return cuda_fail(e, "wd_autotune_f16");
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  if (R) *R = h->tune16_R[key];
  if (threads) *threads = h->tune16_T[key];
  if (ms) *ms = h->tune16_ms[key];
  return WD_OK;
}

extern "C" int wd_set_f16_shape(wd_handle h, int nrhs, int R, int threads) {
  if (h == nullptr) return bad("wd_set_f16_shape: NULL handle");
  if (nrhs < 1) return bad("wd_set_f16_shape: nrhs must be >= 1");
  if (!((R == 0 && threads == 0) || ((R == 1 || R == 2 || R == 4) &&
                                     (threads == 64 || threads == 128 || threads == 256))))
    return bad("wd_set_f16_shape: R in {1, 2, 4} and threads in {64, 128, 256} (or both 0)");
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  h->tune16_R[key] = R;
  h->tune16_T[key] = threads;
  h->tune16_ms[key] = 0.f;
  return WD_OK;
}

extern "C" int wd_set_mixed_restart(wd_handle h, double delta, int max_inner) {
  if (h == nullptr) return bad("wd_set_mixed_restart: NULL handle");
  if (!(delta >= 0.0 && delta < 1.0)) return bad("wd_set_mixed_restart: delta must be in [0, 1)");
  if (delta > 0.0 && max_inner < 1) return bad("wd_set_mixed_restart: max_inner must be >= 1");
  h->mixed_delta = delta;
  h->mixed_inner_max = delta > 0.0 ? max_inner : h->mixed_inner_max;
  return WD_OK;
}

extern "C" int wd_set_contraction(wd_handle h, int tensor_cores) {
  if (h == nullptr) return bad("wd_set_contraction: NULL handle");
  if (tensor_cores != 0 && tensor_cores != 1) return bad("wd_set_contraction: 0 or 1");
  h->tc_contract = tensor_cores;
  return WD_OK;
}

extern "C" int wd_set_eigen_estimates(wd_handle h, int fp32_estimates) {
  if (h == nullptr) return bad("wd_set_eigen_estimates: NULL handle");
  if (fp32_estimates != 0 && fp32_estimates != 1) return bad("wd_set_eigen_estimates: 0 or 1");
  h->eig32 = fp32_estimates;
  return WD_OK;
}

extern "C" int wd_tsgemm(const void *V, int kv, const void *Y, int ldy, int ncol,
                         const void *IN, void *OUT, int beta_one, double sign, long long n,
                         int tensor_cores, wd_stream stream) {
  if (V == nullptr || Y == nullptr || OUT == nullptr || (beta_one && IN == nullptr))
    return bad("wd_tsgemm: NULL pointer");
  if (kv < 1 || ncol < 1 || ldy < ncol || n < 1) return bad("wd_tsgemm: bad sizes");
  if (tensor_cores != 0 && tensor_cores != 1) return bad("wd_tsgemm: tensor_cores must be 0 or 1");
  if (tensor_cores ? !ts_update_tc_supported(kv, ncol) : kv > 128)
    return bad("wd_tsgemm: kv must be <= 88 (tensor cores) or <= 128 (FP64)");
  if (!is_device_pointer(V) || !is_device_pointer(Y) || !is_device_pointer(OUT) ||
      (beta_one && !is_device_pointer(IN)))
    return bad("wd_tsgemm: V, Y, IN and OUT must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  const double2 *v = static_cast<const double2 *>(V), *y = static_cast<const double2 *>(Y);
  const double2 *in = static_cast<const double2 *>(IN);
  double2 *out = static_cast<double2 *>(OUT);
  cudaError_t e;
  if (!tensor_cores) {
    e = launch_ts_update(v, kv, y, ldy, ncol, in, out, beta_one ? 1 : 0, sign, n, nullptr, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? WD_OK : cuda_fail(e, "wd_tsgemm");
  }
  const size_t sb = ts_update_tc_scratch_bytes(kv, ncol, n);
  void *scratch = nullptr;
  e = cudaMallocAsync(&scratch, sb + 256, s);
  if (e != cudaSuccess) return cuda_fail(e, "wd_tsgemm: scratch");
  int *err = reinterpret_cast<int *>(static_cast<unsigned char *>(scratch) + sb);
  int herr = 0;
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_ts_update_tc(v, kv, y, ldy, ncol, in, out, beta_one ? 1 : 0, sign, n, scratch, err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "wd_tsgemm");
  if (herr != 0) {
    set_error("wd_tsgemm: a wait in the tensor-core kernel gave up");
    return WD_TIMEOUT;
  }
  return WD_OK;
}

extern "C" int wd_set_mixed_storage(wd_handle h, int bits) {
  if (h == nullptr) return bad("wd_set_mixed_storage: NULL handle");
  if (bits != 32 && bits != 16) return bad("wd_set_mixed_storage: bits must be 32 or 16");
  h->mixed_bits = bits;
  return WD_OK;
}

// ------------------------------------------------------------------ autotuner

extern "C" int wd_autotune_f32(wd_handle h, int nrhs, int *R, int *threads, float *ms,
                               wd_stream stream) {
  if (h == nullptr) return bad("wd_autotune_f32: NULL handle");
  if (h->eo) return bad("wd_autotune_f32: the FP32 kernel acts on the full operator");
  if (nrhs < 1 || nrhs > 65535) return bad("wd_autotune_f32: nrhs must be in [1, 65535]");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_links32(h, s);
  if (rc != WD_OK) return rc;
  Arena ar;
  ar.pool = h->pool;
  ar.stream = s;
  const size_t v32 = (size_t)nrhs * 6 * h->V;
  float4 *a = ar.take<float4>(v32), *b = ar.take<float4>(v32);
  if (ar.failed) return bad_alloc();
  cudaError_t e = cudaMemsetAsync(a, 0, sizeof(float4) * v32, s);
  if (e == cudaSuccess) e = tune_wilson_f32(h, h->links32, nrhs, a, b, s);
  ar.release();
  if (e != cudaSuccess) return cuda_fail(e, "wd_autotune_f32");
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  if (R) *R = h->tune_R[key];
  if (threads) *threads = h->tune_T[key];
  if (ms) *ms = h->tune_ms[key];
  return WD_OK;
}

extern "C" int wd_set_f32_shape(wd_handle h, int nrhs, int R, int threads) {
  if (h == nullptr) return bad("wd_set_f32_shape: NULL handle");
  if (nrhs < 1) return bad("wd_set_f32_shape: nrhs must be >= 1");
  if (!((R == 0 && threads == 0) || ((R == 1 || R == 2 || R == 4) &&
                                     (threads == 64 || threads == 128 || threads == 256))))
    return bad("wd_set_f32_shape: R in {1, 2, 4} and threads in {64, 128, 256} (or both 0)");
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  h->tune_R[key] = R;
  h->tune_T[key] = threads;
  h->tune_ms[key] = 0.f;
  return WD_OK;
}

// ------------------------------------------------------------------ errors

extern "C" const char *wd_error_string(int status) {
  switch (status) {
    case WD_OK: return "ok";
    case WD_BAD_ARG: return "invalid argument";
    case WD_NOT_CONVERGED: return "not converged";
    case WD_BREAKDOWN: return "Krylov breakdown";
    case WD_SINGULAR_PROJECTION: return "singular projected matrix";
    case WD_TIMEOUT: return "device-side wait timed out";
    case WD_CUDA_ERROR: return "CUDA error";
    case WD_OUT_OF_MEMORY: return "out of device memory";
    default: return "unknown status";
  }
}

extern "C" int wd_last_error_detail(char *buf, size_t len) {
  const std::string &m = g_last_error;
  if (buf != nullptr && len > 0) {
    size_t c = m.size() < len - 1 ? m.size() : len - 1;
    std::memcpy(buf, m.data(), c);
    buf[c] = '\0';
  }
  return (int)m.size();
}
