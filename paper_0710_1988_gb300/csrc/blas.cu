// Streaming vector kernels of BiCGStab and GMRES-DR (FP64), their scalar
// finalizers, and the tall-skinny products V^dagger W and W += V Y.
//
// Every kernel is batched over right-hand sides (blockIdx.y = system) and
// skips systems whose status is not in its mask.  Reductions are
// deterministic: a fixed number of blocks per system, each block reduces
// in a fixed shuffle/shared-memory order and writes one partial, and a
// finalizer sums the partials in block order.
#include <cstdio>

#include "cplx.cuh"
#include "kernels.cuh"
#include "wd_internal.h"

namespace wd {

constexpr int SB_THREADS = 256;

int stream_blocks(long long n) {
  long long b = (n + SB_THREADS * 4 - 1) / (SB_THREADS * 4);
  if (b > 608) b = 608;  // 4 blocks per SM on 152 SMs
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ bool sys_on(const int *status, unsigned mask, int r) {
  return status == nullptr || ((mask >> status[r]) & 1u);
}

// ----------------------------------------------------------------- BiCGStab updates

__global__ void __launch_bounds__(SB_THREADS)
bicg_update_p_kernel(double2 *__restrict__ p, const double2 *__restrict__ rv,
                     const double2 *__restrict__ vv, const BicgScalars *__restrict__ sc,
                     const int *__restrict__ status, long long n) {
  const int r = blockIdx.y;
  if (!sys_on(status, M_ACTIVE, r)) return;
  const BicgScalars S = sc[r];
  // beta = (rho / rho_old) (alpha / omega)
  const double2 beta = cmul(cdiv(S.rho, S.rho_old), cdiv(S.alpha, S.omega));
  const double2 om = S.omega;
  const long long off = (long long)r * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 pi = p[off + i], vi = vv[off + i], ri = rv[off + i];
    // p = r + beta (p - omega v)
    double2 q = csub(pi, cmul(om, vi));
    p[off + i] = cfma(beta, q, ri);
  }
}

__global__ void __launch_bounds__(SB_THREADS)
bicg_update_s_kernel(double2 *__restrict__ s, const double2 *__restrict__ rv,
                     const double2 *__restrict__ vv, const BicgScalars *__restrict__ sc,
                     const int *__restrict__ status, long long n) {
  const int r = blockIdx.y;
  if (!sys_on(status, M_ACTIVE, r)) return;
  const double2 al = sc[r].alpha;
  const double2 mal = make_double2(-al.x, -al.y);
  const long long off = (long long)r * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s[off + i] = cfma(mal, vv[off + i], rv[off + i]);  // s = r - alpha v
}

__global__ void __launch_bounds__(SB_THREADS)
bicg_update_xr_kernel(double2 *__restrict__ x, double2 *__restrict__ rv,
                      const double2 *__restrict__ p, const double2 *__restrict__ sv,
                      const double2 *__restrict__ t, const double2 *__restrict__ rhat,
                      const BicgScalars *__restrict__ sc, const int *__restrict__ status,
                      double *__restrict__ partial, long long n) {
  const int r = blockIdx.y;
  if (!sys_on(status, M_ACTIVE, r)) return;
  const double2 al = sc[r].alpha, om = sc[r].omega;
  const double2 mom = make_double2(-om.x, -om.y);
  const long long off = (long long)r * n;
  double red[3] = {0.0, 0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 si = sv[off + i];
    double2 xi = x[off + i];
    xi = cfma(al, p[off + i], xi);      // x += alpha p + omega s
    xi = cfma(om, si, xi);
    x[off + i] = xi;
    const double2 ri = cfma(mom, t[off + i], si);  // r = s - omega t
    rv[off + i] = ri;
    const double2 h = rhat[off + i];
    red[0] = fma(h.x, ri.x, red[0]);
    red[0] = fma(h.y, ri.y, red[0]);
    red[1] = fma(h.x, ri.y, red[1]);
    red[1] = fma(-h.y, ri.x, red[1]);
    red[2] = fma(ri.x, ri.x, red[2]);
    red[2] = fma(ri.y, ri.y, red[2]);
  }
  block_sum<3>(red);
  if (threadIdx.x == 0) {
    double *d = partial + ((long long)r * gridDim.x + blockIdx.x) * 3;
    d[0] = red[0];
    d[1] = red[1];
    d[2] = red[2];
  }
}

__global__ void __launch_bounds__(SB_THREADS)
sub_norm_kernel(double2 *__restrict__ out, const double2 *__restrict__ a,
                const double2 *__restrict__ b, const int *__restrict__ status, unsigned mask,
                double *__restrict__ partial, long long n) {
  const int r = blockIdx.y;
  if (!sys_on(status, mask, r)) return;
  const long long off = (long long)r * n;
  double red[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = csub(a[off + i], b[off + i]);
    out[off + i] = v;
    red[0] = fma(v.x, v.x, red[0]);
    red[0] = fma(v.y, v.y, red[0]);
  }
  block_sum<1>(red);
  if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(SB_THREADS)
norms_kernel(const double2 *__restrict__ a, const double2 *__restrict__ b,
             double *__restrict__ partial, long long n) {
  const int r = blockIdx.y;
  const long long off = (long long)r * n;
  double red[2] = {0.0, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = a[off + i];
    red[0] = fma(v.x, v.x, red[0]);
    red[0] = fma(v.y, v.y, red[0]);
    if (b != nullptr) {
      const double2 w = b[off + i];
      red[1] = fma(w.x, w.x, red[1]);
      red[1] = fma(w.y, w.y, red[1]);
    }
  }
  block_sum<2>(red);
  if (threadIdx.x == 0) {
    double *d = partial + ((long long)r * gridDim.x + blockIdx.x) * 2;
    d[0] = red[0];
    d[1] = red[1];
  }
}

__global__ void __launch_bounds__(SB_THREADS)
restart_vectors_kernel(double2 *__restrict__ rhat, const double2 *__restrict__ rv,
                       double2 *__restrict__ p, double2 *__restrict__ v,
                       const int *__restrict__ status, unsigned mask, long long n) {
  const int r = blockIdx.y;
  if (!sys_on(status, mask, r)) return;
  const long long off = (long long)r * n;
  const double2 z = make_double2(0.0, 0.0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    rhat[off + i] = rv[off + i];
    p[off + i] = z;
    v[off + i] = z;
  }
}

cudaError_t launch_bicg_update_p(double2 *p, const double2 *r, const double2 *v,
                                 const BicgScalars *sc, const int *status, long long n,
                                 int nrhs, cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  bicg_update_p_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(p, r, v, sc, status, n);
  return cudaGetLastError();
}
cudaError_t launch_bicg_update_s(double2 *sv, const double2 *r, const double2 *v,
                                 const BicgScalars *sc, const int *status, long long n,
                                 int nrhs, cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  bicg_update_s_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(sv, r, v, sc, status, n);
  return cudaGetLastError();
}
cudaError_t launch_bicg_update_xr(double2 *x, double2 *r, const double2 *p, const double2 *sv,
                                  const double2 *t, const double2 *rhat, const BicgScalars *sc,
                                  const int *status, double *partial, long long n, int nrhs,
                                  cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  bicg_update_xr_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(
      x, r, p, sv, t, rhat, sc, status, partial, n);
  return cudaGetLastError();
}
cudaError_t launch_sub_norm(double2 *out, const double2 *a, const double2 *b, const int *status,
                            unsigned mask, double *partial, long long n, int nrhs,
                            cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  sub_norm_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(out, a, b, status, mask,
                                                                      partial, n);
  return cudaGetLastError();
}
cudaError_t launch_norms(const double2 *a, const double2 *b, double *partial, long long n,
                         int nrhs, cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  norms_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(a, b, partial, n);
  return cudaGetLastError();
}
cudaError_t launch_bicg_restart_vectors(double2 *rhat, const double2 *r, double2 *p,
                                        double2 *v, const int *status, unsigned mask,
                                        long long n, int nrhs, cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  restart_vectors_kernel<<<dim3(stream_blocks(n), nrhs), SB_THREADS, 0, s>>>(rhat, r, p, v,
                                                                             status, mask, n);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- finalizers

template <int NQ>
__device__ void reduce_partials(const double *partial, int nb, int r, double (&v)[NQ]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double *src = partial + ((long long)r * nb + b) * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += src[q];
  }
  block_sum<NQ>(v);
}

__device__ __forceinline__ void reset_recurrence(BicgScalars &S, double rr) {
  S.rho = make_double2(rr, 0.0);  // r_hat = r, so <r_hat, r> = ||r||^2
  S.rho_old = make_double2(1.0, 0.0);
  S.alpha = make_double2(1.0, 0.0);
  S.omega = make_double2(1.0, 0.0);
  S.rhat_norm = sqrt(rr);
  S.rnorm = sqrt(rr);
}

__global__ void __launch_bounds__(256)
bicg_finalize_kernel(int kind, const double *__restrict__ partial, int nb, BicgScalars *sc,
                     int *status, double *hist, int hist_len) {
  const int r = blockIdx.x;
  const int st = status[r];
  if (kind == FIN_INIT) {  // partial: ||b||^2, ||r0||^2 (NQ = 2)
    double v[2];
    reduce_partials<2>(partial, nb, r, v);
    if (threadIdx.x == 0) {
      BicgScalars &S = sc[r];
      S.bnorm = sqrt(v[0]);
      const double rr = v[1];
      reset_recurrence(S, rr);
      if (S.bnorm == 0.0) {
        S.true_rel = 0.0;
        status[r] = ST_DONE;
      } else if (S.rnorm / S.bnorm <= S.tol) {
        status[r] = ST_RECURSIVE;
      } else {
        status[r] = ST_RESTART;
      }
    }
    return;
  }
  if (kind == FIN_ALPHA || kind == FIN_OMEGA || kind == FIN_RHO) {
    if (st != ST_ACTIVE) return;
    double v[3];
    reduce_partials<3>(partial, nb, r, v);
    if (threadIdx.x != 0) return;
    BicgScalars &S = sc[r];
    if (kind == FIN_ALPHA) {  // <r_hat, v>, ||v||^2
      const double2 rv = make_double2(v[0], v[1]);
      S.mvp += 1;
      if (hypot(rv.x, rv.y) <= 1e-30 * S.rhat_norm * sqrt(v[2])) {
        status[r] = ST_BREAKDOWN;
        return;
      }
      S.alpha = cdiv(S.rho, rv);
    } else if (kind == FIN_OMEGA) {  // <t, s>, ||t||^2
      if (v[2] == 0.0) {  // t = A s = 0 means s = 0: x += alpha p finishes
        S.omega = make_double2(0.0, 0.0);
      } else {
        S.mvp += 1;
        S.omega = cdiv(make_double2(v[0], v[1]), make_double2(v[2], 0.0));
      }
    } else {  // FIN_RHO: <r_hat, r>, ||r||^2
      S.rho_old = S.rho;
      S.rho = make_double2(v[0], v[1]);
      S.rnorm = sqrt(v[2]);
      S.iters += 1;
      if (hist != nullptr && S.iters <= hist_len)
        hist[(long long)r * hist_len + S.iters - 1] = S.rnorm / S.bnorm;
      if (S.rnorm / S.bnorm <= S.tol)
        status[r] = ST_RECURSIVE;
      else if (S.iters >= S.max_iter)
        status[r] = ST_MAXITER;
      else if (hypot(S.rho.x, S.rho.y) <= 1e-30 * S.rhat_norm * S.rnorm)
        status[r] = ST_BREAKDOWN;
    }
    return;
  }
  if (kind == FIN_TRUE) {  // ||b - A x||^2 (NQ = 1)
    if (st != ST_RECURSIVE && st != ST_BREAKDOWN && st != ST_MAXITER) return;
    double v[1];
    reduce_partials<1>(partial, nb, r, v);
    if (threadIdx.x != 0) return;
    BicgScalars &S = sc[r];
    S.mvp_extra += 1;
    S.true_rel = sqrt(v[0]) / S.bnorm;
    if (st != ST_RECURSIVE) return;  // final anyway; just record
    if (S.true_rel <= S.tol) {
      status[r] = ST_DONE;
    } else if (S.restarts < S.max_restarts) {
      S.restarts += 1;
      reset_recurrence(S, v[0]);
      status[r] = ST_RESTART;
    } else {
      status[r] = ST_FAILED;
    }
    return;
  }
  // FIN_ACTIVATE: restart vectors are in place
  if (threadIdx.x == 0 && st == ST_RESTART) status[r] = ST_ACTIVE;
}

cudaError_t launch_bicg_finalize(int kind, const double *partial, int nb, BicgScalars *sc,
                                 int *status, double *hist, int hist_len, int nrhs,
                                 cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  bicg_finalize_kernel<<<nrhs, 256, 0, s>>>(kind, partial, nb, sc, status, hist, hist_len);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- tall-skinny

constexpr int TS_THREADS = 256;
constexpr int TS_SLOTS = 8;     // (pair, split) work items per thread

// Splits per output pair and elements per staged chunk for P = k*nrhs pairs:
// S is the largest power of two with P*S <= TS_THREADS, the chunk holds
// max(32, S) elements so that every split has work.
static void ts_dot_shape(int P, int *S, int *CH) {
  int sp = 1;
  while (sp < 256 && P * sp * 2 <= TS_THREADS) sp *= 2;
  *S = sp;
  *CH = sp > 32 ? sp : 32;
}

int ts_dot_blocks(long long n, int k, int nrhs) {
  int S, CH;
  ts_dot_shape(k * nrhs, &S, &CH);
  long long ch = (n + CH - 1) / CH;
  long long b = ch < TS_MAX_BLOCKS ? ch : TS_MAX_BLOCKS;
  return (int)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(TS_THREADS)
ts_dot_kernel(const double2 *__restrict__ V, int k, const double2 *__restrict__ W, int nrhs,
              int g5, long long n, int S, int CH, double2 *__restrict__ partial,
              const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  extern __shared__ double2 sm[];
  double2 *Vs = sm;                      // [k][CH]
  double2 *Ws = sm + (size_t)k * CH;     // [nrhs][CH]
  const int P = k * nrhs;
  double2 acc[TS_SLOTS];
#pragma unroll
  for (int q = 0; q < TS_SLOTS; ++q) acc[q] = make_double2(0.0, 0.0);
  const long long nch = (n + CH - 1) / CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long i0 = ch * CH;
    __syncthreads();
    for (int e = threadIdx.x; e < (k + nrhs) * CH; e += blockDim.x) {
      const int row = e / CH, col = e % CH;
      const long long i = i0 + col;
      double2 val = make_double2(0.0, 0.0);
      if (i < n) {
        if (row < k) {
          val = V[(long long)row * n + i];
        } else {
          val = W[(long long)(row - k) * n + i];
          if (g5 && (i % 12) >= 6) val = cneg(val);  // gamma5 = diag(1,1,-1,-1)
        }
      }
      sm[(size_t)row * CH + col] = val;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TS_SLOTS; ++q) {
      const int item = threadIdx.x + q * TS_THREADS;
      if (item < P * S) {
        const int pair = item / S, sp = item % S;
        const int j = pair / nrhs, rr = pair % nrhs;
        double2 a = acc[q];
        for (int e = sp; e < CH; e += S) a = cfmac(Vs[j * CH + e], Ws[rr * CH + e], a);
        acc[q] = a;
      }
    }
  }
  // combine the splits of every pair in a fixed order
  __syncthreads();
  double2 *red = sm;  // [P][S]; the host sizes sm for max((k+nrhs)*CH, P*S)
#pragma unroll
  for (int q = 0; q < TS_SLOTS; ++q) {
    const int item = threadIdx.x + q * TS_THREADS;
    if (item < P * S) red[item] = acc[q];
  }
  __syncthreads();
  for (int pair = threadIdx.x; pair < P; pair += blockDim.x) {
    double2 t = make_double2(0.0, 0.0);
    for (int sp = 0; sp < S; ++sp) t = cadd(t, red[pair * S + sp]);
    partial[(long long)blockIdx.x * P + pair] = t;
  }
}

__global__ void ts_dot_finalize_kernel(const double2 *__restrict__ partial, int nb, int k,
                                       int nrhs, double2 *C, int ldc, double2 *C2, int ldc2,
                                       const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  const int P = k * nrhs;
  for (int pair = blockIdx.x * blockDim.x + threadIdx.x; pair < P;
       pair += gridDim.x * blockDim.x) {
    double2 t = make_double2(0.0, 0.0);
    for (int b = 0; b < nb; ++b) t = cadd(t, partial[(long long)b * P + pair]);
    const int j = pair / nrhs, rr = pair % nrhs;
    C[(long long)j * ldc + rr] = t;
    if (C2 != nullptr) {
      double2 &d = C2[(long long)j * ldc2 + rr];
      d = cadd(d, t);
    }
  }
}

static size_t ts_dot_smem(int k, int nrhs) {
  int S, CH;
  ts_dot_shape(k * nrhs, &S, &CH);
  size_t a = (size_t)(k + nrhs) * CH;
  size_t b = (size_t)k * nrhs * S;
  return (a > b ? a : b) * sizeof(double2);
}

cudaError_t launch_ts_dot(const double2 *V, int k, const double2 *W, int nrhs, int g5,
                          long long n, double2 *partial, const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (k < 1 || nrhs < 1 || k * nrhs > TS_SLOTS * TS_THREADS || k + nrhs > TS_MAX_ROWS)
    return cudaErrorInvalidValue;
  int S, CH;
  ts_dot_shape(k * nrhs, &S, &CH);
  const size_t smem = ts_dot_smem(k, nrhs);
  cudaError_t e = cudaFuncSetAttribute(ts_dot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(TS_MAX_ROWS * 32 * sizeof(double2)));
  if (e != cudaSuccess) return e;
  ts_dot_kernel<<<ts_dot_blocks(n, k, nrhs), TS_THREADS, smem, s>>>(V, k, W, nrhs, g5, n, S, CH,
                                                                    partial, status);
  return cudaGetLastError();
}

cudaError_t launch_ts_dot_finalize(const double2 *partial, int nb, int k, int nrhs,
                                   double2 *C, int ldc, double2 *C2, int ldc2,
                                   const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  const int P = k * nrhs;
  ts_dot_finalize_kernel<<<(P + 127) / 128, 128, 0, s>>>(partial, nb, k, nrhs, C, ldc, C2, ldc2,
                                                         status);
  return cudaGetLastError();
}

constexpr int TU_COLS = 16;
constexpr int TU_THREADS = 256;
constexpr int TU_MAXK = 128;

__global__ void __launch_bounds__(TU_THREADS)
ts_update_kernel(const double2 *__restrict__ V, int kv, const double2 *__restrict__ Y, int ldy,
                 int ncol, const double2 *IN, double2 *OUT, int beta_one, double sign,
                 long long n, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  __shared__ double2 Ys[TU_MAXK * TU_COLS];
  const int c0 = blockIdx.y * TU_COLS;
  const int nc = min(TU_COLS, ncol - c0);
  for (int e = threadIdx.x; e < kv * TU_COLS; e += blockDim.x) {
    const int j = e / TU_COLS, c = e % TU_COLS;
    Ys[e] = c < nc ? cscale(sign, Y[(long long)j * ldy + c0 + c]) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 acc[TU_COLS];
#pragma unroll
    for (int c = 0; c < TU_COLS; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j = 0; j < kv; ++j) {
      const double2 v = V[(long long)j * n + i];
#pragma unroll
      for (int c = 0; c < TU_COLS; ++c) acc[c] = cfma(v, Ys[j * TU_COLS + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < TU_COLS; ++c) {
      if (c < nc) {
        const long long o = (long long)(c0 + c) * n + i;
        OUT[o] = beta_one ? cadd(IN[o], acc[c]) : acc[c];
      }
    }
  }
}

cudaError_t launch_ts_update(const double2 *V, int kv, const double2 *Y, int ldy, int ncol,
                             const double2 *IN, double2 *OUT, int beta_one, double sign,
                             long long n, const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (kv > TU_MAXK || kv < 1 || ncol < 1) return cudaErrorInvalidValue;
  long long blocks = (n + TU_THREADS - 1) / TU_THREADS;
  if (blocks > 1216) blocks = 1216;
  dim3 grid((unsigned)blocks, (ncol + TU_COLS - 1) / TU_COLS);
  ts_update_kernel<<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, ncol, IN, OUT, beta_one, sign, n,
                                              status);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- Arnoldi helpers

__global__ void arnoldi_normalize_finalize_kernel(const double *__restrict__ pw, int nb,
                                                  const double *__restrict__ pw0, int nb0,
                                                  double2 *H, int ldh, int j, double lucky,
                                                  int *status, int *m_eff) {
  if (*status != 0) return;
  double a[1] = {0.0}, b[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a[0] += pw[(long long)i * 2];
  for (int i = threadIdx.x; i < nb0; i += blockDim.x) b[0] += pw0[(long long)i * 3 + 2];
  block_sum<1>(a);
  block_sum<1>(b);
  if (threadIdx.x == 0) {
    const double hn = sqrt(a[0]);
    H[(long long)(j + 1) * ldh + j] = make_double2(hn, 0.0);
    if (hn <= lucky * sqrt(b[0])) {
      *status = 1;
      *m_eff = j + 1;
    }
  }
}

__global__ void scale_by_inverse_entry_kernel(double2 *__restrict__ v,
                                              const double2 *__restrict__ w,
                                              const double2 *__restrict__ H, int idx,
                                              long long n, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  const double inv = 1.0 / H[idx].x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = cscale(inv, w[i]);
}

cudaError_t launch_arnoldi_normalize_finalize(const double *partial_w, int nb,
                                              const double *partial_w0, int nb0, double2 *H,
                                              int ldh, int j, double lucky, int *status,
                                              int *m_eff, cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  arnoldi_normalize_finalize_kernel<<<1, 256, 0, s>>>(partial_w, nb, partial_w0, nb0, H, ldh, j,
                                                      lucky, status, m_eff);
  return cudaGetLastError();
}

__global__ void norm_finalize_kernel(const double *__restrict__ partial, int nb, int stride,
                                     double2 *dst) {
  double a[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a[0] += partial[(long long)i * stride];
  block_sum<1>(a);
  if (threadIdx.x == 0) *dst = make_double2(sqrt(a[0]), 0.0);
}

cudaError_t launch_norm_finalize(const double *partial, int nb, int stride, double2 *dst,
                                 cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  norm_finalize_kernel<<<1, 256, 0, s>>>(partial, nb, stride, dst);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_inverse_entry(double2 *v, const double2 *w, const double2 *H,
                                          int idx, long long n, const int *status,
                                          cudaStream_t s) {
  ProfLaunch prof_(PC_STREAM, s);
  scale_by_inverse_entry_kernel<<<stream_blocks(n), SB_THREADS, 0, s>>>(v, w, H, idx, n, status);
  return cudaGetLastError();
}

}  // namespace wd
