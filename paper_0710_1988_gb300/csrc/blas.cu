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
  if (!sys_on(status, M_ACTIVE, r)) return;  // uniform per block
  // beta = (rho / rho_old) (alpha / omega), once per block: two complex
  // divisions in every thread cost more FP64 issue than the few elements
  // each thread updates
  __shared__ double2 s_bm[2];
  if (threadIdx.x == 0) {
    const BicgScalars S = sc[r];
    const double2 beta = cmul(cdiv(S.rho, S.rho_old), cdiv(S.alpha, S.omega));
    s_bm[0] = beta;
    s_bm[1] = cneg(cmul(beta, S.omega));
  }
  __syncthreads();
  const double2 beta = s_bm[0], mbo = s_bm[1];
  const long long off = (long long)r * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 pi = p[off + i], vi = vv[off + i], ri = rv[off + i];
    // p = r + beta (p - omega v) = r + beta p - (beta omega) v: 8 FMA
    p[off + i] = cfma(mbo, vi, cfma(beta, pi, ri));
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
//
// Both products are FP64-ALU bound on this part (4 DFMA per complex
// element pair against ~0.3 DFMA/byte of machine balance), so the kernels
// are shaped to issue nothing but the DFMAs the product needs: every thread
// walks vector elements, keeps a JT x RT (dot) or NC (update) tile of
// complex accumulators in registers, and the block reduces once at the end.

constexpr int TS_THREADS = 256;

static void ts_dot_tile(int nrhs, int *JT, int *RT) {
  *RT = nrhs >= 2 ? 2 : 1;
  *JT = *RT == 1 ? 16 : 8;
}

static void ts_dot_grid(long long n, int k, int nrhs, dim3 *grid) {
  int JT, RT;
  ts_dot_tile(nrhs, &JT, &RT);
  const int gy = (k + JT - 1) / JT, gz = (nrhs + RT - 1) / RT;
  long long gx = TS_MAX_BLOCKS / (gy * gz);
  const long long need = (n + TS_THREADS - 1) / TS_THREADS;
  if (gx > need) gx = need;
  if (gx < 8) gx = need < 8 ? need : 8;
  if (gx < 1) gx = 1;
  *grid = dim3((unsigned)gx, gy, gz);
}

int ts_dot_blocks(long long n, int k, int nrhs) {
  dim3 g;
  ts_dot_grid(n, k, nrhs, &g);
  return (int)(g.x * g.y * g.z);
}

// Block reduction of a tile of 16 complex sums (32 doubles per thread) in a
// fixed order, written as the block's partials.  Within a warp the 32
// doubles are reduced by recursive halving: at each of the five levels a
// lane keeps half of its values, sends the other half to its partner and
// adds what it receives, so lane i ends with the warp sum of value i after
// 16 + 8 + 4 + 2 + 1 additions (a shuffle tree per value would take 160).
template <int Q = 16>   // complex sums of the tile written (the first Q of the 16)
__device__ __forceinline__ void ts_tile_reduce(double (&vals)[32], double2 *__restrict__ partial) {
  __shared__ double red[32][TS_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int lvl = 0; lvl < 5; ++lvl) {
    const int half = 16 >> lvl;           // values kept after this level
    const bool upper = (lane >> (4 - lvl)) & 1;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double send = upper ? vals[i] : vals[i + half];
      const double keep = upper ? vals[i + half] : vals[i];
      vals[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  red[lane][wid] = vals[0];
  __syncthreads();
  const long long tile = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int w2 = 0; w2 < TS_THREADS / 32; ++w2) {
      a += red[q * 2][w2];
      b += red[q * 2 + 1][w2];
    }
    partial[tile * Q + q] = make_double2(a, b);
  }
}

template <int JT, int RT>
__global__ void __launch_bounds__(TS_THREADS)
ts_dot_kernel(const double2 *__restrict__ V, int k, const double2 *__restrict__ W, int nrhs,
              int g5, long long n, double2 *__restrict__ partial,
              const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  const int j0 = blockIdx.y * JT, r0 = blockIdx.z * RT;
  const int nj = min(JT, k - j0), nr = min(RT, nrhs - r0);
  double2 acc[JT][RT];
#pragma unroll
  for (int j = 0; j < JT; ++j)
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[j][r] = make_double2(0.0, 0.0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 w[RT];
    const bool neg = g5 && (i % 12) >= 6;  // gamma5 = diag(1, 1, -1, -1)
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      w[r] = r < nr ? __ldg(W + (long long)(r0 + r) * n + i) : make_double2(0.0, 0.0);
      if (neg) w[r] = cneg(w[r]);
    }
#pragma unroll
    for (int j = 0; j < JT; ++j) {
      if (j < nj) {
        const double2 v = __ldg(V + (long long)(j0 + j) * n + i);
#pragma unroll
        for (int r = 0; r < RT; ++r) acc[j][r] = cfmac(v, w[r], acc[j][r]);
      }
    }
  }
  double vals[32];
#pragma unroll
  for (int j = 0; j < JT; ++j)
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      vals[(j * RT + r) * 2] = acc[j][r].x;
      vals[(j * RT + r) * 2 + 1] = acc[j][r].y;
    }
  static_assert(JT * RT * 2 == 32, "the tile holds 32 doubles");
  ts_tile_reduce(vals, partial);
}

// One warp per (j, r) pair: the lanes load the gx block partials of the pair
// together (lane b, b + 32, ...) and reduce them with a fixed shuffle tree,
// so the loads overlap instead of forming one dependent chain.
__global__ void ts_dot_finalize_kernel(const double2 *__restrict__ partial, int gx, int gy,
                                       int JT, int RT, int k, int nrhs, double2 *C, int ldc,
                                       double2 *C2, int ldc2, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  const int P = k * nrhs;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int pair = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pair < P; pair += warps) {
    const int j = pair / nrhs, r = pair % nrhs;
    const int ty = j / JT, jj = j % JT, tz = r / RT, rr = r % RT;
    const long long base = ((long long)tz * gy + ty) * gx;
    double2 t = make_double2(0.0, 0.0);
    for (int b = lane; b < gx; b += 32) t = cadd(t, partial[(base + b) * JT * RT + jj * RT + rr]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
    }
    if (lane == 0) {
      C[(long long)j * ldc + r] = t;
      if (C2 != nullptr) {
        double2 &d = C2[(long long)j * ldc2 + r];
        d = cadd(d, t);
      }
    }
  }
}

cudaError_t launch_ts_dot(const double2 *V, int k, const double2 *W, int nrhs, int g5,
                          long long n, double2 *partial, const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (k < 1 || nrhs < 1 || k > 4096 || nrhs > 4096) return cudaErrorInvalidValue;
  dim3 grid;
  ts_dot_grid(n, k, nrhs, &grid);
  int JT, RT;
  ts_dot_tile(nrhs, &JT, &RT);
  if (RT == 1)
    ts_dot_kernel<16, 1><<<grid, TS_THREADS, 0, s>>>(V, k, W, nrhs, g5, n, partial, status);
  else
    ts_dot_kernel<8, 2><<<grid, TS_THREADS, 0, s>>>(V, k, W, nrhs, g5, n, partial, status);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- first Gram-Schmidt pass, double-float

// h = V^dagger w for one vector w with every product and sum carried as a
// pair of FP32 numbers (about 48 significant bits), on this GPU's FP32 pipe
// instead of its much slower FP64 one.  It serves the first pass of
// classical Gram-Schmidt applied twice: the second pass, in FP64, measures
// and removes whatever this one left (its coefficients h2 = V^dagger(w - V h)
// are then of the order of 2^-48 ||w|| instead of 2^-53), and the Hessenberg
// column h + h2 is exact to FP64 rounding.  An operand outside FP32's range
// contributes nothing here and is removed by the FP64 pass.
//  * split: x = hi + lo with hi the top 24 significant bits of x (bit
//    operations, no FP64 instruction) and lo the next 24 (x - hi rounded).
//  * product: Dekker's exact product by FMA, p + e = ah bh, plus the cross
//    terms ah bl + al bh (al bl is below 2^-48 of the product).
//  * sum: Knuth's TwoSum of the running high part and p; the rounding error
//    and the low parts accumulate in the low word.
__device__ __forceinline__ void split_df(double x, float &hi, float &lo) {
  const long long b = __double_as_longlong(x);
  const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;
  if (fe <= 0 || fe >= 255) {   // zero, or outside FP32's normal range
    hi = 0.f;
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu));
  const unsigned rem = (unsigned)b & 0x1FFFFFFFu;       // the 29 fraction bits below hi
  if (rem == 0u || e < 949) {                            // nothing left, or 2^(e-1075) underflows
    lo = 0.f;
    return;
  }
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);   // 2^(e - 1075)
  lo = __uint_as_float(__float_as_uint(__uint2float_rn(rem) * scale) | sign);
}

__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &sh,
                                       float &sl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  const float sum = sh + p;
  const float t = sum - sh;
  const float err = (sh - (sum - t)) + (p - t);
  sl += err + e;
  sh = sum;
}

// Tiles of DF_JT basis vectors: a tile's loads are issued together before
// its arithmetic (the FP32 arithmetic is too quick to hide the loads the way
// the FP64 pipe does in ts_dot_kernel), and the small tile leaves registers
// for four blocks per SM (63 registers, no spills): the kernel is bound by
// instruction issue and latency, so occupancy pays (16^4 tall-skinny time per
// step: 8-vector tiles at three blocks 477 ms, 4 at five 464, 4 at four 450).
constexpr int DF_JT = 4;

static void ts_dot_df_grid(long long n, int k, dim3 *grid) {
  const int gy = (k + DF_JT - 1) / DF_JT;
  long long gx = TS_MAX_BLOCKS / gy;
  const long long need = (n + TS_THREADS - 1) / TS_THREADS;
  if (gx > need) gx = need;
  if (gx < 8) gx = need < 8 ? need : 8;
  if (gx < 1) gx = 1;
  *grid = dim3((unsigned)gx, gy, 1);
}

__global__ void __launch_bounds__(TS_THREADS, 4)
ts_dot_df_kernel(const float2 *__restrict__ Vh, const float2 *__restrict__ Vl, int k,
                 const double2 *__restrict__ W, long long n, double2 *__restrict__ partial,
                 const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  const int j0 = blockIdx.y * DF_JT;
  const int nj = min(DF_JT, k - j0);
  float arh[DF_JT], arl[DF_JT], aih[DF_JT], ail[DF_JT];
#pragma unroll
  for (int j = 0; j < DF_JT; ++j) arh[j] = arl[j] = aih[j] = ail[j] = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float2 vh[DF_JT], vl[DF_JT];
#pragma unroll
    for (int j = 0; j < DF_JT; ++j) {   // rows past the last vector reread it and add nothing
      const long long o = (long long)(j0 + (j < nj ? j : nj - 1)) * n + i;
      vh[j] = __ldg(Vh + o);
      vl[j] = __ldg(Vl + o);
    }
    const double2 w = __ldg(W + i);
    float wrh, wrl, wih, wil;
    split_df(w.x, wrh, wrl);
    split_df(w.y, wih, wil);
#pragma unroll
    for (int j = 0; j < DF_JT; ++j) {
      float vrh = vh[j].x, vrl = vl[j].x, vih = vh[j].y, vil = vl[j].y;
      if (j >= nj) vrh = vrl = vih = vil = 0.f;
      // conj(v) w = (vr wr + vi wi) + i (vr wi - vi wr)
      df_mac(vrh, vrl, wrh, wrl, arh[j], arl[j]);
      df_mac(vih, vil, wih, wil, arh[j], arl[j]);
      df_mac(vrh, vrl, wih, wil, aih[j], ail[j]);
      df_mac(-vih, -vil, wrh, wrl, aih[j], ail[j]);
    }
  }
  // the tile's DF_JT complex sums in the first 2 DF_JT of the 32 reduced values
  double vals[32];
#pragma unroll
  for (int j = 0; j < DF_JT; ++j) {
    vals[2 * j] = (double)arh[j] + (double)arl[j];
    vals[2 * j + 1] = (double)aih[j] + (double)ail[j];
  }
#pragma unroll
  for (int q = 2 * DF_JT; q < 32; ++q) vals[q] = 0.0;
  ts_tile_reduce<DF_JT>(vals, partial);
}

// Each complex128 entry of v as FP32 pairs in two planes: vh[i] = (Re hi,
// Im hi), vl[i] = (Re lo, Im lo).  The basis in the form the double-float
// dot reads (both planes) and the FP32 Gram-Schmidt correction reads (the
// high plane: half the bytes of v), written once per basis vector.
__global__ void __launch_bounds__(256)
split_df_kernel(const double2 *__restrict__ v, float2 *__restrict__ vh, float2 *__restrict__ vl,
                long long count, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 a = v[i];
    float rh, rl, ih, il;
    split_df(a.x, rh, rl);
    split_df(a.y, ih, il);
    vh[i] = make_float2(rh, ih);
    vl[i] = make_float2(rl, il);
  }
}

cudaError_t launch_split_df(const double2 *v, float2 *vh, float2 *vl, long long count,
                            const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  long long blocks = (count + 255) / 256;
  if (blocks > 4 * 1216) blocks = 4 * 1216;
  if (blocks < 1) blocks = 1;
  split_df_kernel<<<(unsigned)blocks, 256, 0, s>>>(v, vh, vl, count, status);
  return cudaGetLastError();
}

cudaError_t launch_ts_dot_df(const float2 *Vh, const float2 *Vl, int k, const double2 *w,
                             long long n, double2 *partial, const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (k < 1 || k > 4096) return cudaErrorInvalidValue;
  dim3 grid;
  ts_dot_df_grid(n, k, &grid);
  ts_dot_df_kernel<<<grid, TS_THREADS, 0, s>>>(Vh, Vl, k, w, n, partial, status);
  return cudaGetLastError();
}

cudaError_t launch_ts_dot_df_finalize(const double2 *partial, long long n, int k, double2 *C,
                                      int ldc, const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  dim3 grid;
  ts_dot_df_grid(n, k, &grid);
  ts_dot_finalize_kernel<<<(k + 3) / 4, 128, 0, s>>>(partial, grid.x, grid.y, DF_JT, 1, k, 1, C,
                                                     ldc, nullptr, 0, status);
  return cudaGetLastError();
}

cudaError_t launch_ts_dot_finalize(const double2 *partial, long long n, int k, int nrhs,
                                   double2 *C, int ldc, double2 *C2, int ldc2,
                                   const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  dim3 grid;
  ts_dot_grid(n, k, nrhs, &grid);
  int JT, RT;
  ts_dot_tile(nrhs, &JT, &RT);
  const int P = k * nrhs;  // one warp per pair, four warps per block
  ts_dot_finalize_kernel<<<(P + 3) / 4, 128, 0, s>>>(partial, grid.x, grid.y, JT, RT, k, nrhs,
                                                     C, ldc, C2, ldc2, status);
  return cudaGetLastError();
}

constexpr int TU_THREADS = 256;
constexpr int TU_MAXK = 128;

template <int NC>
__global__ void __launch_bounds__(TU_THREADS)
ts_update_kernel(const double2 *__restrict__ V, int kv, const double2 *__restrict__ Y, int ldy,
                 int c0, const double2 *IN, double2 *OUT, int beta_one, double sign,
                 long long n, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  __shared__ double2 Ys[TU_MAXK * NC];
  for (int e = threadIdx.x; e < kv * NC; e += blockDim.x) {
    const int j = e / NC, c = e % NC;
    Ys[e] = cscale(sign, Y[(long long)j * ldy + c0 + c]);
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j = 0; j < kv; ++j) {
      const double2 v = __ldg(V + (long long)j * n + i);
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = cfma(v, Ys[j * NC + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const long long o = (long long)(c0 + c) * n + i;
      OUT[o] = beta_one ? cadd(IN[o], acc[c]) : acc[c];
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
  for (int c0 = 0; c0 < ncol;) {
    const int rem = ncol - c0;
    const int nc = rem >= 16 ? 16 : rem >= 8 ? 8 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
    dim3 grid((unsigned)blocks);
    switch (nc) {
      case 16: ts_update_kernel<16><<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, c0, IN, OUT, beta_one, sign, n, status); break;
      case 8: ts_update_kernel<8><<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, c0, IN, OUT, beta_one, sign, n, status); break;
      case 4: ts_update_kernel<4><<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, c0, IN, OUT, beta_one, sign, n, status); break;
      case 2: ts_update_kernel<2><<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, c0, IN, OUT, beta_one, sign, n, status); break;
      default: ts_update_kernel<1><<<grid, TU_THREADS, 0, s>>>(V, kv, Y, ldy, c0, IN, OUT, beta_one, sign, n, status); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c0 += nc;
  }
  return cudaSuccess;
}

// ----------------------------------------------------------------- CGS correction

// w -= V h for the second pass of classical Gram-Schmidt, whose coefficients
// h are of the order of the first pass's rounding (|h| ~ eps ||w||): the
// correction V h then needs only FP32 accuracy relative to itself, which is
// far below FP64 rounding of w, while its products would cost FP64 FMAs.
// FP32 path, taken when ||h||^2 <= 1e-20 (||w0||^2 - ||hsum||^2) (the
// correction below 1e-10 of the vector it corrects; ||w0||^2 from the Wilson
// kernel's partials, hsum the coefficients of both passes): V and h are
// truncated to FP32 by bit operations (no FP64 instruction), the products
// accumulate in FP32, and w is updated in FP64.  Otherwise the FP64 form of
// ts_update.  Every block forms the decision from the same device data in
// the same order, so all take the same path.
__device__ __forceinline__ float f32_trunc(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  const int fe = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);                 // below FP32's normal range
  if (fe >= 255) return __uint_as_float(sign | 0x7F7FFFFFu);  // clamp (not met here)
  return __uint_as_float(sign | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu));
}

__device__ __forceinline__ double f64_widen(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)sign);  // zero (subnormals flushed)
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__global__ void __launch_bounds__(TU_THREADS)
ts_update_correction_kernel(const double2 *__restrict__ V, const float2 *__restrict__ Vh, int kv,
                            const double2 *__restrict__ h, const double2 *__restrict__ hsum,
                            int ldh, const double *__restrict__ part_w, int nbw, double2 *w,
                            long long n, const int *__restrict__ status) {
  if (status != nullptr && *status != 0) return;
  __shared__ float2 hf[TU_MAXK];
  __shared__ double2 hd[TU_MAXK];
  __shared__ int use32;
  if (threadIdx.x < 32) {
    double w2 = 0.0, s2 = 0.0, c2 = 0.0;
    for (int b = threadIdx.x; b < nbw; b += 32) w2 += part_w[(long long)b * 3 + 2];
    for (int r = threadIdx.x; r < kv; r += 32) {
      c2 += cnorm2(h[r]);
      s2 += cnorm2(hsum[(long long)r * ldh]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      w2 += __shfl_xor_sync(0xffffffffu, w2, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if (threadIdx.x == 0) use32 = c2 <= 1e-20 * (w2 - s2) ? 1 : 0;
  }
  for (int r = threadIdx.x; r < kv; r += blockDim.x) {
    hd[r] = h[r];
    hf[r] = make_float2(f32_trunc(h[r].x), f32_trunc(h[r].y));
  }
  __syncthreads();
  const bool fp32 = use32 != 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 o = w[i];
    if (fp32) {
      float ax = 0.f, ay = 0.f;
      for (int r = 0; r < kv; ++r) {
        float vx, vy;
        if (Vh != nullptr) {   // the same truncation, stored: half the bytes of V
          const float2 v = __ldg(Vh + (long long)r * n + i);
          vx = v.x;
          vy = v.y;
        } else {
          const double2 v = __ldg(V + (long long)r * n + i);
          vx = f32_trunc(v.x);
          vy = f32_trunc(v.y);
        }
        const float2 c = hf[r];
        ax = fmaf(vx, c.x, fmaf(-vy, c.y, ax));
        ay = fmaf(vx, c.y, fmaf(vy, c.x, ay));
      }
      o.x -= f64_widen(ax);
      o.y -= f64_widen(ay);
    } else {
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < kv; ++r) acc = cfma(__ldg(V + (long long)r * n + i), hd[r], acc);
      o = csub(o, acc);
    }
    w[i] = o;
  }
}

cudaError_t launch_ts_update_correction(const double2 *V, const float2 *Vh, int kv,
                                        const double2 *h, const double2 *hsum, int ldh,
                                        const double *part_w, int nbw, double2 *w, long long n,
                                        const int *status, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (kv > TU_MAXK || kv < 1) return cudaErrorInvalidValue;
  long long blocks = (n + TU_THREADS - 1) / TU_THREADS;
  if (blocks > 1216) blocks = 1216;
  ts_update_correction_kernel<<<(unsigned)blocks, TU_THREADS, 0, s>>>(V, Vh, kv, h, hsum, ldh,
                                                                     part_w, nbw, w, n, status);
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
  if (status != nullptr && *status != 0) return;  // uniform over the grid
  __shared__ double s_inv;  // one division per block, not per thread
  if (threadIdx.x == 0) s_inv = 1.0 / H[idx].x;
  __syncthreads();
  const double inv = s_inv;
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
