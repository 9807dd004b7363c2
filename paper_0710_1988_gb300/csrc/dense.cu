// Small dense FP64 complex linear algebra on one thread block.
//
//  * LU with partial pivoting and triangular solves: the k x k projected
//    system (U^dagger A V) y = U^dagger r0 of Sec. 2.
//  * The end of a GMRES-DR(m,k) cycle (Morgan's deflated restarting, cited
//    in Sec. 1): least squares min ||c - Hbar d|| by Householder QR; the
//    harmonic Ritz matrix M = H_m + |h_{m+1,m}|^2 f e_m^T (f = H_m^{-dagger}
//    e_m, by a banded LU of H_m); every eigenvalue of M estimated in FP32
//    (Householder reduction to Hessenberg form, shifted QR iteration), each
//    estimate refined in FP64 by inverse iteration on M (one CTA each), the
//    refined pairs checked and the k smallest |theta| kept (if the check
//    fails: FP64 reduction and QR iteration, eigenvectors by inverse
//    iteration on the Hessenberg form); then the orthonormal P_{k+1}, the
//    restarted Hbar_k = P_{k+1}^dagger Hbar_m P_k and c = P_{k+1}^dagger rho.
//
// Matrices are small (m <= 80, k <= 128); these kernels keep their working
// matrices in shared memory.  Every loop is bounded.
#include "cplx.cuh"
#include "kernels.cuh"
#include "wd_internal.h"

namespace wd {

constexpr int LU_THREADS = 256;
constexpr int CE_THREADS = 256;
constexpr int CE_MAXM = 80;
static_assert(CE_THREADS > CE_MAXM, "the least-squares step gives one thread to each column and one more to the right-hand side");

// shared-memory leading dimension of an m-column complex matrix: the next
// value = 1 (mod 8) at or above m
__host__ __device__ inline int cyc_ld(int m) { return m + ((9 - m % 8) % 8); }

__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

__device__ double2 csqrt_(double2 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double w = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(w, z.y / (2.0 * w));
  return make_double2(fabs(z.y) / (2.0 * w), copysign(w, z.y));
}

// Block-wide argmax of (val, idx); ties go to the smaller index.  Result in
// every thread.  blockDim.x multiple of 32, <= 1024.
__device__ void block_argmax(double &val, int &idx) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, val, off);
    const int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    sv[w] = val;
    si[w] = idx;
  }
  __syncthreads();
  if (w == 0) {
    val = lane < nw ? sv[lane] : -1.0;
    idx = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, val, off);
      const int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > val || (ov == val && oi < idx)) {
        val = ov;
        idx = oi;
      }
    }
    if (lane == 0) {
      sv[0] = val;
      si[0] = idx;
    }
  }
  __syncthreads();
  val = sv[0];
  idx = si[0];
  __syncthreads();
}

// Sum of a complex value over the block, result in every thread.
__device__ double2 block_csum_all(double2 v) {
  __shared__ double2 res;
  double t[2] = {v.x, v.y};
  block_sum<2>(t);
  if (threadIdx.x == 0) res = make_double2(t[0], t[1]);
  __syncthreads();
  const double2 r = res;
  __syncthreads();
  return r;
}

__device__ double block_dsum_all(double v) {
  __shared__ double res;
  double t[1] = {v};
  block_sum<1>(t);
  if (threadIdx.x == 0) res = t[0];
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

__device__ __forceinline__ double2 warp_csum_all(double2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// In-place LU with partial pivoting of the k x k matrix A (leading dim ld).
// Returns 1 if an exactly zero pivot was met.  Every thread of the block calls it.
__device__ int lu_factor_block(double2 *A, int ld, int k, int *piv) {
  int singular = 0;
  for (int j = 0; j < k; ++j) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = j + threadIdx.x; i < k; i += blockDim.x) {
      const double v = cabs_(A[i * ld + j]);
      if (v > best || (v == best && i < bi)) {
        best = v;
        bi = i;
      }
    }
    block_argmax(best, bi);
    const int p = bi;
    if (threadIdx.x == 0) piv[j] = p;
    if (p != j) {
      for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double2 t = A[j * ld + c];
        A[j * ld + c] = A[p * ld + c];
        A[p * ld + c] = t;
      }
    }
    __syncthreads();
    const double2 pv = A[j * ld + j];
    if (pv.x == 0.0 && pv.y == 0.0) {
      singular = 1;
      continue;
    }
    const double2 rp = cdiv(make_double2(1.0, 0.0), pv);
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) A[i * ld + j] = cmul(A[i * ld + j], rp);
    __syncthreads();
    const int w = k - j - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, c = j + 1 + e % w;
      A[i * ld + c] = csub(A[i * ld + c], cmul(A[i * ld + j], A[j * ld + c]));
    }
    __syncthreads();
  }
  return singular;
}

// Solve (LU) Y = C in place for nrhs columns of C (row-major, leading dim ldc).
__device__ void lu_solve_block(const double2 *LU, int ld, const int *piv, int k, double2 *C,
                               int ldc, int nrhs) {
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    for (int j = 0; j < k; ++j) {
      const int p = piv[j];
      if (p != j) {
        const double2 t = C[j * ldc + r];
        C[j * ldc + r] = C[p * ldc + r];
        C[p * ldc + r] = t;
      }
    }
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {  // unit lower triangle
    const int w = k - j - 1;
    for (int e = threadIdx.x; e < w * nrhs; e += blockDim.x) {
      const int i = j + 1 + e / nrhs, r = e % nrhs;
      C[i * ldc + r] = csub(C[i * ldc + r], cmul(LU[i * ld + j], C[j * ldc + r]));
    }
    __syncthreads();
  }
  for (int j = k - 1; j >= 0; --j) {  // upper triangle
    const double2 u = LU[j * ld + j];
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
      const double2 v = C[j * ldc + r];
      C[j * ldc + r] = (u.x == 0.0 && u.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(v, u);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < j * nrhs; e += blockDim.x) {
      const int i = e / nrhs, r = e % nrhs;
      C[i * ldc + r] = csub(C[i * ldc + r], cmul(LU[i * ld + j], C[j * ldc + r]));
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(LU_THREADS)
lu_factor_kernel(double2 *A, int k, int *piv, double *info) {
  const int sing = lu_factor_block(A, k, k, piv);
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0, mn = 1e308;
    for (int j = 0; j < k; ++j) {
      const double v = cabs_(A[j * k + j]);
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    }
    info[0] = sing ? 1.0 : 0.0;
    info[1] = mn > 0.0 ? mx / mn : 1e308;  // crude condition estimate from the pivots
  }
}

__global__ void __launch_bounds__(LU_THREADS)
lu_solve_kernel(const double2 *LU, const int *piv, int k, double2 *C, int nrhs) {
  lu_solve_block(LU, k, piv, k, C, nrhs, nrhs);
}

cudaError_t launch_lu_factor(double2 *A, int k, int *piv, double *info, cudaStream_t s) {
  ProfLaunch prof_(PC_DENSE, s);
  lu_factor_kernel<<<1, LU_THREADS, 0, s>>>(A, k, piv, info);
  return cudaGetLastError();
}

cudaError_t launch_lu_solve(const double2 *LU, const int *piv, int k, double2 *C, int nrhs,
                            cudaStream_t s) {
  ProfLaunch prof_(PC_DENSE, s);
  lu_solve_kernel<<<1, LU_THREADS, 0, s>>>(LU, piv, k, C, nrhs);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- GMRES-DR cycle end

// Work buffer of the cycle end (complex entries): G (m x k) and T1 ((m+1) x k)
// in the first 2 (m+1)^2, then the Hessenberg matrix and its transform Z
// (m x m each, leading dimension m).
__host__ __device__ inline double2 *cyc_hess(double2 *work, int m, int k) {
  return work + (size_t)2 * (m + 1) * (m + 1);
}
// reflector j of the Hessenberg reduction: u_j (row j of an m x m array,
// entries j+1 .. iend_j) and (tau_j, iend_j) (tau_j = 0: no reflection)
__host__ __device__ inline double2 *cyc_zg(double2 *work, int m, int k) {
  return work + (size_t)2 * (m + 1) * (m + 1) + (size_t)m * m;
}
__host__ __device__ inline double2 *cyc_tau(double2 *work, int m, int k) {
  return work + (size_t)2 * (m + 1) * (m + 1) + (size_t)2 * m * m;
}
// The harmonic Ritz matrix M (m x m, row-major) shares the Hessenberg slot
// (the FP64 fallback reads it before it writes H there), the refined
// eigenvectors (row q: the vector of estimate q) the reflector slot.
__host__ __device__ inline double2 *cyc_mat(double2 *work, int m, int k) { return cyc_hess(work, m, k); }
__host__ __device__ inline double2 *cyc_vec(double2 *work, int m, int k) { return cyc_zg(work, m, k); }
// [0, m): FP32 eigenvalue estimates; [m, 2m): refined eigenvalues; [2m, 3m):
// relative residuals (.x); [3m]: (largest |M_ij|, 0); [3m + 1]: trace M
__host__ __device__ inline double2 *cyc_est(double2 *work, int m, int k) {
  return work + (size_t)2 * (m + 1) * (m + 1) + (size_t)2 * m * m + m;
}

// One thread per line (column of X from the left, row of Y from the right):
// the left reflection on columns [c0, c1) of X and, in the same pass, the
// right reflection on rows [0, ny) of Y, both over indices i0..i1.  Each
// thread forms its own dot product serially, so every lane of an FP64
// instruction does useful work and no cross-lane reduction is needed; the
// reflector's support is short (i1 - i0 < k + 1 after a restart).
__device__ void reflect_lines(double2 *X, int c0, int c1, double2 *Y, int ny, int ld,
                              const double2 *u, double tau, int i0, int i1) {
  const int nx = X != nullptr ? c1 - c0 : 0;
  for (int t = threadIdx.x; t < nx + ny; t += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    if (t < nx) {  // X <- (I - tau u u^dagger) X, column c
      const int c = c0 + t;
      for (int i = i0; i <= i1; ++i) s = cfmac(u[i], X[i * ld + c], s);
      const double2 f = cscale(tau, s);
      for (int i = i0; i <= i1; ++i) X[i * ld + c] = csub(X[i * ld + c], cmul(u[i], f));
    } else {       // Y <- Y (I - tau u u^dagger), row r
      const int r = t - nx;
      for (int i = i0; i <= i1; ++i) s = cfma(Y[r * ld + i], u[i], s);
      const double2 f = cscale(tau, s);
      for (int i = i0; i <= i1; ++i) Y[r * ld + i] = csub(Y[r * ld + i], cmul(f, cconj(u[i])));
    }
  }
}

// Least squares min || c - Hbar d || for the (me+1) x me leading part of the
// row-major (m+1) x m Hbar.  Writes d (m entries, zero beyond me), rho = c - Hbar d
// (m+1 entries) and ||rho||.
__device__ void cycle_lsq(const CycleEndArgs &a, int me, double2 *sm) {
  const int m = a.m, ld = cyc_ld(m);
  double2 *Hs = sm;                    // (m+1) x ld
  double2 *cz = Hs + (m + 1) * ld;     // m+1
  double2 *u = cz + (m + 1);           // m+1
  double2 *dd = u + (m + 1);           // m
  for (int e = threadIdx.x; e < (m + 1) * m; e += blockDim.x) Hs[(e / m) * ld + e % m] = a.H[e];
  for (int i = threadIdx.x; i <= m; i += blockDim.x) cz[i] = a.c[i];
  // Each reflector spans rows j .. iend, iend the last nonzero row of column
  // j (j + 1 in the Hessenberg part, k after a restart in the leading full
  // block): a shared atomic maximum, triple-buffered as in schur_block so that
  // no slot is reset while another thread may still read or update it.
  __shared__ int s_end[3];
  if (threadIdx.x < 3) s_end[threadIdx.x] = 0;
  __syncthreads();
  for (int j = 0; j < me; ++j) {
    const int slot = j % 3;
    double part = 0.0;
    for (int i = j + threadIdx.x; i <= me; i += blockDim.x) {
      const double2 h = Hs[i * ld + j];
      part += cnorm2(h);
      if (h.x != 0.0 || h.y != 0.0) atomicMax(&s_end[slot], i);
    }
    const double sigma = block_dsum_all(part);  // its barriers order the atomics
    const int iend = s_end[slot];
    if (threadIdx.x == 0) s_end[(j + 2) % 3] = 0;
    if (sigma == 0.0) continue;
    const double2 al = Hs[j * ld + j];
    const double nx = sqrt(sigma), aa = cabs_(al);
    const double2 ph = aa > 0.0 ? cscale(1.0 / aa, al) : make_double2(1.0, 0.0);
    const double2 beta = cscale(-nx, ph);
    for (int i = j + threadIdx.x; i <= iend; i += blockDim.x)
      u[i] = i == j ? csub(al, beta) : Hs[i * ld + j];
    __syncthreads();
    const double tau = 1.0 / (nx * (nx + aa));  // 2 / ||u||^2
    // columns j+1 .. me-1 of Hbar (threads 0 .. me-j-2) and the right-hand
    // side (the last thread; blockDim.x > CE_MAXM keeps the two apart)
    double2 *col = nullptr;
    int cld = ld;
    if (threadIdx.x == blockDim.x - 1) {
      col = cz;
      cld = 1;
    } else if (threadIdx.x < me - j - 1) {
      col = Hs + j + 1 + threadIdx.x;
    }
    if (col != nullptr) {
      double2 sd = make_double2(0.0, 0.0);
      for (int i = j; i <= iend; ++i) sd = cfmac(u[i], col[i * cld], sd);
      const double2 f = cscale(tau, sd);
      for (int i = j; i <= iend; ++i) col[i * cld] = csub(col[i * cld], cmul(u[i], f));
    }
    __syncthreads();
    for (int i = j + threadIdx.x; i <= iend; i += blockDim.x)
      Hs[i * ld + j] = i == j ? beta : make_double2(0.0, 0.0);
    __syncthreads();
  }
  for (int j = me - 1; j >= 0; --j) {
    if (threadIdx.x == 0) {
      const double2 rjj = Hs[j * ld + j];
      dd[j] = (rjj.x == 0.0 && rjj.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(cz[j], rjj);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += blockDim.x) cz[i] = csub(cz[i], cmul(Hs[i * ld + j], dd[j]));
    __syncthreads();
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) a.d[j] = j < me ? dd[j] : make_double2(0.0, 0.0);
  double part = 0.0;
  for (int i = threadIdx.x; i <= m; i += blockDim.x) {
    double2 v = a.c[i];
    for (int j = 0; j < me; ++j) v = csub(v, cmul(a.H[i * m + j], dd[j]));
    a.rho[i] = v;
    part += cnorm2(v);
  }
  const double rr = block_dsum_all(part);
  if (threadIdx.x == 0) a.res[0] = sqrt(rr);
  __syncthreads();
}

// Complex Givens rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0]:
// c = |x| / nrm, s = (x / |x|) conj(y) / nrm, nrm = sqrt(|x|^2 + |y|^2).
__device__ __forceinline__ void givens(double2 x, double2 y, double &c, double2 &s) {
  const double a2 = cnorm2(x), b2 = cnorm2(y);
  if (a2 == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    return;
  }
  const double ra = rsqrt(a2), rn = rsqrt(a2 + b2);
  c = a2 * ra * rn;
  s = cscale(ra * rn, cmul(x, cconj(y)));
}

// givens() computed by one warp (x, y the same on every lane; every lane
// calls it).  An FP64 instruction occupies the warp's pipe as long with one
// active lane as with 32, so the independent products go to separate lanes:
// lane 0 |x|^2, lane 1 |y|^2, lane 2 and 3 Re and Im of x conj(y), then one
// rsqrt (lane 0 of |x|^2, the others of |x|^2 + |y|^2) and two multiplies
// (lane 0 c, lanes 2 and 3 s).  Each value is rounded exactly as in givens().
// Lane 0 writes c and s.
__device__ __forceinline__ void givens_lanes(double2 x, double2 y, int ln, double *gc,
                                             double2 *gs) {
  const double f0 = ln == 1 ? y.x : x.x;
  const double f1 = ln == 0 ? x.x : (ln == 3 ? -y.y : y.x);
  const double f2 = ln == 1 ? y.y : x.y;
  const double f3 = ln == 0 ? x.y : (ln == 3 ? y.x : y.y);
  const double q = fma(f0, f1, f2 * f3);
  const double a2 = __shfl_sync(0xffffffffu, q, 0), b2 = __shfl_sync(0xffffffffu, q, 1);
  if (a2 == 0.0) {  // uniform over the warp
    if (ln == 0) {
      *gc = 0.0;
      *gs = make_double2(1.0, 0.0);
    }
    return;
  }
  const double r = rsqrt(ln == 0 ? a2 : a2 + b2);
  const double ra = __shfl_sync(0xffffffffu, r, 0), rn = __shfl_sync(0xffffffffu, r, 1);
  const double t = ln == 0 ? a2 * ra : ra * rn;
  const double u = ln == 0 ? t * rn : t * q;
  const double sx = __shfl_sync(0xffffffffu, u, 2), sy = __shfl_sync(0xffffffffu, u, 3);
  if (ln == 0) {
    *gc = u;
    *gs = make_double2(sx, sy);
  }
}

// givens_lanes() for a group of 8 lanes starting at lane `base` (ln = lane -
// base): four groups of one warp form four independent rotations with the
// same instructions.  Every lane of the warp calls it (the shuffles take the
// whole warp); lane 0 of the group writes c and s when `write` is set.
__device__ __forceinline__ void givens_group(double2 x, double2 y, int ln, int base, bool write,
                                             double *gc, double2 *gs) {
  const double f0 = ln == 1 ? y.x : x.x;
  const double f1 = ln == 0 ? x.x : (ln == 3 ? -y.y : y.x);
  const double f2 = ln == 1 ? y.y : x.y;
  const double f3 = ln == 0 ? x.y : (ln == 3 ? y.x : y.y);
  const double q = fma(f0, f1, f2 * f3);
  const double a2 = __shfl_sync(0xffffffffu, q, base), b2 = __shfl_sync(0xffffffffu, q, base + 1);
  const double r = rsqrt(ln == 0 ? a2 : a2 + b2);
  const double ra = __shfl_sync(0xffffffffu, r, base), rn = __shfl_sync(0xffffffffu, r, base + 1);
  const double t = ln == 0 ? a2 * ra : ra * rn;
  const double u = ln == 0 ? t * rn : t * q;
  const double sx = __shfl_sync(0xffffffffu, u, base + 2), sy = __shfl_sync(0xffffffffu, u, base + 3);
  if (write && ln == 0) {
    if (a2 == 0.0) {
      *gc = 0.0;
      *gs = make_double2(1.0, 0.0);
    } else {
      *gc = u;
      *gs = make_double2(sx, sy);
    }
  }
}

// Eigenvalues of the m x m matrix A (smem, row-major).  Householder reduction
// to upper Hessenberg form H = Z^dagger A Z, Z = H_0 H_1 ... the product of
// the reflectors, which are stored (Ug: u_j as row j; taug: tau_j, last row of
// u_j) instead of being multiplied out, H is copied to Hg (leading dimension
// m) for the eigenvector step; then shifted complex QR iteration on the
// active block only: its
// diagonal ends up holding the eigenvalues.  Rotations are applied only inside
// the active window [l, hi]: the parts of T outside it and the Schur vectors
// never feed back into the iteration, and the eigenvectors come from H by
// inverse iteration (harmonic_ritz_vector_kernel), so the eigenvalues are those
// of the full Schur iteration, bit for bit, at a fraction of its FP64 work.
// Returns 1 if the QR iteration did not converge in 30 m sweeps.
__device__ int schur_block(double2 *A, int m, int ld, double2 *u, long long *clk, double2 *Hg,
                           double2 *Ug, double2 *taug) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int j = tid; j < m; j += bd) taug[j] = make_double2(0.0, 0.0);
  __syncthreads();
  // Householder reduction to upper Hessenberg form.  Each reflector spans
  // rows j+1 .. iend, iend the last nonzero row of column j: after a
  // GMRES-DR restart only the leading (k+1) x k block is full, so the
  // reflectors stop at row k instead of m - 1.  iend comes from a shared
  // atomic maximum, triple-buffered so that no slot is reset while another
  // thread may still read or update it.
  __shared__ int s_end[3];
  if (tid < 3) s_end[tid] = 0;
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const int slot = j % 3;
    double part = 0.0;
    for (int i = j + 2 + tid; i < m; i += bd) {
      const double2 d = A[i * ld + j];
      part += cnorm2(d);
      if (d.x != 0.0 || d.y != 0.0) atomicMax(&s_end[slot], i);
    }
    const double below = block_dsum_all(part);  // its barriers order the atomics
    const int iend = s_end[slot];
    if (tid == 0) s_end[(j + 2) % 3] = 0;
    if (below == 0.0) continue;
    const double2 al = A[(j + 1) * ld + j];
    const double aa = cabs_(al), nx = sqrt(below + aa * aa);
    const double2 ph = aa > 0.0 ? cscale(1.0 / aa, al) : make_double2(1.0, 0.0);
    const double2 beta = cscale(-nx, ph);
    for (int i = j + 1 + tid; i <= iend; i += bd) u[i] = i == j + 1 ? csub(al, beta) : A[i * ld + j];
    __syncthreads();
    const double tau = 1.0 / (nx * (nx + aa));
    for (int i = j + 1 + tid; i <= iend; i += bd) Ug[(size_t)j * m + i] = u[i];
    if (tid == 0) taug[j] = make_double2(tau, (double)iend);
    // H A on columns j..m-1, then A H
    reflect_lines(A, j, m, nullptr, 0, ld, u, tau, j + 1, iend);
    __syncthreads();
    reflect_lines(nullptr, 0, 0, A, m, ld, u, tau, j + 1, iend);
    __syncthreads();
    for (int i = j + 1 + tid; i <= iend; i += bd)
      A[i * ld + j] = i == j + 1 ? beta : make_double2(0.0, 0.0);
    __syncthreads();
  }
  double part = 0.0;
  for (int e = tid; e < m * m; e += bd) part = fmax(part, cabs1(A[(e / m) * ld + e % m]));
  {
    __shared__ double smax[32];
    for (int off = 16; off > 0; off >>= 1) part = fmax(part, __shfl_down_sync(0xffffffffu, part, off));
    if ((tid & 31) == 0) smax[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double mx = 0.0;
      for (int w = 0; w < (bd >> 5); ++w) mx = fmax(mx, smax[w]);
      smax[0] = mx;
    }
    __syncthreads();
    part = smax[0];
    __syncthreads();
  }
  const double anorm = part > 0.0 ? part : 1.0;
  for (int e = tid; e < m * m; e += bd) Hg[e] = A[(e / m) * ld + e % m];
  __syncthreads();
  if (clk != nullptr && tid == 0) clk[7] = clock64();
  // Shifted QR iteration on the active block [l..hi], with up to QR_BULGES
  // shifts per sweep chased as separate bulges three rows apart.  Warp 4
  // owns the chains, eight lanes per bulge: at each step a lane group
  // applies its bulge's current rotation to the entries the next rotation
  // depends on (rows kk..kk+2 of columns kk, kk+1) and forms the next
  // rotation, all bulges with the same instructions.  Warps 0-3 apply the
  // rotations of every active bulge to the rest of the block: the row
  // rotations in one phase, the column rotations in the next (a row rotation
  // of one bulge and a column rotation of another can share entries; left
  // and right rotations commute, so the two phases give the sequential
  // result).  Bulges three rows apart touch disjoint rows with their row
  // rotations and disjoint columns with their column rotations within a
  // step, and an entry meets the rotations of an earlier sweep before those
  // of a later one, as in one sweep after the other.  (The FP64 unit is
  // shared by the SM's four schedulers and an FP64 warp instruction holds it
  // as long with one active lane as with 32: several bulges overlap the
  // chains of dependent FP64 operations that bound a single sweep.)
  constexpr int QR_BULGES = 4;            // four lane groups of the chain warp
  constexpr int QR_CHAIN0 = 4;            // the chain warp (warps 5-7 wait at the barriers)
  __shared__ double s_gc[3][QR_BULGES];     // rotation of step t in slot t % 3
  __shared__ double2 s_gs[3][QR_BULGES];
  __shared__ double2 s_shift[QR_BULGES];
  __shared__ int s_l[2];    // deflation point of the scan, double-buffered
  const int wid = tid >> 5, lane = tid & 31;
  const int nbulk = 32 * QR_CHAIN0;       // threads of the bulk updates
  long long rotations = 0, t_scan = 0, t_rot = 0, t0 = 0;
  int hi = m - 1, its = 0, total = 0, scan = 0;
  if (tid < 2) s_l[tid] = 0;
  __syncthreads();
  while (hi > 0) {
    if (total >= 30 * m) return 1;
    if (tid == 0) t0 = clock64();
    // l = the largest index in [1, hi] whose subdiagonal entry is negligible
    // (0 if none): one candidate per thread, the maximum by a shared atomic.
    // The slot written now was last read before the previous scan's barrier
    // and is reset for the scan after next.
    const int slot = scan & 1;
    for (int q = 1 + tid; q <= hi; q += bd) {
      double tst = cabs1(A[(q - 1) * ld + q - 1]) + cabs1(A[q * ld + q]);
      if (tst == 0.0) tst = anorm;
      if (cabs1(A[q * ld + q - 1]) <= 2.220446049250313e-16 * tst) atomicMax(&s_l[slot], q);
    }
    __syncthreads();
    const int l = s_l[slot];
    if (tid == 0) s_l[slot ^ 1] = 0;
    ++scan;
    if (l > 0 && tid == 0) A[l * ld + l - 1] = make_double2(0.0, 0.0);
    __syncthreads();
    if (l == hi) {
      --hi;
      its = 0;
      continue;
    }
    ++its;
    ++total;
    const int w = hi - l + 1;                       // rotations per bulge: w - 1
    const int nb = w >= 8 ? QR_BULGES : 1;
    rotations += (long long)nb * (w - 1);
    if (tid == 0) {
      const long long t1 = clock64();
      t_scan += t1 - t0;
      t0 = t1;
      // shifts: the two eigenvalues of the trailing 2 x 2 block (the one
      // nearest its last diagonal entry first), once per pair of bulges (the
      // second pair repeats them, as a second double-shift sweep would);
      // every tenth sweep starts from an exceptional shift
      {
        const int r0 = hi - 1;
        const double2 a = A[(r0) * ld + r0], bb = A[r0 * ld + r0 + 1];
        const double2 c = A[(r0 + 1) * ld + r0], d = A[(r0 + 1) * ld + r0 + 1];
        const double2 p = cscale(0.5, csub(a, d));
        const double2 bc = cmul(bb, c);
        double2 q = csqrt_(cadd(cmul(p, p), bc));
        if (p.x * q.x + p.y * q.y < 0.0) q = cneg(q);
        const double2 den = cadd(p, q);
        const double2 e1 = (den.x == 0.0 && den.y == 0.0) ? d : csub(d, cdiv(bc, den));
        const double2 e2 = csub(cadd(a, d), e1);                  // the other eigenvalue
        for (int b = 0; b < nb; ++b) s_shift[b] = (b & 1) ? e2 : e1;
      }
      if (its % 10 == 0) s_shift[0] = cadd(A[hi * ld + hi], make_double2(cabs1(A[hi * ld + hi - 1]), 0.0));
    }
    __syncthreads();
    if (wid == QR_CHAIN0 && lane == 0)
      givens(csub(A[l * ld + l], s_shift[0]), A[(l + 1) * ld + l], s_gc[0][0], s_gs[0][0]);
    __syncthreads();
    const int nsteps = (w - 1) + 3 * (nb - 1);
    // Step t: the chain warp applies the local part of each bulge's rotation
    // and forms the rotations of step t+1 while warps 0-3 apply the row
    // rotations of step t; a barrier of these five warps; then warps 0-3
    // apply the column rotations of step t (and, after a barrier of their
    // own, the row rotations of step t+1) while the chain warp goes on with
    // step t+1.  The chain's entries of step t+1 (rows kk+1..kk+3 of columns
    // kk+1, kk+2) are written by neither, and a rotation is read from slot
    // t % 3 while the chain writes slot (t + 2) % 3.  Warps 5-7 wait at the
    // barrier that ends the sweep.
    for (int t = 0; t < nsteps; ++t) {
      const int par = t % 3, nxt = (t + 1) % 3;
      // ---- phase 1: chains, and the row rotations of every active bulge
      if (wid == QR_CHAIN0) {
        const int b = lane >> 3, ln = lane & 7, base = lane & ~7;
        const int tb = t - 3 * b;
        const bool act = b < nb && tb >= 0 && tb <= w - 2;
        const bool enter = b < nb && tb == -1;        // first rotation, for the next step
        const int kk = act ? l + tb : l;              // a valid index for idle groups
        const double gc = s_gc[par][b];
        const double2 gs = s_gs[par][b];
        const double2 mgs = cneg(cconj(gs)), cgs = cconj(gs), ngs = cneg(gs);
        // lanes 0..3: row rotation on the 2 x 2 block (kk, kk+1)^2; then
        // lanes 0..5: column rotation on rows kk..kk+2; then lanes 0..3 form
        // the next rotation from column kk
        double2 v = make_double2(0.0, 0.0);
        if (act && ln < 4) {
          const int j = kk + (ln & 1);
          const double2 u0 = A[kk * ld + j], u1 = A[(kk + 1) * ld + j];
          v = (ln < 2) ? cadd(cscale(gc, u0), cmul(gs, u1)) : cadd(cmul(mgs, u0), cscale(gc, u1));
        } else if (act && ln < 6 && kk + 2 <= hi) {
          v = A[(kk + 2) * ld + kk + (ln - 4)];
        }
        const int src = base + (ln & 6);
        double2 p0, p1;
        p0.x = __shfl_sync(0xffffffffu, v.x, src);
        p0.y = __shfl_sync(0xffffffffu, v.y, src);
        p1.x = __shfl_sync(0xffffffffu, v.x, src + 1);
        p1.y = __shfl_sync(0xffffffffu, v.y, src + 1);
        const double2 o = (ln & 1) == 0 ? cadd(cscale(gc, p0), cmul(cgs, p1))
                                        : cadd(cmul(ngs, p0), cscale(gc, p1));
        if (act && (ln < 4 || (ln < 6 && kk + 2 <= hi))) A[(kk + (ln >> 1)) * ld + kk + (ln & 1)] = o;
        double2 x, y;
        x.x = __shfl_sync(0xffffffffu, o.x, base + 2);
        x.y = __shfl_sync(0xffffffffu, o.y, base + 2);
        y.x = __shfl_sync(0xffffffffu, o.x, base + 4);
        y.y = __shfl_sync(0xffffffffu, o.y, base + 4);
        if (enter) {   // the bulge ahead is three rows on: these entries are settled
          x = csub(A[l * ld + l], s_shift[b]);
          y = A[(l + 1) * ld + l];
        }
        givens_group(x, y, ln, base, (act && kk + 1 < hi) || enter, &s_gc[nxt][b],
                     &s_gs[nxt][b]);
      } else if (wid < QR_CHAIN0) {
        // row rotation of bulge b on rows kk, kk+1, block columns c0..hi
        // other than kk, kk+1 (the bulge entry (kk+1, kk-1) becomes 0)
        int off[QR_BULGES + 1];
        off[0] = 0;
        for (int b = 0; b < QR_BULGES; ++b) {
          const int tb = t - 3 * b;
          const bool act = b < nb && tb >= 0 && tb <= w - 2;
          const int kk = l + tb;
          const int c0 = kk > l ? kk - 1 : l;
          off[b + 1] = off[b] + (act ? hi - c0 - 1 : 0);
        }
        for (int e = tid; e < off[QR_BULGES]; e += nbulk) {
          int b = 0;
          while (e >= off[b + 1]) ++b;
          const int kk = l + t - 3 * b;
          const int c0 = kk > l ? kk - 1 : l;
          const int u = e - off[b];
          const int j = c0 + u < kk ? c0 + u : c0 + u + 2;
          const double gc = s_gc[par][b];
          const double2 gs = s_gs[par][b], mgs = cneg(cconj(gs));
          const double2 a1 = A[kk * ld + j], a2 = A[(kk + 1) * ld + j];
          A[kk * ld + j] = cadd(cscale(gc, a1), cmul(gs, a2));
          A[(kk + 1) * ld + j] = (kk > l && j == kk - 1) ? make_double2(0.0, 0.0)
                                                         : cadd(cmul(mgs, a1), cscale(gc, a2));
        }
      }
      if (wid <= QR_CHAIN0) asm volatile("bar.sync 1, %0;" ::"n"(32 * (QR_CHAIN0 + 1)));
      // ---- phase 2: the column rotations of every active bulge on rows l..kk-1
      if (wid < QR_CHAIN0) {
        int off[QR_BULGES + 1];
        off[0] = 0;
        for (int b = 0; b < QR_BULGES; ++b) {
          const int tb = t - 3 * b;
          const bool act = b < nb && tb >= 0 && tb <= w - 2;
          off[b + 1] = off[b] + (act ? tb : 0);            // kk - l rows
        }
        for (int e = tid; e < off[QR_BULGES]; e += nbulk) {
          int b = 0;
          while (e >= off[b + 1]) ++b;
          const int kk = l + t - 3 * b;
          const int row = l + (e - off[b]);
          const double gc = s_gc[par][b];
          const double2 gs = s_gs[par][b], cgs = cconj(gs), ngs = cneg(gs);
          const double2 a1 = A[row * ld + kk], a2 = A[row * ld + kk + 1];
          A[row * ld + kk] = cadd(cscale(gc, a1), cmul(cgs, a2));
          A[row * ld + kk + 1] = cadd(cmul(ngs, a1), cscale(gc, a2));
        }
        asm volatile("bar.sync 2, %0;" ::"n"(32 * QR_CHAIN0));
      }
    }
    __syncthreads();
    if (tid == 0) t_rot += clock64() - t0;
  }
  if (clk != nullptr && tid == 0) {
    clk[8] = total;
    clk[9] = rotations;
    clk[10] = t_scan;
    clk[11] = t_rot;
    clk[12] = 0;
  }
  return 0;
}

// ----------------------------------------------------------------- eigenvalue estimates in FP32
//
// The cycle end needs every eigenvalue of the m x m harmonic Ritz matrix M
// (to keep the k smallest) and the eigenvectors of the kept ones.  Its FP64
// QR iteration is a chain of dependent FP64 instructions on one SM (64 clocks
// each on this GPU).  Instead: all eigenvalues to FP32 accuracy by QR
// iteration in FP32 (4-clock dependent arithmetic), then every estimate
// refined in FP64 by inverse iteration with a Rayleigh-quotient update, one
// CTA per estimate, on the original M.  The refined pairs are accepted only
// when each has a residual of the order of rounding, the values are pairwise
// distinct and they add up to the trace; otherwise the FP64 Hessenberg
// reduction and QR iteration (gmresdr_eig64_kernel) and inverse iteration on
// the Hessenberg form (harmonic_ritz_vector_kernel) give them.

__device__ __forceinline__ float2 fc_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fc_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fc_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fc_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 fc_scale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 fc_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float fc_abs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ float2 fc_div(float2 a, float2 b) {  // Smith's method
  if (fabsf(b.x) >= fabsf(b.y)) {
    const float r = b.y / b.x, d = b.x + r * b.y;
    return make_float2((a.x + r * a.y) / d, (a.y - r * a.x) / d);
  }
  const float r = b.x / b.y, d = b.y + r * b.x;
  return make_float2((r * a.x + a.y) / d, (r * a.y - a.x) / d);
}
__device__ __forceinline__ float2 fc_sqrt(float2 z) {  // principal square root
  const float r = hypotf(z.x, z.y);
  if (r == 0.f) return make_float2(0.f, 0.f);
  const float w = sqrtf(0.5f * (r + fabsf(z.x)));
  if (z.x >= 0.f) return make_float2(w, z.y / (2.f * w));
  return make_float2(fabsf(z.y) / (2.f * w), copysignf(w, z.y));
}

// Sum of a float over the block, result in every thread (fixed order).
__device__ float block_fsum_all(float v) {
  __shared__ float sh[32];
  __shared__ float res;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();  // sh and res may still be read by a previous call
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) res = t;
  }
  __syncthreads();
  return res;
}

// Largest value of a double over the block, result in every thread.
__device__ double block_dmax_all(double v) {
  __shared__ double sh[32];
  __shared__ double res;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, off));
    if (threadIdx.x == 0) res = t;
  }
  __syncthreads();
  return res;
}

// Householder reduction of the m x m FP32 matrix A (row-major, leading
// dimension ld) to upper Hessenberg form, reflectors not kept (only the
// eigenvalues are wanted).  As in the FP64 reduction, reflector j spans rows
// j+1 .. iend, iend the last nonzero row of column j (a shared atomic
// maximum, triple-buffered).  u: m scratch entries.  Block-wide.
__device__ void hess_reduce_f32(float2 *A, int m, int ld, float2 *u) {
  const int tid = threadIdx.x, bd = blockDim.x;
  __shared__ int s_end[3];
  if (tid < 3) s_end[tid] = 0;
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const int slot = j % 3;
    float part = 0.f;
    for (int i = j + 2 + tid; i < m; i += bd) {
      const float2 d = A[i * ld + j];
      part = fmaf(d.x, d.x, fmaf(d.y, d.y, part));
      if (d.x != 0.f || d.y != 0.f) atomicMax(&s_end[slot], i);
    }
    const float below = block_fsum_all(part);  // its barriers order the atomics
    const int iend = s_end[slot];
    if (tid == 0) s_end[(j + 2) % 3] = 0;
    if (below == 0.f) continue;
    const float2 al = A[(j + 1) * ld + j];
    const float aa = hypotf(al.x, al.y), nx = sqrtf(below + aa * aa);
    const float2 ph = aa > 0.f ? fc_scale(1.f / aa, al) : make_float2(1.f, 0.f);
    const float2 beta = fc_scale(-nx, ph);
    for (int i = j + 1 + tid; i <= iend; i += bd) u[i] = i == j + 1 ? fc_sub(al, beta) : A[i * ld + j];
    __syncthreads();
    const float tau = 1.f / (nx * (nx + aa));
    // from the left on columns j+1 .. m-1 (column j is set below)
    for (int c = j + 1 + tid; c < m; c += bd) {
      float2 sd = make_float2(0.f, 0.f);
      for (int i = j + 1; i <= iend; ++i) {
        const float2 ui = u[i], x = A[i * ld + c];
        sd.x = fmaf(ui.x, x.x, fmaf(ui.y, x.y, sd.x));
        sd.y = fmaf(ui.x, x.y, fmaf(-ui.y, x.x, sd.y));
      }
      const float2 f = fc_scale(tau, sd);
      for (int i = j + 1; i <= iend; ++i) A[i * ld + c] = fc_sub(A[i * ld + c], fc_mul(u[i], f));
    }
    __syncthreads();
    // from the right on every row; column j of rows j+1 .. iend becomes (beta, 0, ...)
    for (int r = tid; r < m; r += bd) {
      float2 sd = make_float2(0.f, 0.f);
      for (int i = j + 1; i <= iend; ++i) {
        const float2 ui = u[i], x = A[r * ld + i];
        sd.x = fmaf(x.x, ui.x, fmaf(-x.y, ui.y, sd.x));
        sd.y = fmaf(x.x, ui.y, fmaf(x.y, ui.x, sd.y));
      }
      const float2 f = fc_scale(tau, sd);
      for (int i = j + 1; i <= iend; ++i) A[r * ld + i] = fc_sub(A[r * ld + i], fc_mul(f, fc_conj(u[i])));
      if (r > j && r <= iend) A[r * ld + j] = r == j + 1 ? beta : make_float2(0.f, 0.f);
    }
    __syncthreads();
  }
}

// Eigenvalues of the upper Hessenberg FP32 matrix A by complex single-shift
// QR iteration (the shift: the eigenvalue of the trailing 2 x 2 block nearer
// its last diagonal entry; an exceptional shift every tenth sweep), rotations
// applied inside the active window [l, hi] only (only eigenvalues are
// wanted).  Threads 0 .. QR32_THREADS-1 call it (m <= QR32_THREADS): warp 0
// scans for deflation and forms the shift; then each rotation takes one
// matrix entry per thread, its row update and its column update separated
// by a barrier of these threads.  The rotation's inputs (the entries of
// column kk-1 in rows kk, kk+1) are passed through a double-buffered shared
// slot by the threads that computed them, so no thread reads an entry that
// another may be overwriting.  Eigenvalues end on the diagonal.  Returns 1
// (every calling thread) if 30 m sweeps did not converge.
constexpr int QR32_THREADS = 96;
static_assert(QR32_THREADS >= CE_MAXM && QR32_THREADS % 32 == 0, "one thread per entry of a row or column");

__device__ __forceinline__ void qr32_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(QR32_THREADS) : "memory");
}

__device__ int qr_eig_f32(float2 *A, int m, int ld, long long *clk) {
  const int t = threadIdx.x, lane = t & 31;
  __shared__ int s_l[2];
  __shared__ float2 s_xy[2][2];   // [step parity][x, y] of the next rotation
  __shared__ float s_anorm;
  if (t < 32) {
    float an = 0.f;
    for (int e = lane; e < m * m; e += 32) an = fmaxf(an, fc_abs1(A[(e / m) * ld + e % m]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) an = fmaxf(an, __shfl_xor_sync(0xffffffffu, an, off));
    if (lane == 0) s_anorm = an > 0.f ? an : 1.f;
  }
  int hi = m - 1, its = 0, total = 0, scan = 0;
  long long rotations = 0;
  qr32_bar();
  while (hi > 0) {
    if (total >= 30 * m) return 1;                   // uniform
    const int sp = scan & 1;
    ++scan;
    if (t < 32) {
      // l = the largest index in [1, hi] whose subdiagonal entry is negligible
      const float anorm = s_anorm;
      int l = 0;
      for (int q0 = 1; q0 <= hi; q0 += 32) {
        const int q = q0 + lane;
        bool neg = false;
        if (q <= hi) {
          float tst = fc_abs1(A[(q - 1) * ld + q - 1]) + fc_abs1(A[q * ld + q]);
          if (tst == 0.f) tst = anorm;
          neg = fc_abs1(A[q * ld + q - 1]) <= 1.1920929e-7f * tst;
        }
        const unsigned b = __ballot_sync(0xffffffffu, neg);
        if (b != 0u) l = q0 + 31 - __clz((int)b);
      }
      if (l != hi) {
        // shift, and the first rotation's inputs (read by every lane before
        // lane 0 writes anything)
        const float2 a0 = A[(hi - 1) * ld + hi - 1], b0 = A[(hi - 1) * ld + hi];
        const float2 c0 = A[hi * ld + hi - 1], d0 = A[hi * ld + hi];
        float2 mu;
        if ((its + 1) % 10 == 0) {
          mu = fc_add(d0, make_float2(fc_abs1(c0), 0.f));
        } else {
          const float2 p = fc_scale(0.5f, fc_sub(a0, d0));
          const float2 bc = fc_mul(b0, c0);
          float2 q = fc_sqrt(fc_add(fc_mul(p, p), bc));
          if (p.x * q.x + p.y * q.y < 0.f) q = fc_neg(q);
          const float2 den = fc_add(p, q);
          mu = (den.x == 0.f && den.y == 0.f) ? d0 : fc_sub(d0, fc_div(bc, den));
        }
        const float2 x = fc_sub(A[l * ld + l], mu), y = A[(l + 1) * ld + l];
        if (lane == 0) {
          s_xy[0][0] = x;
          s_xy[0][1] = y;
        }
      }
      if (lane == 0) {
        if (l > 0) A[l * ld + l - 1] = make_float2(0.f, 0.f);
        s_l[sp] = l;
      }
    }
    qr32_bar();
    const int l = s_l[sp];
    if (l == hi) {
      --hi;
      its = 0;
      continue;
    }
    ++its;
    ++total;
    for (int kk = l; kk < hi; ++kk) {
      const int p = (kk - l) & 1;
      const float2 x = s_xy[p][0], y = s_xy[p][1];
      // G = [[c, s], [-conj(s), c]], G [x; y] = [r; 0] (every thread the same)
      float c;
      float2 s;
      const float a2 = fmaf(x.x, x.x, x.y * x.y), b2 = fmaf(y.x, y.x, y.y * y.y);
      if (a2 == 0.f) {
        c = 0.f;
        s = make_float2(1.f, 0.f);
      } else {
        const float ra = rsqrtf(a2), rn = rsqrtf(a2 + b2);
        c = a2 * ra * rn;
        s = fc_scale(ra * rn, fc_mul(x, fc_conj(y)));
      }
      // rows kk, kk+1 on columns c0 .. hi (the bulge (kk+1, kk-1) becomes 0)
      const int c0 = kk > l ? kk - 1 : l;
      const int j = c0 + t;
      if (j <= hi) {
        const float2 a1 = A[kk * ld + j], a3 = A[(kk + 1) * ld + j];
        A[kk * ld + j] = fc_add(fc_scale(c, a1), fc_mul(s, a3));
        A[(kk + 1) * ld + j] = (kk > l && j == kk - 1)
                                   ? make_float2(0.f, 0.f)
                                   : fc_sub(fc_scale(c, a3), fc_mul(fc_conj(s), a1));
      }
      qr32_bar();
      // columns kk, kk+1 on rows l .. min(kk+2, hi); rows kk+1 and kk+2 of
      // column kk are the next rotation's inputs
      const int r1 = kk + 2 < hi ? kk + 2 : hi;
      const int r = l + t;
      if (r <= r1) {
        const float2 a1 = A[r * ld + kk], a3 = A[r * ld + kk + 1];
        const float2 n1 = fc_add(fc_scale(c, a1), fc_mul(fc_conj(s), a3));
        A[r * ld + kk] = n1;
        A[r * ld + kk + 1] = fc_sub(fc_scale(c, a3), fc_mul(s, a1));
        if (kk + 1 < hi && r > kk) s_xy[p ^ 1][r - kk - 1] = n1;
      }
      qr32_bar();
    }
    rotations += hi - l;
  }
  if (clk != nullptr && t == 0) {
    clk[8] = total;
    clk[9] = rotations;
  }
  return 0;
}

// ----------------------------------------------------------------- banded LU in FP64
//
// After a GMRES-DR restart H_m is upper Hessenberg except for its full
// leading (k+1) x k block, and so is M = H_m + |h|^2 f e_m^T (the last column
// of a Hessenberg matrix is full anyway).  Gaussian elimination with partial
// pivoting then only involves, in column j, rows j .. last[j], last[j] the
// largest last-nonzero row of columns 0 .. j (fill stays inside it).

// last[c] = max over columns c' <= c of the last row with a nonzero entry
// in column c' (at least c').  Block-wide; ends with a barrier.
__device__ void column_pattern(const double2 *A, int ld, int m, int *last) {
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    int r = m - 1;
    while (r > c) {
      const double2 v = A[r * ld + c];
      if (v.x != 0.0 || v.y != 0.0) break;
      --r;
    }
    last[c] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 1; c < m; ++c) last[c] = max(last[c], last[c - 1]);
  __syncthreads();
}

// In-place LU of A with partial pivoting inside the band: step j swaps rows
// j and piv[j] (columns > j; the multipliers of earlier columns stay in
// place) and eliminates rows j+1 .. last[j], keeping the multipliers below
// the diagonal and 1 / pivot in rp[j].  A pivot that is exactly zero is
// replaced by `tiny`.  Block-wide.
__device__ void lu_banded_block(double2 *A, int ld, int m, const int *last, int *piv, double2 *rp,
                                double tiny) {
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31;
  for (int j = 0; j < m; ++j) {
    const int lj = last[j];
    if (tid < 32) {
      // pivot: the largest |re| + |im| in rows j .. lj (ties: the smaller row)
      double best = -1.0;
      int bi = j;
      for (int i = j + lane; i <= lj; i += 32) {
        const double v = cabs1(A[i * ld + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      const int p = bi;
      double2 pv = A[p * ld + j];
      if (pv.x == 0.0 && pv.y == 0.0) pv = make_double2(tiny, 0.0);
      const double2 r = cdiv(make_double2(1.0, 0.0), pv);
      const double2 ujj = A[j * ld + j];
      __syncwarp();
      // multipliers of rows j+1 .. lj after the swap (row p receives row j)
      for (int i = j + 1 + lane; i <= lj; i += 32) A[i * ld + j] = cmul(i == p ? ujj : A[i * ld + j], r);
      if (lane == 0) {
        A[j * ld + j] = pv;
        piv[j] = p;
        rp[j] = r;
      }
    }
    __syncthreads();
    const int p = piv[j];
    if (p != j)
      for (int c = j + 1 + tid; c < m; c += bd) {
        const double2 t0 = A[j * ld + c];
        A[j * ld + c] = A[p * ld + c];
        A[p * ld + c] = t0;
      }
    __syncthreads();
    const int nr = lj - j, nc = m - j - 1;
    for (int e = tid; e < nr * nc; e += bd) {
      const int i = j + 1 + e / nc, c = j + 1 + e % nc;
      A[i * ld + c] = csub(A[i * ld + c], cmul(A[i * ld + j], A[j * ld + c]));
    }
    __syncthreads();
  }
}

// y <- A^{-1} y with the factors of lu_banded_block.  Every lane of one warp.
__device__ void lu_banded_solve_warp(const double2 *A, int ld, int m, const int *last,
                                     const int *piv, const double2 *rp, double2 *y) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j + 1 < m; ++j) {
    const int p = piv[j];
    double2 yj = y[j];
    if (p != j) {
      const double2 yp = y[p];
      __syncwarp();
      if (lane == 0) {
        y[p] = yj;
        y[j] = yp;
      }
      yj = yp;
      __syncwarp();
    }
    for (int i = j + 1 + lane; i <= last[j]; i += 32) y[i] = csub(y[i], cmul(A[i * ld + j], yj));
    __syncwarp();
  }
  for (int j = m - 1; j >= 0; --j) {
    const double2 yj = cmul(y[j], rp[j]);
    __syncwarp();
    if (lane == 0) y[j] = yj;
    for (int i = lane; i < j; i += 32) y[i] = csub(y[i], cmul(A[i * ld + j], yj));
    __syncwarp();
  }
}

// w <- A^{-dagger} w with the same factors.  Elimination wrote
// U = E_{m-2} S_{m-2} ... E_0 S_0 A (S_j the swap, E_j = I - l_j e_j^T), so
// A^dagger w' = w is solved by U^dagger g = w (forward substitution), then
// for j = m-2 .. 0: g_j -= l_j^dagger g (E_j^dagger), swap g_j, g_piv[j].
// Every lane of one warp.
__device__ void lu_banded_solve_adj_warp(const double2 *A, int ld, int m, const int *last,
                                         const int *piv, const double2 *rp, double2 *w) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < m; ++j) {
    const double2 wj = cmul(w[j], cconj(rp[j]));   // w_j / conj(u_jj)
    __syncwarp();
    if (lane == 0) w[j] = wj;
    for (int i = j + 1 + lane; i < m; i += 32) w[i] = csub(w[i], cmulc(A[j * ld + i], wj));
    __syncwarp();
  }
  for (int j = m - 2; j >= 0; --j) {
    double2 sd = make_double2(0.0, 0.0);
    for (int i = j + 1 + lane; i <= last[j]; i += 32) sd = cfmac(A[i * ld + j], w[i], sd);
    sd = warp_csum_all(sd);
    const int p = piv[j];
    const double2 wj = csub(w[j], sd), wp = w[p];
    __syncwarp();
    if (lane == 0) {
      w[j] = p != j ? wp : wj;
      if (p != j) w[p] = wj;
    }
    __syncwarp();
  }
}

// y <- y / ||y||_2.  Every lane of one warp.
__device__ void warp_normalize(double2 *y, int m) {
  const int lane = threadIdx.x & 31;
  double n2 = 0.0;
  for (int i = lane; i < m; i += 32) n2 += cnorm2(y[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, off);
  const double inv = n2 > 0.0 ? rsqrt(n2) : 1.0;
  for (int i = lane; i < m; i += 32) y[i] = cscale(inv, y[i]);
  __syncwarp();
}

__global__ void __launch_bounds__(CE_THREADS) gmresdr_cycle_end_kernel(CycleEndArgs a) {
  extern __shared__ double2 sm[];
  __shared__ int piv[CE_MAXM], last[CE_MAXM];
  __shared__ double2 rp[CE_MAXM];
  __shared__ int s_fail;
  const int m = a.m, k = a.k, tid = threadIdx.x, bd = blockDim.x;
  const int me = *a.m_eff;
  if (tid == 0) {
    a.flags[0] = 0;
    a.flags[1] = me < m ? 1 : 0;
    a.flags[2] = 0;
  }
#define STAMP(i) \
  if (a.clk != nullptr && tid == 0) a.clk[i] = clock64();
  STAMP(0)
  cycle_lsq(a, me, sm);
  STAMP(1)
  if (!a.do_restart || me < m) return;
  const double res = a.res[0];
  double2 *P = a.P;
  if (k == 0) {  // plain GMRES(m) restart: v_1 = V_{m+1} rho / ||rho||
    for (int i = tid; i <= m; i += bd)
      P[i] = res > 0.0 ? cscale(1.0 / res, a.rho[i]) : make_double2(0.0, 0.0);
    if (tid == 0) a.ck[0] = make_double2(res, 0.0);
    return;
  }
  // leading dimension = 1 mod 8 complex numbers: row-strided (column) access
  // by consecutive threads then walks all shared-memory banks
  const int ld = cyc_ld(m);
  double2 *A = sm;               // m x ld: H_m, then M
  double2 *Z = A + m * ld;       // m x ld: LU of H_m, then the FP32 copy of M
  double2 *v1 = Z + m * ld;      // m+1
  double2 *v2 = v1 + (m + 1);    // m+1
  // harmonic Ritz matrix M = H_m + |h_{m+1,m}|^2 f e_m^T with H_m^dagger f = e_m
  double hmax = 0.0;
  for (int e = tid; e < m * m; e += bd) {
    const int i = e / m, j = e % m;
    const double2 h = a.H[i * m + j];
    A[i * ld + j] = h;
    Z[i * ld + j] = h;
    hmax = fmax(hmax, cabs1(h));
  }
  for (int i = tid; i < m; i += bd) v1[i] = make_double2(i == m - 1 ? 1.0 : 0.0, 0.0);
  hmax = block_dmax_all(hmax);
  column_pattern(Z, ld, m, last);
  lu_banded_block(Z, ld, m, last, piv, rp, 2.220446049250313e-16 * (hmax > 0.0 ? hmax : 1.0));
  if (tid < 32) lu_banded_solve_adj_warp(Z, ld, m, last, piv, rp, v1);
  __syncthreads();
  STAMP(2)
  const double hh = cnorm2(a.H[m * m + m - 1]);
  for (int i = tid; i < m; i += bd) A[i * ld + m - 1] = cadd(A[i * ld + m - 1], cscale(hh, v1[i]));
  __syncthreads();
  // M to the work buffer (for the refinement and the FP64 fallback), with its
  // largest entry and its trace
  double2 *Mg = cyc_mat(a.work, m, k);
  double2 *est = cyc_est(a.work, m, k);
  double mmax = 0.0;
  double2 tpart = make_double2(0.0, 0.0);
  for (int e = tid; e < m * m; e += bd) {
    const int i = e / m, j = e % m;
    const double2 v = A[i * ld + j];
    Mg[e] = v;
    mmax = fmax(mmax, cabs1(v));
    if (i == j) tpart = cadd(tpart, v);
  }
  mmax = block_dmax_all(mmax);
  const double2 tr = block_csum_all(tpart);
  if (tid == 0) {
    est[3 * m] = make_double2(mmax, 0.0);
    est[3 * m + 1] = tr;
    if (!a.eig32) a.flags[2] = 3;      // FP64 iteration requested
  }
  if (!a.eig32) return;
  // FP32 copy scaled by a power of two (entries below 1 in magnitude)
  int ex = 0;
  frexp(mmax > 0.0 ? mmax : 1.0, &ex);
  const double sc = ldexp(1.0, -ex);
  float2 *A32 = reinterpret_cast<float2 *>(Z);
  for (int e = tid; e < m * m; e += bd) {
    const int i = e / m, j = e % m;
    const double2 v = A[i * ld + j];
    A32[i * ld + j] = make_float2((float)(v.x * sc), (float)(v.y * sc));
  }
  __syncthreads();
  hess_reduce_f32(A32, m, ld, reinterpret_cast<float2 *>(v2));
  STAMP(7)
  if (tid < QR32_THREADS) {
    const int f = qr_eig_f32(A32, m, ld, a.clk);
    if (tid == 0) s_fail = f;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) a.flags[2] = 1;      // estimates failed: the FP64 iteration runs
  } else {
    const double isc = 1.0 / sc;
    for (int i = tid; i < m; i += bd) {
      const float2 t = A32[i * ld + i];
      est[i] = make_double2((double)t.x * isc, (double)t.y * isc);
    }
  }
  STAMP(3)
#undef STAMP
}

// Refinement of eigenvalue estimate q of M (one CTA per estimate): two passes
// of inverse iteration, each an LU of M - sigma I (banded) and two solves from
// the previous vector (b = (1, ..., 1) at first), then sigma = y^dagger M y
// for the normalised y.  sigma starts at the FP32 estimate, accurate to
// ~1e-7 ||M||, so the second pass starts from a shift accurate to the square
// of that.  Writes the refined value, ||M y - sigma y|| / max |M_ij| and y.
constexpr int HRR_THREADS = 256;

__global__ void __launch_bounds__(HRR_THREADS) harmonic_ritz_refine_kernel(CycleEndArgs a) {
  extern __shared__ double2 sm[];
  __shared__ int piv[CE_MAXM], last[CE_MAXM];
  __shared__ double2 rp[CE_MAXM];
  const int m = a.m, k = a.k, q = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  if (*a.m_eff < m || a.flags[2] != 0) return;        // uniform
  const int ld = cyc_ld(m);
  double2 *U = sm;                   // m x ld
  double2 *y = U + m * ld;           // m
  double2 *z = y + m;                // m: M y
  const double2 *Mg = cyc_mat(a.work, m, k);
  double2 *est = cyc_est(a.work, m, k);
  const double anorm = est[3 * m].x > 0.0 ? est[3 * m].x : 1.0;
  double2 sigma = est[q];
  for (int pass = 0; pass < 2; ++pass) {
    for (int e = tid; e < m * m; e += bd) {
      const int i = e / m, j = e % m;
      const double2 v = Mg[e];
      U[i * ld + j] = i == j ? csub(v, sigma) : v;
    }
    if (pass == 0)
      for (int i = tid; i < m; i += bd) y[i] = make_double2(1.0, 0.0);
    __syncthreads();
    if (pass == 0) column_pattern(U, ld, m, last);
    lu_banded_block(U, ld, m, last, piv, rp, 2.220446049250313e-16 * anorm);
    if (tid < 32)
      for (int it = 0; it < 2; ++it) {
        lu_banded_solve_warp(U, ld, m, last, piv, rp, y);
        warp_normalize(y, m);
      }
    __syncthreads();
    double2 part = make_double2(0.0, 0.0);
    for (int i = tid; i < m; i += bd) {
      double2 sd = make_double2(0.0, 0.0);
      for (int j = 0; j < m; ++j) sd = cfma(Mg[i * m + j], y[j], sd);
      z[i] = sd;
      part = cfmac(y[i], sd, part);
    }
    sigma = block_csum_all(part);      // its barriers order z
  }
  double rpart = 0.0;
  for (int i = tid; i < m; i += bd) rpart += cnorm2(csub(z[i], cmul(sigma, y[i])));
  const double rn = sqrt(block_dsum_all(rpart));
  if (tid == 0) {
    est[m + q] = sigma;
    est[2 * m + q] = make_double2(rn / anorm, 0.0);
  }
  double2 *Y = cyc_vec(a.work, m, k);
  for (int i = tid; i < m; i += bd) Y[(size_t)q * m + i] = y[i];
}

// Order (|theta|, Re, Im, index) of the m values th: the ranks of the k
// smallest into sel.  Block-wide; ends with a barrier.
__device__ void select_smallest(const double2 *th, int m, int k, int *sel) {
  __shared__ double s_abs[CE_MAXM];
  for (int i = threadIdx.x; i < m; i += blockDim.x) s_abs[i] = cabs_(th[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double2 ti = th[i];
    const double ai = s_abs[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double2 tj = th[j];
      const double aj = s_abs[j];
      const bool less = aj < ai || (aj == ai && (tj.x < ti.x || (tj.x == ti.x && (tj.y < ti.y ||
                                                   (tj.y == ti.y && j < i)))));
      rank += less ? 1 : 0;
    }
    if (rank < k) sel[rank] = i;
  }
  __syncthreads();
}

// Acceptance of the refined pairs and selection of the k smallest |theta|:
// every relative residual <= 1e-10, the values pairwise farther apart than
// 1e-9 max |M_ij| (two estimates refined to the same eigenvalue would leave
// another one out), and their sum within 1e-8 m max |M_ij| of the trace.
// Then theta and the vectors of the kept values (columns of G).  Otherwise
// flags[2] = 2 and the FP64 QR iteration takes over.
__global__ void __launch_bounds__(CE_THREADS) harmonic_ritz_select_kernel(CycleEndArgs a) {
  __shared__ int sel[CE_MAXM];
  __shared__ int s_bad;
  const int m = a.m, k = a.k, tid = threadIdx.x, bd = blockDim.x;
  if (*a.m_eff < m || a.flags[2] != 0) return;        // uniform
  const double2 *est = cyc_est(a.work, m, k);
  const double2 *th = est + m;
  const double anorm = est[3 * m].x > 0.0 ? est[3 * m].x : 1.0;
  const double sep2 = (1e-9 * anorm) * (1e-9 * anorm);
  if (tid == 0) s_bad = 0;
  __syncthreads();
  double2 part = make_double2(0.0, 0.0);
  for (int i = tid; i < m; i += bd) {
    const double2 ti = th[i];
    bool bad = !(est[2 * m + i].x <= 1e-10);          // also a NaN residual
    for (int j = 0; j < m; ++j)
      if (j != i && cnorm2(csub(th[j], ti)) <= sep2) bad = true;
    if (bad) atomicOr(&s_bad, 1);
    part = cadd(part, ti);
  }
  const double2 sum = block_csum_all(part);           // its barriers order the atomics
  const bool bad = s_bad != 0 || !(cabs_(csub(sum, est[3 * m + 1])) <= 1e-8 * m * anorm);
  if (a.clk != nullptr && tid == 0) a.clk[12] = bad ? 1 : 0;
  if (bad) {
    if (tid == 0) a.flags[2] = 2;
    return;
  }
  select_smallest(th, m, k, sel);
  for (int q = tid; q < k; q += bd) a.theta[q] = th[sel[q]];
  double2 *G = a.work;
  const double2 *Y = cyc_vec(a.work, m, k);
  for (int e = tid; e < m * k; e += bd) {
    const int i = e / k, q = e % k;
    G[e] = Y[(size_t)sel[q] * m + i];
  }
}

// The FP64 path, when the estimates were not accepted: eigenvalues of M by
// the FP64 QR iteration (schur_block), the k smallest into theta; their
// vectors then come from harmonic_ritz_vector_kernel.
__global__ void __launch_bounds__(CE_THREADS) gmresdr_eig64_kernel(CycleEndArgs a) {
  extern __shared__ double2 sm[];
  __shared__ int sel[CE_MAXM];
  const int m = a.m, k = a.k, tid = threadIdx.x, bd = blockDim.x;
  if (*a.m_eff < m || a.flags[2] == 0) return;        // uniform
  const int ld = cyc_ld(m);
  double2 *A = sm;               // m x ld
  double2 *Z = A + m * ld;       // m x ld (unused here: the layout of the cycle end)
  double2 *v1 = Z + m * ld;      // m+1
  double2 *v2 = v1 + (m + 1);    // m+1
  const double2 *Mg = cyc_mat(a.work, m, k);
  for (int e = tid; e < m * m; e += bd) A[(e / m) * ld + e % m] = Mg[e];
  __syncthreads();
  // (schur_block writes H over M in the work buffer after reading it here)
  if (schur_block(A, m, ld, v2, nullptr, cyc_hess(a.work, m, k), cyc_zg(a.work, m, k),
                  cyc_tau(a.work, m, k))) {
    if (tid == 0) a.flags[0] = 1;
    return;
  }
  __syncthreads();
  __shared__ double2 s_th[CE_MAXM];
  for (int i = tid; i < m; i += bd) s_th[i] = A[i * ld + i];
  __syncthreads();
  select_smallest(s_th, m, k, sel);
  for (int q = tid; q < k; q += bd) a.theta[q] = s_th[sel[q]];
}

// (FP64 path) Eigenvector of the Hessenberg matrix H (global Hg, leading
// dimension m) for the selected harmonic Ritz value theta_q, one CTA per q: LU of
// H - theta I with partial pivoting between the two rows each column
// touches, two inverse-iteration solves from b = (1, ..., 1), then g = Z y
// (Z the product of the reduction's stored reflectors), into column q of G
// (m x k).  theta_q is an eigenvalue of H to rounding, so the solves
// amplify its eigenvector by the inverse of that rounding; a pivot that is
// exactly zero is replaced by eps ||H||.
constexpr int HRV_THREADS = 128;

__global__ void __launch_bounds__(HRV_THREADS) harmonic_ritz_vector_kernel(CycleEndArgs a) {
  extern __shared__ double2 sm[];
  const int m = a.m, k = a.k, q = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  if (*a.m_eff < m || a.flags[0] != 0 || a.flags[2] == 0) return;   // uniform: not needed
  const int ld = cyc_ld(m);
  double2 *U = sm;                   // m x ld: LU factors of H - theta I
  double2 *y = U + m * ld;           // m
  __shared__ double s_mult_re[CE_MAXM], s_mult_im[CE_MAXM];
  __shared__ int s_swap[CE_MAXM];
  __shared__ double s_red[HRV_THREADS / 32];
  const double2 *Hg = cyc_hess(a.work, m, k), *Ug = cyc_zg(a.work, m, k);
  const double2 theta = a.theta[q];
  double part = 0.0;
  for (int e = tid; e < m * m; e += bd) {
    const int i = e / m, j = e % m;
    double2 h = Hg[e];
    part = fmax(part, cabs1(h));
    if (i == j) h = csub(h, theta);
    U[i * ld + j] = h;
  }
  // ||H|| (largest entry), for the zero-pivot replacement
  for (int off = 16; off > 0; off >>= 1) part = fmax(part, __shfl_down_sync(0xffffffffu, part, off));
  if ((tid & 31) == 0) s_red[tid >> 5] = part;
  __syncthreads();
  double hn = 0.0;
  for (int w = 0; w < bd / 32; ++w) hn = fmax(hn, s_red[w]);
  const double tiny = 2.220446049250313e-16 * (hn > 0.0 ? hn : 1.0);
  // LU of the Hessenberg matrix: column j has nonzeros in rows <= j + 1
  for (int j = 0; j + 1 < m; ++j) {
    const double2 p0 = U[j * ld + j], p1 = U[(j + 1) * ld + j];
    const bool sw = cabs1(p1) > cabs1(p0);
    __syncthreads();
    if (sw)
      for (int c = j + tid; c < m; c += bd) {
        const double2 t0 = U[j * ld + c];
        U[j * ld + c] = U[(j + 1) * ld + c];
        U[(j + 1) * ld + c] = t0;
      }
    __syncthreads();
    double2 piv = U[j * ld + j];
    if (piv.x == 0.0 && piv.y == 0.0) piv = make_double2(tiny, 0.0);
    const double2 l = cdiv(U[(j + 1) * ld + j], piv);
    if (tid == 0) {
      s_swap[j] = sw ? 1 : 0;
      s_mult_re[j] = l.x;
      s_mult_im[j] = l.y;
      U[j * ld + j] = piv;
    }
    for (int c = j + 1 + tid; c < m; c += bd)
      U[(j + 1) * ld + c] = csub(U[(j + 1) * ld + c], cmul(l, U[j * ld + c]));
    __syncthreads();
  }
  if (tid == 0) {
    const double2 pl = U[(m - 1) * ld + m - 1];
    if (pl.x == 0.0 && pl.y == 0.0) U[(m - 1) * ld + m - 1] = make_double2(tiny, 0.0);
  }
  for (int i = tid; i < m; i += bd) y[i] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    // forward: apply the row swaps and multipliers (one thread, a short chain)
    if (tid == 0) {
      for (int j = 0; j + 1 < m; ++j) {
        if (s_swap[j]) {
          const double2 t0 = y[j];
          y[j] = y[j + 1];
          y[j + 1] = t0;
        }
        y[j + 1] = csub(y[j + 1], cmul(make_double2(s_mult_re[j], s_mult_im[j]), y[j]));
      }
    }
    __syncthreads();
    // back substitution, column oriented: y_j = y_j / u_jj, then y_i -= u_ij y_j
    for (int j = m - 1; j >= 0; --j) {
      const double2 yj = cdiv(y[j], U[j * ld + j]);
      __syncthreads();
      if (tid == 0) y[j] = yj;
      for (int i = tid; i < j; i += bd) y[i] = csub(y[i], cmul(U[i * ld + j], yj));
      __syncthreads();
    }
    // normalise (the first solve's vector can be very large)
    double n2 = 0.0, mx = 0.0;
    for (int i = tid; i < m; i += bd) mx = fmax(mx, cabs1(y[i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if ((tid & 31) == 0) s_red[tid >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < bd / 32; ++w) mx = fmax(mx, s_red[w]);
    __syncthreads();
    const double inv = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int i = tid; i < m; i += bd) {
      y[i] = cscale(inv, y[i]);
      n2 += cnorm2(y[i]);
    }
    for (int off = 16; off > 0; off >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, off);
    if ((tid & 31) == 0) s_red[tid >> 5] = n2;
    __syncthreads();
    n2 = 0.0;
    for (int w = 0; w < bd / 32; ++w) n2 += s_red[w];
    __syncthreads();
    const double inv2 = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
    for (int i = tid; i < m; i += bd) y[i] = cscale(inv2, y[i]);
    __syncthreads();
  }
  // g = Z y = H_0 (H_1 (... (H_{m-3} y))) by the stored reflectors, one
  // warp, then into column q of G
  if (tid < 32) {
    const double2 *taug = cyc_tau(a.work, m, k);
    for (int j = m - 3; j >= 0; --j) {
      const double2 ti = taug[j];
      if (ti.x == 0.0) continue;                       // uniform: no reflection
      const int iend = (int)ti.y;
      double2 sdot = make_double2(0.0, 0.0);
      for (int i = j + 1 + tid; i <= iend; i += 32) sdot = cfmac(Ug[(size_t)j * m + i], y[i], sdot);
      sdot = warp_csum_all(sdot);
      const double2 f = cscale(ti.x, sdot);
      for (int i = j + 1 + tid; i <= iend; i += 32)
        y[i] = csub(y[i], cmul(Ug[(size_t)j * m + i], f));
      __syncwarp();
    }
  }
  __syncthreads();
  double2 *G = a.work;
  for (int i = tid; i < m; i += bd) G[i * k + q] = y[i];
}

// The restarted basis from the harmonic Ritz vectors G (m x k, columns):
// P_k = QR of [G; 0], p_{k+1} = rho orthonormalised, Hbar_k, c_k.
__global__ void __launch_bounds__(CE_THREADS) gmresdr_restart_basis_kernel(CycleEndArgs a) {
  extern __shared__ double2 sm[];
  const int m = a.m, k = a.k, tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = bd >> 5;
  if (*a.m_eff < m || a.flags[0] != 0) return;        // uniform
  double2 *P = a.P;
  const int ldp = k + 1;
  double2 *v1 = sm;                  // m+1
  double2 *v2 = v1 + (m + 1);        // m+1
  double2 *G = a.work;
#define STAMP(i) \
  if (a.clk != nullptr && tid == 0) a.clk[i] = clock64();
  STAMP(4)
  // P_k = QR of [g_1..g_k; 0] by Gram-Schmidt applied twice; p_{k+1} from rho
  double2 *coef = v2;
  for (int c = 0; c <= k; ++c) {
    for (int i = tid; i <= m; i += bd)
      v1[i] = c < k ? (i < m ? G[i * k + c] : make_double2(0.0, 0.0)) : a.rho[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = wid; j < c; j += nw) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = lane; i <= m; i += 32) s = cfmac(P[i * ldp + j], v1[i], s);
        s = warp_csum_all(s);
        if (lane == 0) coef[j] = s;
      }
      __syncthreads();
      for (int i = tid; i <= m; i += bd) {
        double2 v = v1[i];
        for (int j = 0; j < c; ++j) v = csub(v, cmul(P[i * ldp + j], coef[j]));
        v1[i] = v;
      }
      __syncthreads();
    }
    double part2 = 0.0;
    for (int i = tid; i <= m; i += bd) part2 += cnorm2(v1[i]);
    const double nv = sqrt(block_dsum_all(part2));
    if (nv == 0.0 && tid == 0) a.flags[0] = 2;
    for (int i = tid; i <= m; i += bd) P[i * ldp + c] = nv > 0.0 ? cscale(1.0 / nv, v1[i]) : v1[i];
    __syncthreads();
  }
  STAMP(5)
  // T1 = Hbar_m P_k ((m+1) x k) in the work buffer, then Hk = P^dagger T1, ck = P^dagger rho
  double2 *T1 = a.work + (size_t)m * k;
  for (int e = tid; e < (m + 1) * k; e += bd) {
    const int i = e / k, b = e % k;
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < m; ++l) s = cfma(a.H[i * m + l], P[l * ldp + b], s);
    T1[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < (k + 1) * k; e += bd) {
    const int r = e / k, b = e % k;
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i <= m; ++i) s = cfmac(P[i * ldp + r], T1[i * k + b], s);
    a.Hk[e] = s;
  }
  for (int r = tid; r <= k; r += bd) {
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i <= m; ++i) s = cfmac(P[i * ldp + r], a.rho[i], s);
    a.ck[r] = s;
  }
  __syncthreads();
  STAMP(6)
#undef STAMP
}


size_t gmresdr_cycle_end_smem(int m) {
  const size_t lsq = (size_t)(m + 1) * cyc_ld(m) + 3 * (m + 1);
  const size_t eig = (size_t)2 * m * cyc_ld(m) + 2 * (m + 1);
  return (lsq > eig ? lsq : eig) * sizeof(double2);
}

cudaError_t launch_gmresdr_cycle_end(const CycleEndArgs &a, cudaStream_t s) {
  ProfLaunch prof_(PC_DENSE, s);
  if (a.m > CE_MAXM || a.m < 1 || a.k < 0 || a.k >= a.m) return cudaErrorInvalidValue;
  const size_t smem = gmresdr_cycle_end_smem(a.m);
  const size_t smem_vec = ((size_t)a.m * cyc_ld(a.m) + a.m) * sizeof(double2);
  const size_t smem_ref = ((size_t)a.m * cyc_ld(a.m) + 2 * a.m) * sizeof(double2);
  static thread_local int attr_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    const int big = (int)gmresdr_cycle_end_smem(CE_MAXM);
    e = cudaFuncSetAttribute(gmresdr_cycle_end_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gmresdr_eig64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(harmonic_ritz_vector_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(((size_t)CE_MAXM * cyc_ld(CE_MAXM) + CE_MAXM) * sizeof(double2)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(harmonic_ritz_refine_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(((size_t)CE_MAXM * cyc_ld(CE_MAXM) + 2 * CE_MAXM) * sizeof(double2)));
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  gmresdr_cycle_end_kernel<<<1, CE_THREADS, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || !a.do_restart || a.k == 0) return e;
  // every FP32 estimate refined in FP64 (one CTA each), acceptance and
  // selection; the FP64 QR iteration and its eigenvector kernel return at
  // once unless the estimates were rejected; then the restarted basis (all
  // return at once after a lucky breakdown or a failed eigenvalue iteration)
  harmonic_ritz_refine_kernel<<<a.m, HRR_THREADS, smem_ref, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  harmonic_ritz_select_kernel<<<1, CE_THREADS, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gmresdr_eig64_kernel<<<1, CE_THREADS, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  harmonic_ritz_vector_kernel<<<a.k, HRV_THREADS, smem_vec, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gmresdr_restart_basis_kernel<<<1, CE_THREADS, 2 * (a.m + 1) * sizeof(double2), s>>>(a);
  return cudaGetLastError();
}

}  // namespace wd
