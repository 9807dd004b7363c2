// Kernel-level declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include "wd_internal.h"

namespace wd {

struct LatticeGeom {
  int L[4];
  long long V;
  // Division by L[0], L[1], L[2] of site indices below 2^31 as a multiply
  // and a shift (Granlund and Montgomery, "Division by invariant integers
  // using multiplication", 1994): q = (n * dm) >> dsh with dsh = 31 + l,
  // l = ceil(log2 d), dm = floor(2^dsh / d) + 1, exact for n < 2^31.
  unsigned long long dm[3];
  int dsh[3];
};

enum { EPI_NONE = 0, EPI_DOT = 1, EPI_TSTT = 2 };

// Per-system solver status.  Kernels take a bit mask of the statuses they
// act on and skip every other system.
enum SysStatus {
  ST_ACTIVE = 0,       // iterating
  ST_RECURSIVE = 1,    // recursive residual below tol: check the true one
  ST_BREAKDOWN = 2,    // final
  ST_MAXITER = 3,      // final
  ST_DONE = 4,         // true residual below tol: final
  ST_FAILED = 5,       // true residual above tol, restarts used up: final
  ST_RESTART = 6,      // transient: restart from the true residual
  ST_IDLE = 7          // not part of this phase
};
constexpr unsigned M_ACTIVE = 1u << ST_ACTIVE;
constexpr unsigned M_RECURSIVE = 1u << ST_RECURSIVE;
constexpr unsigned M_RESTART = 1u << ST_RESTART;
constexpr unsigned M_ALL = 0xffffffffu;

// BiCGStab scalars of one system, device resident.
struct BicgScalars {
  double2 rho, rho_old, alpha, omega;
  double bnorm, rhat_norm, rnorm, true_rel, tol;
  int iters, max_iter, restarts, max_restarts;
  long long mvp, mvp_extra;
  // mixed solver only: tol is the target of the low-precision recursion;
  // tol_outer the FP64 true-residual target; delta > 0 selects restarted
  // refinement (inner target delta x the residual at the last restart)
  double tol_outer, delta;
};

LatticeGeom geom_of(const wd_context *h);
int wilson_blocks(const wd_context *h);

// Wilson apply with an optional fused reduction epilogue; blocks of systems
// whose status is not in `mask` do nothing (status == nullptr: all act).
cudaError_t launch_wilson_f64_epi(const wd_context *h, const double2 *in, double2 *out,
                                  int nrhs, int dagger, int epi, const double2 *aux,
                                  double *partial, const int *status, cudaStream_t s,
                                  unsigned mask = M_ACTIVE);

// ----------------------------------------------------------------- BLAS1
// Number of blocks (per system) every streaming kernel uses; fixed so that
// the reduction order, and hence every result, is reproducible.
int stream_blocks(long long n);

cudaError_t launch_bicg_update_p(double2 *p, const double2 *r, const double2 *v,
                                 const BicgScalars *sc, const int *status, long long n,
                                 int nrhs, cudaStream_t s);
cudaError_t launch_bicg_update_s(double2 *sv, const double2 *r, const double2 *v,
                                 const BicgScalars *sc, const int *status, long long n,
                                 int nrhs, cudaStream_t s);
cudaError_t launch_bicg_update_xr(double2 *x, double2 *r, const double2 *p, const double2 *sv,
                                  const double2 *t, const double2 *rhat, const BicgScalars *sc,
                                  const int *status, double *partial, long long n, int nrhs,
                                  cudaStream_t s);
// out = a - b, partial <- ||out||^2 ; systems in mask only
cudaError_t launch_sub_norm(double2 *out, const double2 *a, const double2 *b, const int *status,
                            unsigned mask, double *partial, long long n, int nrhs,
                            cudaStream_t s);
// partial <- ||a||^2 (and ||b||^2 when b != nullptr), all systems
cudaError_t launch_norms(const double2 *a, const double2 *b, double *partial, long long n,
                         int nrhs, cudaStream_t s);
// for systems in mask: rhat = r, p = 0, v = 0
cudaError_t launch_bicg_restart_vectors(double2 *rhat, const double2 *r, double2 *p,
                                        double2 *v, const int *status, unsigned mask,
                                        long long n, int nrhs, cudaStream_t s);

// Scalar finalizers (one block per system): reduce nb block partials of NQ
// doubles in a fixed order, then update the scalars and status.
enum FinKind { FIN_INIT, FIN_ALPHA, FIN_OMEGA, FIN_RHO, FIN_TRUE, FIN_ACTIVATE };
cudaError_t launch_bicg_finalize(int kind, const double *partial, int nb, BicgScalars *sc,
                                 int *status, double *hist, int hist_len, int nrhs,
                                 cudaStream_t s);

// ----------------------------------------------------------------- tall-skinny
// C[j][r] = sum_i conj(V[j][i]) * (g5 ? gamma5 W[r] : W[r])[i],  j < k, r < nrhs.
// launch_ts_dot writes ts_dot_blocks(n, k, nrhs) tiles of block partials to
// `partial` (k*nrhs complex per ... tile layout private to blas.cu, at most
// TS_MAX_BLOCKS * 16 complex); launch_ts_dot_finalize, given the same
// (n, k, nrhs), sums them in block order into C[j*ldc + r] and, when
// C2 != nullptr, also adds them to C2[j*ldc2 + r].
constexpr int TS_MAX_BLOCKS = 608;  // blocks of one ts_dot launch, all tiles
int ts_dot_blocks(long long n, int k, int nrhs);
inline size_t ts_dot_partial_count(long long n, int k, int nrhs) {
  return (size_t)ts_dot_blocks(n, k, nrhs) * 16;  // JT*RT = 16 for every tile shape
}
cudaError_t launch_ts_dot(const double2 *V, int k, const double2 *W, int nrhs, int g5,
                          long long n, double2 *partial, const int *status,
                          cudaStream_t s);
cudaError_t launch_ts_dot_finalize(const double2 *partial, long long n, int k, int nrhs,
                                   double2 *C, int ldc, double2 *C2, int ldc2,
                                   const int *status, cudaStream_t s);
// launch_ts_dot for one vector (nrhs = 1, no gamma5) in double-float
// arithmetic (about 48 bits, on the FP32 pipe): the first pass of CGS2, whose
// error the FP64 second pass removes.  V in the split form of
// launch_split_df (k vectors of n entries in each plane).  Its partials (at
// most ts_dot_partial_count(n, k, 1)) are summed by launch_ts_dot_df_finalize
// into C[j * ldc], j < k.
cudaError_t launch_ts_dot_df(const float2 *Vh, const float2 *Vl, int k, const double2 *w,
                             long long n, double2 *partial, const int *status, cudaStream_t s);
// vh[i] = (Re hi, Im hi), vl[i] = (Re lo, Im lo) of v[i] (hi: the top 24
// significant bits, lo: the next 24; an entry outside FP32's normal range
// gives zeros), i < count.
cudaError_t launch_split_df(const double2 *v, float2 *vh, float2 *vl, long long count,
                            const int *status, cudaStream_t s);
cudaError_t launch_ts_dot_df_finalize(const double2 *partial, long long n, int k, double2 *C,
                                      int ldc, const int *status, cudaStream_t s);
// OUT[c][i] = (beta_one ? IN[c][i] : 0) + sign * sum_j V[j][i] Y[j*ldy + c],
// c < ncol, kv <= 128.  OUT may alias IN (in-place update) but not V.
cudaError_t launch_ts_update(const double2 *V, int kv, const double2 *Y, int ldy, int ncol,
                             const double2 *IN, double2 *OUT, int beta_one, double sign,
                             long long n, const int *status, cudaStream_t s);

// w -= V h for the second classical Gram-Schmidt pass: FP32 products when
// ||h||^2 <= 1e-20 (||w0||^2 - ||hsum||^2) (part_w: Wilson-kernel partials,
// [3 b + 2] = block b's share of ||w0||^2; hsum: column of both passes'
// coefficients, stride ldh), else FP64 (blas.cu).
// Vh: nullptr, or V's high FP32 parts in the layout of launch_split_df (read
// instead of V on the FP32 path).
cudaError_t launch_ts_update_correction(const double2 *V, const float2 *Vh, int kv,
                                        const double2 *h, const double2 *hsum, int ldh,
                                        const double *part_w, int nbw, double2 *w, long long n,
                                        const int *status, cudaStream_t s);
// The same product on the tensor cores (exact-split BF16 emulation to FP64
// accuracy, tc_gemm.cu): kv <= 88, any ncol; OUT may alias IN but not V.
// scratch: ts_update_tc_scratch_bytes(kv, ncol, n) device bytes; *err (device)
// is set to 1 if a wait of the kernel gave up (never in normal operation).
bool ts_update_tc_supported(int kv, int ncol);
size_t ts_update_tc_scratch_bytes(int kv, int ncol, long long n);
cudaError_t launch_ts_update_tc(const double2 *V, int kv, const double2 *Y, int ldy, int ncol,
                                const double2 *IN, double2 *OUT, int beta_one, double sign,
                                long long n, void *scratch, int *err, cudaStream_t s);

// ----------------------------------------------------------------- Arnoldi helpers
// partial -> ||w||^2 reduced; H[(j+1)*ldh + j] = ||w||; v = w / ||w||;
// lucky breakdown when ||w|| <= lucky * ||w0|| sets *status = 1 and m_eff.
cudaError_t launch_arnoldi_normalize_finalize(const double *partial_w, int nb,
                                              const double *partial_w0, int nb0,
                                              double2 *H, int ldh, int j, double lucky,
                                              int *status, int *m_eff, cudaStream_t s);
// *dst = sqrt(sum_i partial[i*stride]) for i < nb (deterministic order)
cudaError_t launch_norm_finalize(const double *partial, int nb, int stride, double2 *dst,
                                 cudaStream_t s);
// v = w / Re(H[idx]) unless *status != 0
cudaError_t launch_scale_by_inverse_entry(double2 *v, const double2 *w, const double2 *H,
                                          int idx, long long n, const int *status,
                                          cudaStream_t s);

// ----------------------------------------------------------------- small dense (1 CTA)
// LU with partial pivoting of a k x k matrix (row-major), in place; piv[k].
// info[0] = 0 ok, 1 singular; info[1] bits of an estimate of cond (double).
cudaError_t launch_lu_factor(double2 *A, int k, int *piv, double *info, cudaStream_t s);
// Solve A Y = C for nrhs columns (C row-major k x nrhs, overwritten by Y).
cudaError_t launch_lu_solve(const double2 *LU, const int *piv, int k, double2 *C, int nrhs,
                            cudaStream_t s);

struct CycleEndArgs {
  const double2 *H;    // (m+1) x m row-major Hbar_m
  const double2 *c;    // m+1
  int m, k;
  const int *m_eff;    // Arnoldi columns actually built (lucky breakdown)
  double2 *d;          // m: least-squares solution
  double2 *rho;        // m+1: c - Hbar d
  double *res;         // [0] ||rho||
  double2 *P;          // (m+1) x (k+1) row-major
  double2 *Hk;         // (k+1) x k row-major: P^dagger Hbar P_k
  double2 *ck;         // k+1: P^dagger rho
  double2 *theta;      // k harmonic Ritz values
  int *flags;          // [0] eig failure, [1] lucky, [2] FP32 estimates rejected (FP64 path)
  double2 *work;       // scratch >= 2*(m+1)*(m+1) + 2*m*m + 4*m + 2 complex
  long long *clk;      // nullptr, or 10 slots: SM clock at phase boundaries, QR sweeps, rotations
  int do_restart;
  int eig32;           // 1: FP32 estimates refined in FP64 first, 0: FP64 QR iteration only
};
cudaError_t launch_gmresdr_cycle_end(const CycleEndArgs &a, cudaStream_t s);
size_t gmresdr_cycle_end_smem(int m);

// ----------------------------------------------------------------- even-odd (evenodd.cu)
// B full -> Bhat (even half); be, bo: scratch half vectors (nrhs each)
cudaError_t launch_eo_prepare(wd_context *h, const double2 *B, double2 *Bhat, double2 *be,
                              double2 *bo, int nrhs, cudaStream_t s);
// B full, Xe even half -> X full
cudaError_t launch_eo_reconstruct(wd_context *h, const double2 *B, const double2 *Xe, double2 *X,
                                  double2 *be, double2 *bo, int nrhs, cudaStream_t s);

// ----------------------------------------------------------------- gradients (force.cu)
cudaError_t launch_link_force(const wd_context *h, const double2 *lam, const double2 *x, double *f,
                              cudaStream_t s);
// partial[b] (stream_blocks(n) of them) of Re sum conj(lam) (x + i mu g5 x - ax)
cudaError_t launch_dkappa(const double2 *lam, const double2 *x, const double2 *ax, double mu,
                          long long n, double *partial, cudaStream_t s);
cudaError_t launch_gamma5(const double2 *in, double2 *out, long long n, cudaStream_t s);

}  // namespace wd
