// Internal solver drivers (FP64).  All vector arguments are device pointers
// in the boundary spinor layout; scratch comes from `ar`.
#pragma once

#include "wd_internal.h"

namespace wd {

// BiCGStab for nrhs systems A X = B.  R0 (optional) is the initial residual
// B - A X already computed by the caller.  hist_host (optional, nrhs x
// hist_len) receives ||r|| / ||b|| after every iteration.
int bicgstab_batched(wd_context *h, const double2 *B, double2 *X, const double2 *R0, int nrhs,
                     double tol, int max_iter, wd_stats *stats, cudaStream_t s,
                     double *hist_host, int hist_len, Arena &ar);

// W = A V, G = U^dagger W, LU factors of G (Sec. 2).
int deflation_build(wd_deflation_space *d, cudaStream_t s, Arena &ar);

// X += V y, R0 -= W y with y = G^{-1} U^dagger R0 (Sec. 2), nrhs systems.
int deflate_batched(wd_deflation_space *d, double2 *X, double2 *R0, int nrhs, cudaStream_t s,
                    Arena &ar);

// GMRES-DR(m,k).  hist_host (optional) receives ||rho|| / ||r0|| per cycle.
int gmresdr_run(wd_context *h, const double2 *b, double2 *x, int m, int k, double tol,
                int max_mv, double2 *V_out, double2 *Hbar_host, double2 *theta_host,
                wd_stats *stats, cudaStream_t s, double *hist_host, int hist_len, Arena &ar);

// Mixed precision: FP32 Krylov vectors (or, with h->mixed_bits = 16, p, v
// and t in FP16 storage), FP64 reliable updates every reliable_every
// iterations; R0 = B - A X on entry (FP64).
int bicgstab_mixed_batched(wd_context *h, const double2 *B, double2 *X, const double2 *R0,
                           int nrhs, double tol, int max_iter, int reliable_every,
                           wd_stats *stats, cudaStream_t s, Arena &ar);
int ensure_links32(wd_context *h, cudaStream_t s);
int ensure_links16(wd_context *h, cudaStream_t s);

// Sec. 4: A(mu_i) X_i = B for i < nshift in the given order, X = [nshift][nrhs][n],
// each shift projected over the earlier solutions when project != 0.
int tm_shifts_run(wd_context *h, const double2 *B, double2 *X, int nrhs, const double *mus,
                  int nshift, double tol, int max_iter, int project, int mixed,
                  wd_stats *stats, cudaStream_t s, Arena &ar);

}  // namespace wd
