/*
 * wd.h - C ABI of the GB300 deflated-BiCGStab library (libwd.so).
 *
 * Method: Abdel-Rehim, Morgan, Wilcox, "Deflated BiCGStab for linear
 * equations in QCD problems" (Lattice 2007).  GMRES-DR(m,k) takes the
 * first right-hand side and also yields k approximate right eigenvectors
 * V (Sec. 1).  Every later right-hand side gets the k x k
 * left-right projection (U^dagger A V) y = U^dagger r0, x0 += V y, with
 * U = gamma5 V from gamma5 A gamma5 = A^dagger, and then plain BiCGStab
 * (Sec. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice extents lat = {Lx, Ly, Lz, Lt}, all >= 1, periodic; volume
 *    V = Lx*Ly*Lz*Lt, vector length n = 12*V complex numbers.
 *  - Site index s = x + Lx*(y + Ly*(z + Lz*t)).
 *  - Spinor layout (boundary): complex128 (two doubles, re then im)
 *    psi[s][sigma][a], spin sigma = 0..3, colour a = 0..2, i.e. 192 bytes
 *    per site; a batch of nrhs spinors is nrhs such arrays back to back.
 *  - Gauge layout (boundary): complex128 U[s][mu][a][b], mu = 0..3 for
 *    x, y, z, t, 576 bytes per site.
 *  - Operator: A = 1 - kappa*D + i*mu*gamma5 with the Wilson hopping term
 *      (D psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu),
 *    chiral gamma basis, gamma5 = diag(1, 1, -1, -1).  mu = 0 is plain
 *    Wilson (Sec. 1); mu != 0 is the twisted-mass operator of Sec. 4.
 *  - Pointers named "device or host" are classified with
 *    cudaPointerGetAttributes: device (or managed) memory is used in
 *    place; host memory is staged through library-owned device buffers and
 *    the call then synchronises `stream` before it returns.  All other
 *    vector pointers must be device memory.  The caller owns every buffer
 *    it passes; the library never keeps a caller pointer after a call.
 *  - All GPU work is enqueued on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream).  Calls that report results to the host
 *    (solvers, stats) synchronise that stream.  One handle must not be
 *    used from two streams or threads at once.
 *  - Every function returns a status; nothing aborts or throws across the
 *    ABI.  On error, wd_last_error_detail() gives a one-line reason.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_context *wd_handle;
typedef struct wd_deflation_space *wd_deflation;
typedef struct CUstream_st *wd_stream;   /* identical to cudaStream_t */

enum wd_status {
  WD_OK = 0,
  WD_BAD_ARG = 1,              /* invalid size, pointer or parameter */
  WD_NOT_CONVERGED = 2,        /* tolerance not reached; x and stats still
                                  written (the paper's "F", Sec. 3) */
  WD_BREAKDOWN = 3,            /* a Krylov scalar vanished (rho, <r_hat,v>) */
  WD_SINGULAR_PROJECTION = 4,  /* U^dagger A V numerically singular */
  WD_TIMEOUT = 5,              /* a bounded device-side wait expired */
  WD_CUDA_ERROR = 6,           /* a CUDA call failed (see detail) */
  WD_OUT_OF_MEMORY = 7
};

/* Per-solve statistics.  mvp counts the matrix-vector products inside the
 * Krylov iteration, as the paper's tables do (Sec. 3, Sec. 4); mvp_extra
 * counts products spent on initial and true residuals and on setup. */
typedef struct {
  long long mvp;
  long long mvp_extra;
  int iters;         /* BiCGStab iterations (2 MVPs each) */
  int cycles;        /* GMRES-DR cycles */
  int restarts;      /* BiCGStab restarts from the true residual */
  int converged;     /* 1 if true residual <= tol */
  int breakdown;
  double rel_res;    /* recursive (BiCGStab) or least-squares (GMRES-DR)
                        residual norm / ||b|| */
  double true_rel_res;  /* ||b - A x|| / ||b|| recomputed at the end */
  double ms;         /* wall time of the call on `stream` */
} wd_stats;

/* ---------------------------------------------------------- operator */

/* Create a handle for A = 1 - kappa*D + i*mu*gamma5 on lattice `lat`.
 * links: device or host pointer, boundary gauge layout, V*4*9 complex128;
 * the handle copies it into its own device storage, so the caller may
 * free it afterwards.  Sec. 1 (Wilson matrix), Sec. 4 (twisted mass). */
int wd_create(const int lat[4], const void *links, double kappa, double mu,
              wd_handle *out);

/* Select the operator every vector entry point acts on: even_odd = 0 is A
 * on full vectors (n = 12 V); even_odd = 1 is the even-odd Schur complement
 * of Sec. 3 ("the even-odd preconditioned system"),
 *   A_hat = (1 + i mu gamma5) - kappa^2 D_eo (1 + i mu gamma5)^{-1} D_oe,
 * on even-site half vectors (n = 6 V complex128, site s of parity 0 stored at
 * s / 2).  Needs all extents even.  wd_apply, gmresdr_solve, the deflation
 * and D-BiCGStab entry points then use A_hat and half vectors (the mixed
 * solver with FP32 storage as well); tm_multishift_solve keeps full-lattice
 * vectors and solves each shift through A_hat (see there); the FP16
 * kernels, wd_gradients and wd_apply_f32_noalloc need even_odd = 0. */
int wd_set_operator(wd_handle h, int even_odd);

/* Even-odd helpers (handle in even-odd mode; device pointers; nrhs vectors):
 *  wd_eo_prepare:     Bhat = b_e + kappa D_eo (1 + i mu gamma5)^{-1} b_o
 *                     (B full, Bhat half).
 *  wd_eo_reconstruct: X = [x_e ; x_o], x_o = (1 + i mu gamma5)^{-1}
 *                     (b_o + kappa D_oe x_e) (B, X full, Xe half). */
int wd_eo_prepare(wd_handle h, const void *B, void *Bhat, int nrhs, wd_stream stream);
int wd_eo_reconstruct(wd_handle h, const void *B, const void *Xe, void *X, int nrhs,
                      wd_stream stream);

/* Change kappa and mu of an existing handle (no data movement). */
int wd_set_params(wd_handle h, double kappa, double mu);

/* out = A in (dagger = 0) or A^dagger in (dagger = 1) for nrhs spinors.
 * in, out: device pointers, boundary spinor layout, nrhs*n complex128
 * each, in != out (no aliasing).  Sec. 1. */
int wd_apply(wd_handle h, const void *in, void *out, int nrhs, int dagger,
             wd_stream stream);

/* ---------------------------------------------------------- solvers */

/* GMRES-DR(m,k) for A x = b (Sec. 1, Sec. 3; Morgan's deflated restarting).
 *  b:        device or host, n complex128.
 *  x:        device or host, n complex128; initial guess in, solution out.
 *  m, k:     subspace size and number of kept harmonic Ritz vectors,
 *            1 <= m <= 80, 0 <= k < m, m <= n.
 *  tol:      stop when the least-squares residual norm / ||b - A x0|| <= tol,
 *            tested at the end of each cycle.
 *  max_mv:   budget of counted MVPs (m for the first cycle, m-k later).
 *  V_out:    NULL or device, k*n complex128: orthonormal basis of the k
 *            harmonic Ritz vectors after the final restart (Sec. 2's V).
 *  Hbar_out: NULL or host, (k+1)*k complex128 row-major: A V = V_{k+1} Hbar.
 *  theta_out:NULL or host, k complex128: the kept harmonic Ritz values,
 *            ordered by (|theta|, Re, Im).
 *  stats:    NULL or host.
 * Returns WD_OK, WD_NOT_CONVERGED (x, V still written) or an error. */
int gmresdr_solve(wd_handle h, const void *b, void *x, int m, int k,
                  double tol, int max_mv, void *V_out, void *Hbar_out,
                  void *theta_out, wd_stats *stats, wd_stream stream);

/* Per-cycle history of the handle's last gmresdr_solve (Sec. 1, Sec. 3): the
 * least-squares residual norm / ||b - A x0|| at the end of each cycle, the
 * quantity the convergence test uses.  Copies min(cycles, len) values into
 * out (host, may be NULL when len = 0) and returns the number of cycles, or
 * -WD_BAD_ARG for a NULL handle or a negative len. */
int gmresdr_history(wd_handle h, double *out, int len);

/* Build the deflation space of Sec. 2 once for many right-hand sides:
 * W = A V (k MVPs), G = U^dagger A V and its LU factors.
 *  V: device, k*n complex128, orthonormal columns (e.g. from gmresdr_solve).
 *  U: NULL for U = gamma5 V (Sec. 1), else device, k*n complex128.
 * The handle copies V and U; 1 <= k <= 128. */
int wd_deflation_create(wd_handle h, const void *V, const void *U, int k,
                        wd_deflation *out, wd_stream stream);
void wd_deflation_destroy(wd_deflation d);

/* D-BiCGStab(k) for A X = B, nrhs right-hand sides batched (Sec. 2):
 * x0 = X on entry, r0 = B - A x0, y = (U^dagger A V)^{-1} U^dagger r0,
 * x0 += V y, then BiCGStab from x0 for every right-hand side at once,
 * each with its own scalars and convergence mask.  d = NULL gives plain
 * BiCGStab.  Convergence: ||r|| / ||b|| <= tol on the recursive residual,
 * then on the true residual (restart from it at most 3 times).
 *  B: device or host, nrhs*n complex128.  X: device or host, in/out.
 *  stats: NULL or host array of nrhs.
 * Returns WD_OK when every system converged, else WD_NOT_CONVERGED or
 * WD_BREAKDOWN (solutions and stats still written). */
int dbicgstab_solve_deflated(wd_handle h, wd_deflation d, const void *B,
                             void *X, int nrhs, double tol, int max_iter,
                             wd_stats *stats, wd_stream stream);

/* One-shot form: wd_deflation_create(V, U, k) + dbicgstab_solve_deflated +
 * destroy.  k = 0 (V = U = NULL) is plain BiCGStab. */
int dbicgstab_solve(wd_handle h, const void *B, void *X, int nrhs,
                    const void *V, const void *U, int k, double tol,
                    int max_iter, wd_stats *stats, wd_stream stream);

/* ---------------------------------------------------------- Sec. 4 shifts */

/* Twisted-mass systems A(mu_i) x_i = b for shifts mu_0, mu_1, ... solved
 * serially in the given order (Sec. 4; the paper prefers heaviest first).
 * With project != 0, before shift i every right-hand side is projected over
 * its own earlier solutions Q = [x_0 .. x_{i-1}]: Q^dagger A_i^dagger A_i Q d
 * = Q^dagger A_i^dagger b, x0 = Q d (i products per right-hand side, counted
 * in mvp_extra); then BiCGStab (FP64, or mixed = 1 for the FP32 iteration
 * with FP64 reliable updates) from x0 for all right-hand sides at once.
 * The handle's kappa is used for every shift; its mu is restored on return.
 *  B: device, nrhs*n complex128.  X: device, nshift*nrhs*n complex128,
 *  X[i][r] = solution of shift i, right-hand side r.  mus: host, nshift.
 *  stats: NULL or host array of nshift*nrhs, [i][r].
 * In even-odd mode B and X stay full-lattice vectors (n = 12 V): each
 * shift's source is prepared with that shift's mu, the Schur system is
 * solved (projected over the earlier shifts' even-site solutions; mixed = 1
 * needs FP32 storage) and the solution is reconstructed; tol applies to the
 * Schur residual. */
int tm_multishift_solve(wd_handle h, const void *B, void *X, int nrhs,
                        const double *mus, int nshift, double tol, int max_iter,
                        int project, int mixed, wd_stats *stats, wd_stream stream);

/* ---------------------------------------------------------- differentiation */

/* Not in the paper: gradients of a real loss through x = A^{-1} b.
 * LAM = A^{-dagger} G for nrhs right-hand sides, by gamma5-hermiticity
 * (Sec. 1): A^dagger = gamma5 A(-mu) gamma5, so LAM = gamma5 A(-mu)^{-1}
 * gamma5 G is one more D-BiCGStab solve with the same operator when mu = 0
 * (then the deflation space of A serves; for mu != 0 pass d = NULL or a
 * space built for -mu).  G, LAM: device, nrhs*n complex128. */
int dbicgstab_solve_adjoint(wd_handle h, wd_deflation d, const void *G, void *LAM,
                            int nrhs, double tol, int max_iter, wd_stats *stats,
                            wd_stream stream);

/* The same adjoint solve through the mixed-precision solver
 * (dbicgstab_solve_mixed: FP32 or FP16 iteration per wd_set_mixed_storage,
 * strategy per wd_set_mixed_restart, FP64 true residual <= tol). */
int dbicgstab_solve_adjoint_mixed(wd_handle h, wd_deflation d, const void *G, void *LAM,
                                  int nrhs, double tol, int max_iter, int reliable_every,
                                  wd_stats *stats, wd_stream stream);

/* For L real with dL = Re(g^dagger dx), x = A^{-1} b and lam = A^{-dagger} g:
 *  force  (NULL or device, V*4*8 double, [site][mu][a]): dL/domega for links
 *         moved as U_mu(s) -> exp(i omega_a lambda_a/2) U_mu(s) (Gell-Mann
 *         lambda_a), i.e. -kappa Im tr[lambda_a/2 (W1 - W2)], see force.cu;
 *  dkappa (NULL or host double): dL/dkappa = Re(lam^dagger D x).
 * (dL/db = lam itself.)  lam, x: device, n complex128 (one right-hand side). */
int wd_gradients(wd_handle h, const void *lam, const void *x, void *force,
                 double *dkappa, wd_stream stream);

/* ---------------------------------------------------------- mixed precision */

/* The same D-BiCGStab(k) solve with the BiCGStab iteration in FP32 storage
 * and arithmetic (vectors, links and Wilson apply) and FP64 reliable
 * updates: every `reliable_every` iterations, and when the FP32 recursive
 * residual reaches tol, x is accumulated in FP64 and r = b - A x is
 * recomputed with the FP64 operator.  The deflation projection (Sec. 2)
 * and the convergence test (FP64 true residual <= tol) are FP64.  Arguments
 * and results as dbicgstab_solve_deflated; reliable_every >= 1 (50 is the
 * workload's choice).  Not in the paper, which states no precision.  In
 * even-odd mode the iteration runs on the Schur operator (FP32 storage
 * only; B and X are the prepared even half vectors, as for the FP64 solver). */
int dbicgstab_solve_mixed(wd_handle h, wd_deflation d, const void *B, void *X,
                          int nrhs, double tol, int max_iter, int reliable_every,
                          wd_stats *stats, wd_stream stream);

/* out = A in (dagger = 0) or A^dagger in, computed by the FP32 kernel of
 * the mixed solver: in and out are FP64 device vectors in the boundary
 * layout, rounded to FP32 on entry and widened on exit.  In even-odd mode
 * (wd_set_operator(h, 1)) A is the Schur operator on even half vectors. */
int wd_apply_f32(wd_handle h, const void *in, void *out, int nrhs, int dagger,
                 wd_stream stream);

/* Autotuner of the FP32 Wilson kernel (not in the paper): times every launch
 * shape (R = 1, 2, 4 right-hand sides per thread, 64/128/256 threads per
 * block) for nrhs right-hand sides on this lattice and keeps the fastest in
 * the handle (nrhs >= 33 share one slot).  The mixed solver runs it on
 * first use of an nrhs; R, threads, ms (NULL or host) report the choice.
 * wd_set_f32_shape fixes a shape by hand (R = threads = 0: back to the
 * default, R = 1 and 128 threads). */
int wd_autotune_f32(wd_handle h, int nrhs, int *R, int *threads, float *ms,
                    wd_stream stream);
int wd_set_f32_shape(wd_handle h, int nrhs, int R, int threads);

/* Strategy of the mixed solver (not in the paper).  delta = 0 (default):
 * reliable updates -- every reliable_every iterations, and whenever the
 * low-precision recursive residual reaches tol, x and r = b - A x are
 * refreshed in FP64 and the BiCGStab recurrence continues with the replaced
 * residual.  0 < delta < 1: restarted refinement -- the low-precision
 * BiCGStab runs until its recursive residual has fallen by delta (or
 * max_inner iterations pass), then the FP64 residual is recomputed and the
 * recurrence restarts from it (r_hat = r, p = v = 0).  Reliable updates keep
 * the Krylov space across refreshes; restarted refinement converges where the
 * low-precision recurrence loses too much accuracy (e.g. twisted mass near
 * kappa_c), and restarting at least every few hundred iterations (the
 * handle's initial max_inner is 300) also ends BiCGStab stagnation there.
 * Applies to
 * dbicgstab_solve_mixed and tm_multishift_solve with mixed = 1; wd_stats
 * .restarts counts the restarts.  WD_BAD_ARG for delta outside [0, 1) or
 * max_inner < 1 with delta > 0. */
int wd_set_mixed_restart(wd_handle h, double delta, int max_inner);

/* Storage of the mixed solver's iteration (not in the paper): bits = 32
 * (default) keeps every Krylov vector in FP32; bits = 16 stores the links
 * and the three vectors the operator reads or writes (p, v, t) in FP16,
 * each site's 12 complex numbers scaled by that site's largest component
 * (one FP32 norm per site), while r, r_hat and the solution increment stay
 * FP32.  Arithmetic is FP32 either way and the reliable updates and the
 * convergence test are FP64, so the tolerance means the same; FP16 storage
 * halves the bytes of the operator and may take more iterations.  Applies
 * to dbicgstab_solve_mixed and to tm_multishift_solve with mixed = 1.
 * Returns WD_BAD_ARG for any other bits. */
int wd_set_mixed_storage(wd_handle h, int bits);

/* How the wide tall-skinny products V Y (complex128, V of kv <= 88 vectors,
 * Y kv x ncol with ncol >= 8) are computed: GMRES-DR's restart V_{k+1} =
 * V_{m+1} P_{k+1} (Sec. 1) and the projection's x0 += V y, r0 -= (A V) y
 * for batches of right-hand sides (Sec. 2).  tensor_cores = 1 (default):
 * on the tensor cores by exact-split emulation (each FP64 value as eight
 * 7-bit BF16 digits against its row's or column's largest exponent, every
 * partial sum exact in FP32; error of the order of an FP64 product's
 * rounding relative to row maximum x column maximum, results deterministic);
 * 0: FP64 fused multiply-adds on the CUDA cores.  Other values: WD_BAD_ARG. */
int wd_set_contraction(wd_handle h, int tensor_cores);

/* How GMRES-DR's restart finds the harmonic Ritz pairs (Sec. 1: the
 * eigenpairs of H_m + |h_{m+1,m}|^2 f e_m^T, the k of smallest modulus
 * kept).  fp32_estimates = 1 (default): every eigenvalue estimated in FP32
 * (Hessenberg reduction and shifted QR iteration), each refined in FP64 by
 * inverse iteration on the matrix itself, one thread block per estimate;
 * the refined pairs are used when each residual is at rounding level, the
 * values are pairwise distinct and they sum to the trace, otherwise the
 * next mode runs for that restart.  0: FP64 Hessenberg reduction and QR
 * iteration, eigenvectors by inverse iteration on the Hessenberg form.
 * Both give the pairs to FP64 rounding.  Other values: WD_BAD_ARG. */
int wd_set_eigen_estimates(wd_handle h, int fp32_estimates);

/* The tall-skinny product itself, without a handle (Sec. 1 restart, Sec. 2
 * projection updates): for c < ncol,
 *   OUT[c] = (beta_one ? IN[c] : 0) + sign * sum_{r < kv} V[r] Y[r*ldy + c],
 * V: kv vectors of n complex128 ([r][n]), Y: kv x ncol complex128 (row
 * stride ldy >= ncol), IN, OUT: ncol vectors of n; all device pointers.
 * OUT may alias IN, not V.  tensor_cores = 1: exact-split tensor-core form
 * (kv <= 88; error of the order of an FP64 product's rounding relative to
 * row maximum x column maximum), 0: FP64 FMAs (kv <= 128).  Allocates its
 * small scratch on `stream` (stream-ordered) and waits for the stream.
 * Returns WD_BAD_ARG (sizes, NULL pointers, host pointers), WD_TIMEOUT
 * (a wait inside the tensor-core kernel gave up) or WD_CUDA_ERROR. */
int wd_tsgemm(const void *V, int kv, const void *Y, int ldy, int ncol, const void *IN,
              void *OUT, int beta_one, double sign, long long n, int tensor_cores,
              wd_stream stream);

/* out = A in computed by the FP16-storage kernel: in and out are FP64 device
 * vectors in the boundary layout, rounded to the half format on entry
 * (per-site norm, see above) and widened on exit; FP32 arithmetic. */
int wd_apply_f16(wd_handle h, const void *in, void *out, int nrhs, int dagger,
                 wd_stream stream);

/* Autotuner and fixed shapes of the FP16-storage Wilson kernel, as
 * wd_autotune_f32 / wd_set_f32_shape (separate slots per handle). */
int wd_autotune_f16(wd_handle h, int nrhs, int *R, int *threads, float *ms,
                    wd_stream stream);
int wd_set_f16_shape(wd_handle h, int nrhs, int R, int threads);

/* ---------------------------------------------------------- no allocation */

/* The paper has no counterpart to this entry point: it is a service for
 * callers that cannot allocate device memory at the time they apply the
 * operator, e.g. a process that has handed all device memory to another
 * allocator (a framework's caching allocator, a fixed budget), or code that
 * must not synchronise the device (cudaMalloc/cudaFree may).  Same result as
 * wd_apply_f32 (FP64 device vectors in and out, FP32 arithmetic inside), but
 * the FP32 links and the two FP32 staging vectors live in one static device
 * array of WD_NOALLOC_SCRATCH_BYTES (64 MiB), held by every GPU that loads
 * the library until the process exits, and the call allocates nothing.
 *  - Needs V * (12 + 12 * nrhs) * 16 bytes <= WD_NOALLOC_SCRATCH_BYTES (e.g.
 *    16^4 with nrhs <= 4); larger requests return WD_BAD_ARG.
 *  - The FP32 links are rebuilt on every call (the array is shared), so at
 *    small nrhs a call costs more than wd_apply_f32.
 *  - The handle's device must be current.  The first call on each device
 *    looks up the array's device address and keeps it; make that call before
 *    any stream capture.  The address is that of the device's primary
 *    context (the CUDA runtime's): do not call this after resetting the
 *    device or from another context.
 *  - All calls share the array and keep the last call's contents (every
 *    region is rewritten before it is read); calls whose GPU work overlaps
 *    race, so order them yourself (one stream, or events). */
#define WD_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int wd_apply_f32_noalloc(wd_handle h, const void *in, void *out, int nrhs,
                         int dagger, wd_stream stream);

/* ---------------------------------------------------------- instrumentation */

/* Kernel timing, not part of the paper's method: CUDA events bracket every
 * launch of the enabled categories on the launching stream.  Categories:
 * 0 FP64 Wilson apply (dslash), 1 streaming vector kernels and scalar
 * finalizers, 2 tall-skinny products (V^dagger W, W += V Y), 3 single-block
 * dense kernels (LU, GMRES-DR cycle end), 4 FP32/FP16 Wilson apply of the
 * mixed solver, 5 its two per-iteration vector updates (p, and x with r).
 * While any category is on, the mixed solver launches its kernels one by
 * one instead of replaying CUDA graphs. */
typedef struct {
  long long launches[6];
  double ms[6];                        /* summed launch durations */
  long long dslash_site_updates;       /* lattice sites x systems the FP64
                                          dslash launches processed */
  long long dslash_low_site_updates;   /* the same for category 4 */
} wd_profile;

/* Enable the categories whose bit is set in mask (0 disables) and reset the
 * counters.  Timing adds two event records per launch of an enabled kind. */
int wd_profile_enable(wd_handle h, unsigned mask);
/* Resolve the recorded events (waits for them) and copy the counters. */
int wd_profile_read(wd_handle h, wd_profile *out);

/* FP64 fused multiply-add throughput of the current device, measured (not
 * part of the paper's method: the denominator of the FP64 kernels' roofline,
 * since every FP64 kernel of the solver path is bound by the FP64 pipe).
 * Launches 4 blocks of 256 threads per SM, each thread running 8 independent
 * FMA chains for `iters` steps, `reps` times after one warm-up launch, timed
 * by CUDA events on `stream` (blocks until done).  *tflops = 2 flops per FMA
 * / elapsed time; *ms (may be NULL) = time per launch.  1 <= iters <= 2^24,
 * 1 <= reps <= 1000, else WD_BAD_ARG. */
int wd_probe_fp64_peak(int iters, int reps, double *tflops, double *ms, wd_stream stream);

/* BF16 tensor-core throughput of the current device, measured (not part of
 * the paper's method: the rate the exact-split contraction of
 * wd_set_contraction draws on).  One CTA per SM issues `iters` tcgen05 MMAs
 * of M = 128, N = 256, K = 16 (BF16 in shared memory, FP32 accumulation in
 * tensor memory), `reps` launches after one warm-up, timed by CUDA events on
 * `stream`; *tflops counts 2 flops per multiply-add.  1 <= iters <= 2^20,
 * 1 <= reps <= 100, else WD_BAD_ARG; WD_TIMEOUT if a completion wait gave up. */
int wd_probe_bf16_mma_peak(int iters, int reps, double *tflops, double *ms, wd_stream stream);

/* ---------------------------------------------------------- housekeeping */

void wd_destroy(wd_handle h);
const char *wd_error_string(int status);
/* Copies the last error's one-line reason (this thread) into buf. Returns
 * its full length. */
int wd_last_error_detail(char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* WD_H */
