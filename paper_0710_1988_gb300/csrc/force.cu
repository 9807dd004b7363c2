// Gradient kernels of L = Re(eta^dagger x), x = A^{-1} b, given the adjoint
// lambda = A^{-dagger} eta (not in the paper: the differentiation growth
// line of the workload).
//
//  link force   dL/domega_{s,mu,a} = -kappa Im tr[T_a (W1 - W2)] for links
//               moved as U_mu(s) -> exp(i omega_a T_a) U_mu(s), T_a = lambda_a/2,
//               W1 = U_mu(s) sum_spin [(1 - gamma_mu) x(s+mu)] lambda(s)^dagger,
//               W2 = sum_spin [(1 + gamma_mu) x(s)] lambda(s+mu)^dagger U_mu(s)^dagger.
//  dL/dkappa    Re(lambda^dagger D x) with D x = (x + i mu gamma5 x - A x) / kappa.
//  gamma5       out = gamma5 in (diag(1, 1, -1, -1) in spin).
#include "cplx.cuh"
#include "kernels.cuh"
#include "spin.cuh"
#include "wd_internal.h"

namespace wd {

// acc = (1 + S gamma_mu) p, through the projector structure of spin.cuh
template <int MU, int S>
__device__ __forceinline__ void spin_proj_full(const double2 (&p)[12], double2 (&o)[12]) {
  double2 h[6];
  project<MU, S>(p, h);
#pragma unroll
  for (int i = 0; i < 12; ++i) o[i] = make_double2(0.0, 0.0);
  reconstruct<MU, S>(o, h);
}

template <int MU>
__device__ void force_dir(const double2 *__restrict__ links, const double2 *__restrict__ lam,
                          const double2 *__restrict__ x, long long s, long long sp, double kappa,
                          double *__restrict__ f) {
  double2 xs[12], xp[12], ls[12], lp[12], phi[12], psi[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    xs[i] = x[12 * s + i];
    xp[i] = x[12 * sp + i];
    ls[i] = lam[12 * s + i];
    lp[i] = lam[12 * sp + i];
  }
  spin_proj_full<MU, -1>(xp, phi);  // (1 - gamma_mu) x(s+mu)
  spin_proj_full<MU, +1>(xs, psi);  // (1 + gamma_mu) x(s)
  double2 o1[9], o2[9], u[9];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
#pragma unroll
      for (int sg = 0; sg < 4; ++sg) {
        a = cfma(phi[3 * sg + c], cconj(ls[3 * sg + d]), a);
        b = cfma(psi[3 * sg + c], cconj(lp[3 * sg + d]), b);
      }
      o1[3 * c + d] = a;
      o2[3 * c + d] = b;
    }
#pragma unroll
  for (int i = 0; i < 9; ++i) u[i] = links[(s * 4 + MU) * 9 + i];
  double2 M[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 w1 = make_double2(0.0, 0.0), w2 = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        w1 = cfma(u[3 * i + k], o1[3 * k + j], w1);        // (U o1)_ij
        w2 = cfma(o2[3 * i + k], cconj(u[3 * j + k]), w2);  // (o2 U^dagger)_ij
      }
      M[3 * i + j] = csub(w1, w2);
    }
  // tr(lambda_a M) / 2 for the Gell-Mann matrices; keep -kappa * Im
  const double2 m00 = M[0], m01 = M[1], m02 = M[2], m10 = M[3], m11 = M[4], m12 = M[5];
  const double2 m20 = M[6], m21 = M[7], m22 = M[8];
  double2 t[8];
  t[0] = cadd(m01, m10);
  t[1] = cmuli(csub(m01, m10));                  // -i m10 + i m01
  t[2] = csub(m00, m11);
  t[3] = cadd(m02, m20);
  t[4] = cmuli(csub(m02, m20));
  t[5] = cadd(m12, m21);
  t[6] = cmuli(csub(m12, m21));
  t[7] = cscale(0.57735026918962576451, csub(cadd(m00, m11), cscale(2.0, m22)));
  double *out = f + (s * 4 + MU) * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) out[a] = -kappa * 0.5 * t[a].y;
}

__global__ void __launch_bounds__(128)
link_force_kernel(const double2 *__restrict__ links, const double2 *__restrict__ lam,
                  const double2 *__restrict__ x, LatticeGeom g, double kappa,
                  double *__restrict__ f) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const Nbrs nb = neighbours(s, g.L);
  force_dir<0>(links, lam, x, s, nb.up[0], kappa, f);
  force_dir<1>(links, lam, x, s, nb.up[1], kappa, f);
  force_dir<2>(links, lam, x, s, nb.up[2], kappa, f);
  force_dir<3>(links, lam, x, s, nb.up[3], kappa, f);
}

cudaError_t launch_link_force(const wd_context *h, const double2 *lam, const double2 *x, double *f,
                              cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  link_force_kernel<<<(unsigned)((h->V + 127) / 128), 128, 0, s>>>(h->links, lam, x, geom_of(h),
                                                                  h->kappa, f);
  return cudaGetLastError();
}

// partial <- Re sum conj(lam) (x + i mu gamma5 x - ax) (block partials, NQ = 1)
__global__ void __launch_bounds__(256)
dkappa_kernel(const double2 *__restrict__ lam, const double2 *__restrict__ x,
              const double2 *__restrict__ ax, double mu, long long n,
              double *__restrict__ partial) {
  double red[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 xv = x[i];
    const double g = (i % 12) < 6 ? mu : -mu;
    const double2 dx = make_double2(xv.x - g * xv.y - ax[i].x, xv.y + g * xv.x - ax[i].y);
    const double2 l = lam[i];
    red[0] = fma(l.x, dx.x, fma(l.y, dx.y, red[0]));
  }
  block_sum<1>(red);
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

cudaError_t launch_dkappa(const double2 *lam, const double2 *x, const double2 *ax, double mu,
                          long long n, double *partial, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  dkappa_kernel<<<stream_blocks(n), 256, 0, s>>>(lam, x, ax, mu, n, partial);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
gamma5_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = (i % 12) < 6 ? v : make_double2(-v.x, -v.y);
  }
}

cudaError_t launch_gamma5(const double2 *in, double2 *out, long long n, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  gamma5_kernel<<<stream_blocks(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace wd
