// Wilson-Dirac operator A = 1 - kappa*D + i*mu*gamma5 in FP64 (Sec. 1, Sec. 4).
//
// One thread per (site, right-hand side).  Each of the 8 hops projects the
// neighbour spinor onto the 2-spin subspace of (1 -/+ gamma_mu), multiplies
// the two colour vectors by the link (or its adjoint) and rebuilds the
// lower spin pair from the upper one, so a hop costs 2 SU(3) mat-vecs
// instead of 4.  In the chiral basis gamma_mu = [[0, B], [B^dagger, 0]]
// with B = -i sigma_k (k = x, y, z) and B = 1 (t):
//   (1 - gamma_mu) psi = [h ; -B^dagger h],  h = psi_up - B psi_dn
//   (1 + gamma_mu) psi = [h ; +B^dagger h],  h = psi_up + B psi_dn
// A^dagger = gamma5 A(-mu) gamma5 (gamma5-hermiticity, Sec. 1) swaps the
// two projectors and flips the sign of mu.
//
// Optional fused epilogues write one block-partial (3 doubles) per block for
// the BiCGStab scalars: EPI_DOT   <aux, out>, <out, out>   (aux = r_hat)
//                       EPI_TSTT  <out, in>,  <out, out>
#include "cplx.cuh"
#include "wd_internal.h"
#include "kernels.cuh"
#include "spin.cuh"

namespace wd {

// chi = U h (ADJ = false) or U^dagger h (ADJ = true), two colour vectors
template <bool ADJ>
__device__ __forceinline__ void su3_mul(const double2 *__restrict__ u, const double2 (&h)[6],
                                        double2 (&c)[6]) {
  double2 m[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) m[i] = __ldg(u + i);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (ADJ)
          acc = cfmac(m[3 * b + a], h[3 * sp + b], acc);
        else
          acc = cfma(m[3 * a + b], h[3 * sp + b], acc);
      }
      c[3 * sp + a] = acc;
    }
  }
}

__device__ __forceinline__ void load_spinor(const double2 *__restrict__ p, double2 (&v)[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) v[i] = __ldg(p + i);
}

// out = init + U^dagger h: the product accumulates onto init in its FMA chain.
__device__ __forceinline__ void su3_adj_mul_acc(const double2 *__restrict__ u,
                                                const double2 (&h)[6], const double2 (&init)[6],
                                                double2 (&out)[6]) {
  double2 m[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) m[i] = __ldg(u + i);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      double2 acc = init[3 * sp + a];
#pragma unroll
      for (int b = 0; b < 3; ++b) acc = cfmac(m[3 * b + a], h[3 * sp + b], acc);
      out[3 * sp + a] = acc;
    }
}

// Both hops of direction MU.  With chi_f = U_MU(x) h_f (forward, projector
// sign S) and chi_b = U_MU(x - MU)^dagger h_b (backward, sign -S), the pair
// contributes [chi_f + chi_b ; S B^dagger (chi_f - chi_b)] (the lower spin
// pair of each hop is S or -S times B^dagger of its upper pair).  The sum is
// formed by starting chi_b's FMA chain at chi_f and the difference as
// 2 chi_f - sum, which saves the separate additions of the two hops; FIRST
// assigns instead of accumulating.
template <int MU, int S, bool FIRST>
__device__ __forceinline__ void hop_pair(const double2 *__restrict__ psi,
                                         const double2 *__restrict__ links, long long qf,
                                         long long s, long long qb, double2 (&acc)[12]) {
  double2 sum[6], dif[6];
  {
    double2 p[12], h[6], cf[6];
    load_spinor(psi + 12 * qf, p);
    project<MU, S>(p, h);
    su3_mul<false>(links + (s * 4 + MU) * 9, h, cf);
    load_spinor(psi + 12 * qb, p);
    project<MU, -S>(p, h);
    su3_adj_mul_acc(links + (qb * 4 + MU) * 9, h, cf, sum);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      dif[i] = make_double2(fma(2.0, cf[i].x, -sum[i].x), fma(2.0, cf[i].y, -sum[i].y));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 c0 = dif[a], c1 = dif[3 + a];
    // B^dagger applied to (c0, c1): rows 6+a and 9+a of the lower spin pair
    double2 l6, l9;
    if (MU == 0) {        // B^dagger = (i c1, i c0)
      l6 = cmuli(c1);
      l9 = cmuli(c0);
    } else if (MU == 1) { // (c1, -c0)
      l6 = c1;
      l9 = cneg(c0);
    } else if (MU == 2) { // (i c0, -i c1)
      l6 = cmuli(c0);
      l9 = cmulmi(c1);
    } else {              // (c0, c1)
      l6 = c0;
      l9 = c1;
    }
    if (S < 0) {
      l6 = cneg(l6);
      l9 = cneg(l9);
    }
    if (FIRST) {
      acc[a] = sum[a];
      acc[3 + a] = sum[3 + a];
      acc[6 + a] = l6;
      acc[9 + a] = l9;
    } else {
      acc[a] = cadd(acc[a], sum[a]);
      acc[3 + a] = cadd(acc[3 + a], sum[3 + a]);
      acc[6 + a] = cadd(acc[6 + a], l6);
      acc[9 + a] = cadd(acc[9 + a], l9);
    }
  }
}

template <bool DAG, int EPI>
__global__ void __launch_bounds__(128)
wilson_f64_kernel(const double2 *__restrict__ links, const double2 *__restrict__ in,
                  double2 *__restrict__ out, LatticeGeom g, double kappa, double mu,
                  const double2 *__restrict__ aux, double *__restrict__ partial,
                  const int *__restrict__ status, unsigned mask,
                  unsigned long long *__restrict__ sites) {
  const int r = blockIdx.y;
  if (status != nullptr && !((mask >> status[r]) & 1u)) return;  // uniform per block
  if (sites != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(sites, (unsigned long long)g.V);  // work accounting for the profiler
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double2 *psi = in + (long long)r * 12 * g.V;
  double red[3] = {0.0, 0.0, 0.0};
  if (s < g.V) {
    const Nbrs nb = neighbours(s, g.L);
    const long long xp = nb.up[0], xm = nb.dn[0], yp = nb.up[1], ym = nb.dn[1];
    const long long zp = nb.up[2], zm = nb.dn[2], tp = nb.up[3], tm = nb.dn[3];

    constexpr int F = DAG ? +1 : -1;  // projector sign on forward hops (-F on backward)
    double2 acc[12];
    hop_pair<0, F, true>(psi, links, xp, s, xm, acc);
    hop_pair<1, F, false>(psi, links, yp, s, ym, acc);
    hop_pair<2, F, false>(psi, links, zp, s, zm, acc);
    hop_pair<3, F, false>(psi, links, tp, s, tm, acc);

    double2 p[12];
    load_spinor(psi + 12 * s, p);
    const double tmu = DAG ? -mu : mu;
    double2 *o = out + (long long)r * 12 * g.V + 12 * s;
    const double2 *ax = (EPI == EPI_DOT) ? aux + (long long)r * 12 * g.V + 12 * s : nullptr;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 v;
      v.x = fma(-kappa, acc[c].x, p[c].x);
      v.y = fma(-kappa, acc[c].y, p[c].y);
      if (tmu != 0.0) {  // + i mu gamma5 psi, gamma5 = diag(1, 1, -1, -1)
        const double m = c < 6 ? tmu : -tmu;
        v.x = fma(-m, p[c].y, v.x);
        v.y = fma(m, p[c].x, v.y);
      }
      o[c] = v;
      if (EPI == EPI_DOT) {  // <aux, out> = sum conj(aux) out
        const double2 a = __ldg(ax + c);
        red[0] = fma(a.x, v.x, red[0]);
        red[0] = fma(a.y, v.y, red[0]);
        red[1] = fma(a.x, v.y, red[1]);
        red[1] = fma(-a.y, v.x, red[1]);
        red[2] = fma(v.x, v.x, red[2]);
        red[2] = fma(v.y, v.y, red[2]);
      } else if (EPI == EPI_TSTT) {  // <out, in> and <out, out>
        red[0] = fma(v.x, p[c].x, red[0]);
        red[0] = fma(v.y, p[c].y, red[0]);
        red[1] = fma(v.x, p[c].y, red[1]);
        red[1] = fma(-v.y, p[c].x, red[1]);
        red[2] = fma(v.x, v.x, red[2]);
        red[2] = fma(v.y, v.y, red[2]);
      }
    }
  }
  if (EPI != EPI_NONE) {
    constexpr int NQ = 3;
    block_sum<NQ>(red);
    if (threadIdx.x == 0) {
      double *dst = partial + ((long long)r * gridDim.x + blockIdx.x) * NQ;
#pragma unroll
      for (int q = 0; q < NQ; ++q) dst[q] = red[q];
    }
  }
}

LatticeGeom geom_of(const wd_context *h) {
  LatticeGeom g;
  for (int i = 0; i < 4; ++i) g.L[i] = h->dims[i];
  g.V = h->V;
  for (int i = 0; i < 3; ++i) {
    const unsigned long long d = (unsigned long long)h->dims[i];
    int l = 0;
    while ((1ULL << l) < d) ++l;
    g.dsh[i] = 31 + l;
    g.dm[i] = (1ULL << g.dsh[i]) / d + 1;
  }
  return g;
}

int eo_blocks(const wd_context *h);
cudaError_t launch_schur_f64_epi(const wd_context *h, const double2 *in, double2 *out, int nrhs,
                                 int dagger, int epi, const double2 *aux, double *partial,
                                 const int *status, cudaStream_t s, unsigned mask);

int wilson_blocks(const wd_context *h) {
  return h->eo ? eo_blocks(h) : (int)((h->V + 127) / 128);
}

cudaError_t launch_wilson_f64_epi(const wd_context *h, const double2 *in, double2 *out,
                                  int nrhs, int dagger, int epi, const double2 *aux,
                                  double *partial, const int *status, cudaStream_t s,
                                  unsigned mask) {
  if (h->eo)  // even-odd Schur operator on even half vectors
    return launch_schur_f64_epi(h, in, out, nrhs, dagger, epi, aux, partial, status, s, mask);
  dim3 grid(wilson_blocks(h), nrhs);
  LatticeGeom g = geom_of(h);
  ProfLaunch prof(PC_DSLASH, s);
  unsigned long long *cnt = prof_site_counter();
  if (dagger) {
    if (epi == EPI_DOT)
      wilson_f64_kernel<true, EPI_DOT><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
    else if (epi == EPI_TSTT)
      wilson_f64_kernel<true, EPI_TSTT><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
    else
      wilson_f64_kernel<true, EPI_NONE><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
  } else {
    if (epi == EPI_DOT)
      wilson_f64_kernel<false, EPI_DOT><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
    else if (epi == EPI_TSTT)
      wilson_f64_kernel<false, EPI_TSTT><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
    else
      wilson_f64_kernel<false, EPI_NONE><<<grid, 128, 0, s>>>(h->links, in, out, g, h->kappa, h->mu, aux, partial, status, mask, cnt);
  }
  return cudaGetLastError();
}

cudaError_t launch_wilson_f64(const wd_context *h, const double2 *in, double2 *out, int nrhs,
                              int dagger, cudaStream_t s) {
  return launch_wilson_f64_epi(h, in, out, nrhs, dagger, EPI_NONE, nullptr, nullptr, nullptr, s,
                               M_ALL);
}

}  // namespace wd
