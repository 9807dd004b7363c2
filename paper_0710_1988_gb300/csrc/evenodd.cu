// Even-odd preconditioned Wilson operator (Sec. 3 solves "the even-odd
// preconditioned system"; the paper does not write it out):
//
//   A_hat x_e = (1 + i mu gamma5) x_e - kappa^2 D_eo A_oo^{-1} D_oe x_e,
//   A_oo^{-1} = (1 - i mu gamma5) / (1 + mu^2),
//   b_hat = b_e + kappa D_eo A_oo^{-1} b_o,   x_o = A_oo^{-1} (b_o + kappa D_oe x_e).
//
// Half-lattice vectors hold the sites of one parity, compact index s / 2
// (Lx even: the two sites of an x-pair have opposite parities), in the
// boundary spinor layout.  A_hat^dagger = gamma5 A_hat(-mu) gamma5: the hop
// kernels swap projectors and the diagonal terms flip mu, as in dslash.cu.
#include <cmath>

#include "cplx.cuh"
#include "kernels.cuh"
#include "spin.cuh"
#include "wd_internal.h"

namespace wd {

enum { EO_SCHUR1 = 0, EO_SCHUR2 = 1, EO_AXPY = 2 };

template <bool ADJ>
__device__ __forceinline__ void su3_mul_eo(const double2 *__restrict__ u, const double2 (&h)[6],
                                           double2 (&c)[6]) {
  double2 m[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) m[i] = __ldg(u + i);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        acc = ADJ ? cfmac(m[3 * b + a], h[3 * sp + b], acc) : cfma(m[3 * a + b], h[3 * sp + b], acc);
      c[3 * sp + a] = acc;
    }
}

template <int MU, int S, bool ADJ>
__device__ __forceinline__ void hop_eo(const double2 *__restrict__ src, const double2 *__restrict__ links,
                                       long long q, long long ql, double2 (&acc)[12]) {
  double2 p[12], h[6], c[6];
  const double2 *ps = src + 12 * (q >> 1);
#pragma unroll
  for (int i = 0; i < 12; ++i) p[i] = __ldg(ps + i);
  project<MU, S>(p, h);
  su3_mul_eo<ADJ>(links + (ql * 4 + MU) * 9, h, c);
  reconstruct<MU, S>(acc, c);
}

// out (parity pout, compact) from h = D_{pout, 1-pout} src:
//  EO_SCHUR1: out = (1 - i mu g5) h / (1 + mu^2)
//  EO_SCHUR2: out = (1 + i mu g5) same - kappa^2 h   (+ reduction epilogue)
//  EO_AXPY:   out = same + kappa h
template <bool DAG, int MODE, int EPI>
__global__ void __launch_bounds__(128)
wilson_eo_kernel(const double2 *__restrict__ links, const double2 *__restrict__ src,
                 const double2 *__restrict__ same, double2 *__restrict__ out, LatticeGeom g,
                 int pout, double kappa, double mu, double inv_1mu2,
                 const double2 *__restrict__ aux,
                 double *__restrict__ partial, const int *__restrict__ status, unsigned mask,
                 unsigned long long *__restrict__ sites) {
  const int r = blockIdx.y;
  if (status != nullptr && !((mask >> status[r]) & 1u)) return;
  if (sites != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(sites, (unsigned long long)g.V);  // two half hops = one full MVP of work
  const long long Vh = g.V / 2;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long off = (long long)r * 12 * Vh;
  double red[3] = {0.0, 0.0, 0.0};
  if (i < Vh) {
    // full site of parity pout in the x-pair (2i, 2i+1)
    const long long s0 = 2 * i;
    long long t1 = s0 / g.L[0];
    const int y = (int)(t1 % g.L[1]);
    t1 /= g.L[1];
    const int z = (int)(t1 % g.L[2]);
    const int t = (int)(t1 / g.L[2]);
    const long long s = s0 + (((y + z + t) & 1) != pout ? 1 : 0);
    const Nbrs nb = neighbours(s, g.L);
    constexpr int F = DAG ? +1 : -1;
    constexpr int B = -F;
    const double2 *sr = src + off;
    double2 acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = make_double2(0.0, 0.0);
    hop_eo<0, F, false>(sr, links, nb.up[0], s, acc);
    hop_eo<0, B, true>(sr, links, nb.dn[0], nb.dn[0], acc);
    hop_eo<1, F, false>(sr, links, nb.up[1], s, acc);
    hop_eo<1, B, true>(sr, links, nb.dn[1], nb.dn[1], acc);
    hop_eo<2, F, false>(sr, links, nb.up[2], s, acc);
    hop_eo<2, B, true>(sr, links, nb.dn[2], nb.dn[2], acc);
    hop_eo<3, F, false>(sr, links, nb.up[3], s, acc);
    hop_eo<3, B, true>(sr, links, nb.dn[3], nb.dn[3], acc);
    const double tmu = DAG ? -mu : mu;
    double2 *o = out + off + 12 * i;
    double2 sm[12];
    if (MODE != EO_SCHUR1) {
#pragma unroll
      for (int c = 0; c < 12; ++c) sm[c] = __ldg(same + off + 12 * i + c);
    }
    const double inv = inv_1mu2;  // 1 / (1 + mu^2), formed once on the host
    const double k2 = kappa * kappa;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double gm = c < 6 ? tmu : -tmu;  // mu * gamma5 entry
      double2 v;
      if (MODE == EO_SCHUR1) {           // (1 - i mu g5) h / (1 + mu^2)
        v.x = (acc[c].x + gm * acc[c].y) * inv;
        v.y = (acc[c].y - gm * acc[c].x) * inv;
      } else if (MODE == EO_SCHUR2) {    // (1 + i mu g5) same - kappa^2 h
        v.x = fma(-k2, acc[c].x, sm[c].x - gm * sm[c].y);
        v.y = fma(-k2, acc[c].y, sm[c].y + gm * sm[c].x);
      } else {                           // same + kappa h
        v.x = fma(kappa, acc[c].x, sm[c].x);
        v.y = fma(kappa, acc[c].y, sm[c].y);
      }
      o[c] = v;
      if (EPI == EPI_DOT) {
        const double2 a = __ldg(aux + off + 12 * i + c);
        red[0] = fma(a.x, v.x, fma(a.y, v.y, red[0]));
        red[1] = fma(a.x, v.y, fma(-a.y, v.x, red[1]));
        red[2] = fma(v.x, v.x, fma(v.y, v.y, red[2]));
      } else if (EPI == EPI_TSTT) {
        red[0] = fma(v.x, sm[c].x, fma(v.y, sm[c].y, red[0]));
        red[1] = fma(v.x, sm[c].y, fma(-v.y, sm[c].x, red[1]));
        red[2] = fma(v.x, v.x, fma(v.y, v.y, red[2]));
      }
    }
  }
  if (EPI != EPI_NONE) {
    block_sum<3>(red);
    if (threadIdx.x == 0) {
      double *d = partial + ((long long)r * gridDim.x + blockIdx.x) * 3;
      d[0] = red[0];
      d[1] = red[1];
      d[2] = red[2];
    }
  }
}

int eo_blocks(const wd_context *h) { return (int)((h->V / 2 + 127) / 128); }

template <bool DAG>
static void launch_eo(int mode, int epi, dim3 grid, cudaStream_t s, const wd_context *h,
                      const double2 *src, const double2 *same, double2 *out, int pout,
                      const double2 *aux, double *partial, const int *status, unsigned mask,
                      unsigned long long *cnt) {
  const LatticeGeom g = geom_of(h);
  const double inv = 1.0 / std::fma(h->mu, h->mu, 1.0);  // as the device contracts it
#define EO_LAUNCH(M, E)                                                                   \
  wilson_eo_kernel<DAG, M, E><<<grid, 128, 0, s>>>(h->links, src, same, out, g, pout, h->kappa, \
                                                   h->mu, inv, aux, partial, status, mask, cnt)
  if (mode == EO_SCHUR1) EO_LAUNCH(EO_SCHUR1, EPI_NONE);
  else if (mode == EO_AXPY) EO_LAUNCH(EO_AXPY, EPI_NONE);
  else if (epi == EPI_DOT) EO_LAUNCH(EO_SCHUR2, EPI_DOT);
  else if (epi == EPI_TSTT) EO_LAUNCH(EO_SCHUR2, EPI_TSTT);
  else EO_LAUNCH(EO_SCHUR2, EPI_NONE);
#undef EO_LAUNCH
}

static int ensure_eo_tmp(wd_context *h, int nrhs) {
  const size_t need = (size_t)nrhs * 12 * (h->V / 2);
  if (h->eo_tmp_cap >= need) return 0;
  if (h->eo_tmp) cudaFree(h->eo_tmp);
  h->eo_tmp = nullptr;
  h->eo_tmp_cap = 0;
  if (cudaMalloc(&h->eo_tmp, need * sizeof(double2)) != cudaSuccess) return 1;
  h->eo_tmp_cap = need;
  return 0;
}

// out = A_hat in (or A_hat^dagger in), both even half vectors, with the
// reduction epilogues of the full operator on the second half hop.
cudaError_t launch_schur_f64_epi(const wd_context *hc, const double2 *in, double2 *out, int nrhs,
                                 int dagger, int epi, const double2 *aux, double *partial,
                                 const int *status, cudaStream_t s, unsigned mask) {
  wd_context *h = const_cast<wd_context *>(hc);
  if (ensure_eo_tmp(h, nrhs)) return cudaErrorMemoryAllocation;
  ProfLaunch prof(PC_DSLASH, s);
  unsigned long long *cnt = prof_site_counter();
  dim3 grid(eo_blocks(h), nrhs);
  if (dagger) {
    launch_eo<true>(EO_SCHUR1, EPI_NONE, grid, s, h, in, nullptr, h->eo_tmp, 1, nullptr, nullptr, status, mask, nullptr);
    launch_eo<true>(EO_SCHUR2, epi, grid, s, h, h->eo_tmp, in, out, 0, aux, partial, status, mask, cnt);
  } else {
    launch_eo<false>(EO_SCHUR1, EPI_NONE, grid, s, h, in, nullptr, h->eo_tmp, 1, nullptr, nullptr, status, mask, nullptr);
    launch_eo<false>(EO_SCHUR2, epi, grid, s, h, h->eo_tmp, in, out, 0, aux, partial, status, mask, cnt);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------- split / merge / diagonal

// full [rhs][V][12] <-> halves [rhs][V/2][12] of parity 0 (e) and 1 (o)
__global__ void eo_split_kernel(const double2 *__restrict__ full, double2 *__restrict__ e,
                                double2 *__restrict__ o, LatticeGeom g, int merge) {
  const int r = blockIdx.y;
  const long long Vh = g.V / 2;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.V;
       s += (long long)gridDim.x * blockDim.x) {
    long long t1 = s / g.L[0];
    const int x = (int)(s % g.L[0]);
    const int y = (int)(t1 % g.L[1]);
    t1 /= g.L[1];
    const int z = (int)(t1 % g.L[2]);
    const int t = (int)(t1 / g.L[2]);
    double2 *half = ((x + y + z + t) & 1) ? o : e;
    double2 *hp = half + ((long long)r * Vh + (s >> 1)) * 12;
    const long long fo = ((long long)r * g.V + s) * 12;
    if (merge) {
      double2 *f = const_cast<double2 *>(full);
#pragma unroll
      for (int c = 0; c < 12; ++c) f[fo + c] = hp[c];
    } else {
#pragma unroll
      for (int c = 0; c < 12; ++c) hp[c] = full[fo + c];
    }
  }
}

// out = (1 - i mu gamma5) in / (1 + mu^2), half vectors
__global__ void aoo_inv_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                               double mu, long long n) {
  const double inv = 1.0 / (1.0 + mu * mu);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double gm = (i % 12) < 6 ? mu : -mu;
    const double2 v = in[i];
    out[i] = make_double2((v.x + gm * v.y) * inv, (v.y - gm * v.x) * inv);
  }
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 1216 ? 1216 : (b < 1 ? 1 : b));
}

// b_hat = b_e + kappa D_eo A_oo^{-1} b_o  for nrhs full vectors B
cudaError_t launch_eo_prepare(wd_context *h, const double2 *B, double2 *Bhat, double2 *be,
                              double2 *bo, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  const LatticeGeom g = geom_of(h);
  const long long nh = (long long)nrhs * 12 * (h->V / 2);
  eo_split_kernel<<<dim3(grid_for(h->V), nrhs), 256, 0, s>>>(B, be, bo, g, 0);
  aoo_inv_kernel<<<grid_for(nh), 256, 0, s>>>(bo, bo, h->mu, nh);
  launch_eo<false>(EO_AXPY, EPI_NONE, dim3(eo_blocks(h), nrhs), s, h, bo, be, Bhat, 0, nullptr,
                   nullptr, nullptr, M_ALL, nullptr);
  return cudaGetLastError();
}

// X (full) from x_e: x_o = A_oo^{-1} (b_o + kappa D_oe x_e)
cudaError_t launch_eo_reconstruct(wd_context *h, const double2 *B, const double2 *Xe, double2 *X,
                                  double2 *be, double2 *bo, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  const LatticeGeom g = geom_of(h);
  const long long nh = (long long)nrhs * 12 * (h->V / 2);
  eo_split_kernel<<<dim3(grid_for(h->V), nrhs), 256, 0, s>>>(B, be, bo, g, 0);
  launch_eo<false>(EO_AXPY, EPI_NONE, dim3(eo_blocks(h), nrhs), s, h, Xe, bo, be, 1, nullptr,
                   nullptr, nullptr, M_ALL, nullptr);  // be <- b_o + kappa D_oe x_e (odd)
  aoo_inv_kernel<<<grid_for(nh), 256, 0, s>>>(be, bo, h->mu, nh);
  eo_split_kernel<<<dim3(grid_for(h->V), nrhs), 256, 0, s>>>(X, const_cast<double2 *>(Xe), bo, g, 1);
  return cudaGetLastError();
}

}  // namespace wd
