// FP32 even-odd Schur operator for the mixed solver (the Sec. 3 system in
// low precision):
//
//   A_hat x_e = (1 + i mu gamma5) x_e - kappa^2 D_eo A_oo^{-1} D_oe x_e,
//   A_oo^{-1} = (1 - i mu gamma5) / (1 + mu^2),
//
// as two half-lattice hop kernels, the second one carrying the reduction
// epilogues of the full FP32 kernel.  Half vectors use the FP32 layout of
// mixed.cu on the sites of one parity: float4 [rhs][6][V/2], compact index
// s / 2 (Lx even: the two sites of an x-pair have opposite parities).  The
// links are the full-lattice FP32 links of mixed.cu.
#include "cplx.cuh"
#include "kernels.cuh"
#include "mixed.h"
#include "spin.cuh"
#include "wd_internal.h"

namespace wd {

namespace {

__device__ __forceinline__ float2 fcfma_eo(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcfmac_eo(float2 a, float2 b, float2 c) {  // c + conj(a) b
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcmul_eo(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// 12 complex components of a half-vector site (compact index c, stride Vh);
// FUSED: the value of base - alpha base2.
template <bool FUSED>
__device__ __forceinline__ void ld_half32(const float4 *__restrict__ base,
                                          const float4 *__restrict__ base2, float2 alpha,
                                          long long Vh, long long c, float2 (&p)[12]) {
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    const float4 f = __ldg(base + g * Vh + c);
    p[2 * g] = make_float2(f.x, f.y);
    p[2 * g + 1] = make_float2(f.z, f.w);
  }
  if (FUSED) {
    const float2 ma = make_float2(-alpha.x, -alpha.y);
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const float4 f = __ldg(base2 + g * Vh + c);
      p[2 * g] = fcfma_eo(ma, make_float2(f.x, f.y), p[2 * g]);
      p[2 * g + 1] = fcfma_eo(ma, make_float2(f.z, f.w), p[2 * g + 1]);
    }
  }
}

// link U_mu at full site s: rows 0, 1 stored, row 2 = conj(row0 x row1)
__device__ __forceinline__ void ld_link_eo(const float4 *__restrict__ L, long long V, int mu,
                                           long long s, float2 (&u)[9]) {
  const float4 f0 = __ldg(L + (mu * 3 + 0) * V + s);
  const float4 f1 = __ldg(L + (mu * 3 + 1) * V + s);
  const float4 f2 = __ldg(L + (mu * 3 + 2) * V + s);
  u[0] = make_float2(f0.x, f0.y);
  u[1] = make_float2(f0.z, f0.w);
  u[2] = make_float2(f1.x, f1.y);
  u[3] = make_float2(f1.z, f1.w);
  u[4] = make_float2(f2.x, f2.y);
  u[5] = make_float2(f2.z, f2.w);
  float2 t;
  t = ssub(fcmul_eo(u[1], u[5]), fcmul_eo(u[2], u[4]));
  u[6] = make_float2(t.x, -t.y);
  t = ssub(fcmul_eo(u[2], u[3]), fcmul_eo(u[0], u[5]));
  u[7] = make_float2(t.x, -t.y);
  t = ssub(fcmul_eo(u[0], u[4]), fcmul_eo(u[1], u[3]));
  u[8] = make_float2(t.x, -t.y);
}

// one hop: neighbour q (full index, other parity) read from the half vector
template <int MU, int S, bool ADJ, bool FUSED>
__device__ __forceinline__ void hop_eo32(const float4 *__restrict__ links,
                                         const float4 *__restrict__ src,
                                         const float4 *__restrict__ src2, float2 alpha,
                                         long long V, long long q, long long ql,
                                         float2 (&acc)[12]) {
  float2 u[9], p[12], h[6], c[6];
  ld_link_eo(links, V, MU, ql, u);
  ld_half32<FUSED>(src, src2, alpha, V / 2, q >> 1, p);
  project<MU, S>(p, h);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        v = ADJ ? fcfmac_eo(u[3 * b + a], h[3 * sp + b], v) : fcfma_eo(u[3 * a + b], h[3 * sp + b], v);
      c[3 * sp + a] = v;
    }
  reconstruct<MU, S>(acc, c);
}

}  // namespace

enum { EO32_SCHUR1 = 0, EO32_SCHUR2 = 1 };

// out (parity pout, compact) from h = D_{pout, 1-pout} src:
//  EO32_SCHUR1: out = (1 - i mu g5) h / (1 + mu^2)
//  EO32_SCHUR2: out = (1 + i mu g5) same - kappa^2 h, with the epilogues
//               EPI_DOT (<aux, out>, ||out||^2) and EPI_TSTT (<out, same>,
//               ||out||^2).
// FUSED: the even operand is s = r - alpha v, read from (src, src2) in
// SCHUR1 and from (same, same2) in SCHUR2.
template <bool DAG, int MODE, int EPI, bool FUSED>
__global__ void __launch_bounds__(128, 6)  // 80 registers, as the full FP32 kernel
wilson_eo32_kernel(const float4 *__restrict__ links, const float4 *__restrict__ src,
                   const float4 *__restrict__ src2, const float4 *__restrict__ same,
                   const float4 *__restrict__ same2, float4 *__restrict__ out, LatticeGeom g,
                   int pout, float kappa, float mu, const BicgScalars *__restrict__ sc,
                   const float4 *__restrict__ aux, double *__restrict__ partial,
                   const int *__restrict__ status, unsigned mask,
                   unsigned long long *__restrict__ sites, int nrhs) {
  // Blocks are numbered system fastest: the nrhs blocks that cover one range
  // of sites run side by side and share the links through L2, which a
  // half-lattice hop reads in full (every link touches one site of each
  // parity).
  const int r = (int)(blockIdx.x % (unsigned)nrhs);
  const long long sb = blockIdx.x / (unsigned)nrhs;  // site block
  const long long nsb = gridDim.x / (unsigned)nrhs;
  if (status != nullptr && !((mask >> status[r]) & 1u)) return;  // uniform per block
  const long long V = g.V, Vh = g.V / 2;
  if (sites != nullptr && sb == 0 && threadIdx.x == 0)
    atomicAdd(sites, (unsigned long long)Vh);  // work accounting for the profiler
  const float2 alpha = FUSED ? make_float2((float)sc[r].alpha.x, (float)sc[r].alpha.y)
                             : make_float2(0.f, 0.f);
  const long long off = (long long)r * 6 * Vh;
  const long long i = sb * blockDim.x + threadIdx.x;
  float red[3] = {0.f, 0.f, 0.f};
  if (i < Vh) {
    // the site of parity pout in the x-pair (2i, 2i + 1)
    const unsigned s0 = (unsigned)(2 * i);
    const unsigned q0 = fast_div(s0, g.dm[0], g.dsh[0]);
    const unsigned q1 = fast_div(q0, g.dm[1], g.dsh[1]);
    const unsigned t = fast_div(q1, g.dm[2], g.dsh[2]);
    const unsigned y = q0 - q1 * (unsigned)g.L[1], z = q1 - t * (unsigned)g.L[2];
    const unsigned s = s0 + ((int)((y + z + t) & 1u) != pout ? 1u : 0u);
    const Nbrs32 nb = neighbours32(s, g);
    constexpr int F = DAG ? +1 : -1;
    constexpr int B = -F;
    const float4 *sr = src + off;
    const float4 *sr2 = FUSED && MODE == EO32_SCHUR1 ? src2 + off : nullptr;
    constexpr bool FS = FUSED && MODE == EO32_SCHUR1;
    float2 acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = make_float2(0.f, 0.f);
    hop_eo32<0, F, false, FS>(links, sr, sr2, alpha, V, nb.up[0], s, acc);
    hop_eo32<0, B, true, FS>(links, sr, sr2, alpha, V, nb.dn[0], nb.dn[0], acc);
    hop_eo32<1, F, false, FS>(links, sr, sr2, alpha, V, nb.up[1], s, acc);
    hop_eo32<1, B, true, FS>(links, sr, sr2, alpha, V, nb.dn[1], nb.dn[1], acc);
    hop_eo32<2, F, false, FS>(links, sr, sr2, alpha, V, nb.up[2], s, acc);
    hop_eo32<2, B, true, FS>(links, sr, sr2, alpha, V, nb.dn[2], nb.dn[2], acc);
    hop_eo32<3, F, false, FS>(links, sr, sr2, alpha, V, nb.up[3], s, acc);
    hop_eo32<3, B, true, FS>(links, sr, sr2, alpha, V, nb.dn[3], nb.dn[3], acc);
    const float tmu = DAG ? -mu : mu;
    float2 sm[12];
    if (MODE == EO32_SCHUR2)
      ld_half32<FUSED>(same + off, FUSED ? same2 + off : nullptr, alpha, Vh, i, sm);
    const float inv = 1.f / (1.f + tmu * tmu);
    const float k2 = kappa * kappa;
    float2 o[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float gm = c < 6 ? tmu : -tmu;  // mu * gamma5 entry
      float2 v;
      if (MODE == EO32_SCHUR1) {
        v.x = fmaf(gm, acc[c].y, acc[c].x) * inv;
        v.y = fmaf(-gm, acc[c].x, acc[c].y) * inv;
      } else {
        v.x = fmaf(-k2, acc[c].x, fmaf(-gm, sm[c].y, sm[c].x));
        v.y = fmaf(-k2, acc[c].y, fmaf(gm, sm[c].x, sm[c].y));
      }
      o[c] = v;
    }
    float4 *ob = out + off;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      ob[q * Vh + i] = make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
    if (EPI == EPI_DOT) {
      const float4 *ab = aux + off;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float4 f = __ldg(ab + q * Vh + i);
        const float2 a0 = make_float2(f.x, f.y), a1 = make_float2(f.z, f.w);
        const float2 o0 = o[2 * q], o1 = o[2 * q + 1];
        red[0] = fmaf(a0.x, o0.x, fmaf(a0.y, o0.y, red[0]));
        red[1] = fmaf(a0.x, o0.y, fmaf(-a0.y, o0.x, red[1]));
        red[2] = fmaf(o0.x, o0.x, fmaf(o0.y, o0.y, red[2]));
        red[0] = fmaf(a1.x, o1.x, fmaf(a1.y, o1.y, red[0]));
        red[1] = fmaf(a1.x, o1.y, fmaf(-a1.y, o1.x, red[1]));
        red[2] = fmaf(o1.x, o1.x, fmaf(o1.y, o1.y, red[2]));
      }
    } else if (EPI == EPI_TSTT) {  // <t, s>, ||t||^2 with s = same
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        red[0] = fmaf(o[c].x, sm[c].x, fmaf(o[c].y, sm[c].y, red[0]));
        red[1] = fmaf(o[c].x, sm[c].y, fmaf(-o[c].y, sm[c].x, red[1]));
        red[2] = fmaf(o[c].x, o[c].x, fmaf(o[c].y, o[c].y, red[2]));
      }
    }
  }
  if (EPI != EPI_NONE) {
    __shared__ double sh[3][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v = red[q];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
      if (lane == 0) sh[q][w] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 3)
      partial[((long long)r * nsb + sb) * 3 + threadIdx.x] =
          ((sh[threadIdx.x][0] + sh[threadIdx.x][1]) + sh[threadIdx.x][2]) + sh[threadIdx.x][3];
  }
}

int schur32_blocks(const wd_context *h) { return (int)((h->V / 2 + 127) / 128); }

// out = A_hat in (dagger: A_hat^dagger) on even half vectors, tmp an odd
// half vector per system; epi and FUSED (epi == EPI_TSTT: in = r, in2 = v,
// the operand is s = r - alpha v) as launch_wilson_f32.
cudaError_t launch_schur_f32(const Mixed32 &m, const float4 *in, const float4 *in2, float4 *out,
                             float4 *tmp, int nrhs, int dagger, int epi, const BicgScalars *sc,
                             const float4 *aux, double *partial, const int *status,
                             unsigned mask, cudaStream_t s) {
  ProfLaunch prof(PC_DSLASH_LOW, s);
  const wd_context *h = m.h;
  const LatticeGeom g = geom_of(h);
  const dim3 grid((unsigned)schur32_blocks(h) * (unsigned)nrhs);
  const float kap = (float)h->kappa, mu = (float)h->mu;
  unsigned long long *cnt = prof_site_counter_low();
#define EO32(D, M, E, FU, SRC, SRC2, SAME, SAME2, OUT, POUT, CNT)                               \
  wilson_eo32_kernel<D, M, E, FU><<<grid, 128, 0, s>>>(m.links, SRC, SRC2, SAME, SAME2, OUT, g, \
                                                       POUT, kap, mu, sc, aux, partial, status, \
                                                       mask, CNT, nrhs)
  if (epi == EPI_TSTT) {
    EO32(false, EO32_SCHUR1, EPI_NONE, true, in, in2, nullptr, nullptr, tmp, 1, nullptr);
    EO32(false, EO32_SCHUR2, EPI_TSTT, true, tmp, nullptr, in, in2, out, 0, cnt);
  } else if (epi == EPI_DOT) {
    EO32(false, EO32_SCHUR1, EPI_NONE, false, in, nullptr, nullptr, nullptr, tmp, 1, nullptr);
    EO32(false, EO32_SCHUR2, EPI_DOT, false, tmp, nullptr, in, nullptr, out, 0, cnt);
  } else if (dagger) {
    EO32(true, EO32_SCHUR1, EPI_NONE, false, in, nullptr, nullptr, nullptr, tmp, 1, nullptr);
    EO32(true, EO32_SCHUR2, EPI_NONE, false, tmp, nullptr, in, nullptr, out, 0, cnt);
  } else {
    EO32(false, EO32_SCHUR1, EPI_NONE, false, in, nullptr, nullptr, nullptr, tmp, 1, nullptr);
    EO32(false, EO32_SCHUR2, EPI_NONE, false, tmp, nullptr, in, nullptr, out, 0, cnt);
  }
#undef EO32
  return cudaGetLastError();
}

}  // namespace wd
