// FP16-storage variant of the mixed-precision BiCGStab: the vectors the
// Wilson operator reads and writes (p, v, t) and the links are stored in
// half precision, arithmetic is FP32, r, r_hat and the solution increment
// stay FP32, and the FP64 reliable updates of solvers_mixed.cu are unchanged.
//
// Layouts (device, internal):
//  * half spinor  uint4 [rhs][g][V], g = 0..2: complex components 4g..4g+3 as
//    __half2 (re, im), scaled by a per-site norm  float [rhs][V]  (the largest
//    |re| or |im| of the site), so every stored value lies in [-1, 1]:
//    48 + 4 bytes per site.
//  * half links   uint2 [mu][q][V], q = 0..4: the nine entries of U_mu row by
//    row, two complex numbers per uint2 (the last one padded), |u_ij| <= 1, no
//    norm: 40 bytes per link.  (Row 2 is stored rather than rebuilt as
//    conj(row0 x row1): this kernel is bound by instruction issue, not by
//    loads, so two more 8-byte loads cost less than the 27 arithmetic
//    instructions of the rebuild.)
#include <cuda_fp16.h>

#include "cplx.cuh"
#include "kernels.cuh"
#include "mixed.h"
#include "spin.cuh"
#include "wd_internal.h"

namespace wd {

namespace {

__device__ __forceinline__ float2 h2f(unsigned int u) {
  __half2 h = *reinterpret_cast<const __half2 *>(&u);
  return __half22float2(h);
}
__device__ __forceinline__ unsigned int f2h(float2 f) {
  __half2 h = __float22half2_rn(f);
  return *reinterpret_cast<unsigned int *>(&h);
}
__device__ __forceinline__ float2 fcfma16(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcfmac16(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcmul16(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 f2of(double2 a) { return make_float2((float)a.x, (float)a.y); }

}  // namespace

// The stored half values of a site without its norm (the caller applies k).
__device__ __forceinline__ float ld_h_raw(const uint4 *__restrict__ base,
                                          const float *__restrict__ nrm, long long V, long long s,
                                          float2 (&p)[12]) {
  const float k = __ldg(nrm + s);
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const uint4 q = __ldg(base + g * V + s);
    p[4 * g] = h2f(q.x);
    p[4 * g + 1] = h2f(q.y);
    p[4 * g + 2] = h2f(q.z);
    p[4 * g + 3] = h2f(q.w);
  }
  return k;
}

__device__ __forceinline__ void ld_h(const uint4 *__restrict__ base, const float *__restrict__ nrm,
                                     long long V, long long s, float2 (&p)[12]) {
  const float k = __ldg(nrm + s);
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const uint4 q = __ldg(base + g * V + s);
    const float2 a = h2f(q.x), b = h2f(q.y), c = h2f(q.z), d = h2f(q.w);
    p[4 * g] = make_float2(a.x * k, a.y * k);
    p[4 * g + 1] = make_float2(b.x * k, b.y * k);
    p[4 * g + 2] = make_float2(c.x * k, c.y * k);
    p[4 * g + 3] = make_float2(d.x * k, d.y * k);
  }
}

__device__ __forceinline__ void st_h(uint4 *__restrict__ base, float *__restrict__ nrm, long long V,
                                     long long s, const float2 (&p)[12]) {
  float k = 0.f;
#pragma unroll
  for (int c = 0; c < 12; ++c) k = fmaxf(k, fmaxf(fabsf(p[c].x), fabsf(p[c].y)));
  const float inv = k > 0.f ? 1.f / k : 0.f;
  nrm[s] = k;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    uint4 q;
    q.x = f2h(make_float2(p[4 * g].x * inv, p[4 * g].y * inv));
    q.y = f2h(make_float2(p[4 * g + 1].x * inv, p[4 * g + 1].y * inv));
    q.z = f2h(make_float2(p[4 * g + 2].x * inv, p[4 * g + 2].y * inv));
    q.w = f2h(make_float2(p[4 * g + 3].x * inv, p[4 * g + 3].y * inv));
    base[g * V + s] = q;
  }
}

__device__ __forceinline__ void ld_f(const float4 *__restrict__ base, long long V, long long s,
                                     float2 (&p)[12]) {
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    const float4 f = __ldg(base + g * V + s);
    p[2 * g] = make_float2(f.x, f.y);
    p[2 * g + 1] = make_float2(f.z, f.w);
  }
}

__device__ __forceinline__ void st_f(float4 *__restrict__ base, long long V, long long s,
                                     const float2 (&p)[12]) {
#pragma unroll
  for (int g = 0; g < 6; ++g)
    base[g * V + s] = make_float4(p[2 * g].x, p[2 * g].y, p[2 * g + 1].x, p[2 * g + 1].y);
}

constexpr int LINK16_Q = 5;   // uint2 per FP16 link

__device__ __forceinline__ void ld_link16(const uint2 *__restrict__ L, long long V, int mu,
                                          long long s, float2 (&u)[9]) {
#pragma unroll
  for (int q = 0; q < LINK16_Q; ++q) {
    const uint2 a = __ldg(L + (mu * LINK16_Q + q) * V + s);
    u[2 * q] = h2f(a.x);
    if (2 * q + 1 < 9) u[2 * q + 1] = h2f(a.y);
  }
}

// Input of the hop: a half vector, or (FUSED) r (FP32) - alpha v (half).
// Returns the factor still to be applied: the site's norm for a plain half
// vector (p holds its stored values; the hop scales its product once), 1
// for the fused input (the norm is folded into alpha).
template <bool FUSED>
__device__ __forceinline__ float ld_hop16(const uint4 *__restrict__ in, const float *__restrict__ in_n,
                                          const float4 *__restrict__ r32, float2 alpha, long long V,
                                          long long s, float2 (&p)[12]) {
  if (FUSED) {
    float2 q[12];
    ld_f(r32, V, s, p);
    const float k = ld_h_raw(in, in_n, V, s, q);
    const float2 ma = make_float2(-alpha.x * k, -alpha.y * k);
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = fcfma16(ma, q[c], p[c]);
    return 1.f;
  }
  return ld_h_raw(in, in_n, V, s, p);
}

template <bool FUSED>
__device__ __forceinline__ void ld_in16(const uint4 *__restrict__ in, const float *__restrict__ in_n,
                                        const float4 *__restrict__ r32, float2 alpha, long long V,
                                        long long s, float2 (&p)[12]) {
  if (FUSED) {
    float2 q[12];
    ld_f(r32, V, s, p);
    ld_h(in, in_n, V, s, q);
    const float2 ma = make_float2(-alpha.x, -alpha.y);
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = fcfma16(ma, q[c], p[c]);
  } else {
    ld_h(in, in_n, V, s, p);
  }
}

template <bool ADJ>
__device__ __forceinline__ void su3_mul16(const float2 (&m)[9], const float2 (&h)[6],
                                          float2 (&c)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        acc = ADJ ? fcfmac16(m[3 * b + a], h[3 * sp + b], acc) : fcfma16(m[3 * a + b], h[3 * sp + b], acc);
      c[3 * sp + a] = acc;
    }
}

template <int MU, int S, bool ADJ, int R, bool FUSED>
__device__ __forceinline__ void hop16(const uint2 *__restrict__ links, const Half16 &in,
                                      const float4 *__restrict__ r32, const float2 (&alpha)[R],
                                      const bool (&on)[R], int r0, long long V, long long q,
                                      long long ql, float2 (&acc)[R][12]) {
  float2 u[9];
  ld_link16(links, V, MU, ql, u);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!on[r]) continue;
    float2 p[12], h[6], c[6];
    const float k = ld_hop16<FUSED>(in.v + (long long)(r0 + r) * 3 * V, in.n + (long long)(r0 + r) * V,
                                    FUSED ? r32 + (long long)(r0 + r) * 6 * V : nullptr, alpha[r], V,
                                    q, p);
    project<MU, S>(p, h);
    su3_mul16<ADJ>(u, h, c);
    if (!FUSED) {
#pragma unroll
      for (int e = 0; e < 6; ++e) c[e] = make_float2(c[e].x * k, c[e].y * k);
    }
    reconstruct<MU, S>(acc[r], c);
  }
}

// out (half) = A in;  EPI_DOT: + <aux32, out>, ||out||^2;  EPI_TSTT (FUSED,
// in = v, r32 = r): out = A s with s = r - alpha v, + <out, s>, ||out||^2.
template <int R, int TPB, bool DAG, int EPI, bool FUSED>
__global__ void __launch_bounds__(TPB)
wilson_f16_kernel(const uint2 *__restrict__ links, Half16 in, const float4 *__restrict__ r32,
                  Half16 out, LatticeGeom g, float kappa, float mu, int nrhs,
                  const BicgScalars *__restrict__ sc, const float4 *__restrict__ aux,
                  double *__restrict__ partial, const int *__restrict__ status, unsigned mask,
                  unsigned long long *__restrict__ sites) {
  // Blocks are numbered system-row fastest: the nrow blocks that cover the
  // same sites run next to each other and share the links and the
  // neighbour spinors' cache lines through L2.
  const int nrow = (nrhs + R - 1) / R;
  const int row = (int)(blockIdx.x % (unsigned)nrow);
  const long long sb = blockIdx.x / (unsigned)nrow;   // site block
  const long long nsb = (g.V + TPB - 1) / TPB;        // site blocks
  const int r0 = row * R;
  const long long V = g.V;
  bool on[R];
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    on[r] = r0 + r < nrhs && (status == nullptr || ((mask >> status[r0 + r]) & 1u));
    any |= on[r];
  }
  if (!any) return;
  if (sites != nullptr && sb == 0 && threadIdx.x == 0) {
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) cnt += on[r] ? 1 : 0;
    atomicAdd(sites, (unsigned long long)V * cnt);  // work accounting for the profiler
  }
  float2 alpha[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    alpha[r] = (FUSED && on[r]) ? f2of(sc[r0 + r].alpha) : make_float2(0.f, 0.f);
  const long long s = sb * TPB + threadIdx.x;
  float red[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r) red[r][0] = red[r][1] = red[r][2] = 0.f;
  if (s < V) {
    const Nbrs32 nb = neighbours32((unsigned)s, g);
    float2 acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[r][c] = make_float2(0.f, 0.f);
    constexpr int F = DAG ? +1 : -1;
    constexpr int B = -F;
    hop16<0, F, false, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.up[0], s, acc);
    hop16<0, B, true, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.dn[0], nb.dn[0], acc);
    hop16<1, F, false, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.up[1], s, acc);
    hop16<1, B, true, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.dn[1], nb.dn[1], acc);
    hop16<2, F, false, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.up[2], s, acc);
    hop16<2, B, true, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.dn[2], nb.dn[2], acc);
    hop16<3, F, false, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.up[3], s, acc);
    hop16<3, B, true, R, FUSED>(links, in, r32, alpha, on, r0, V, nb.dn[3], nb.dn[3], acc);
    const float tmu = DAG ? -mu : mu;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!on[r]) continue;
      const int q = r0 + r;
      float2 p[12], o[12];
      ld_in16<FUSED>(in.v + (long long)q * 3 * V, in.n + (long long)q * V,
                     FUSED ? r32 + (long long)q * 6 * V : nullptr, alpha[r], V, s, p);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        float2 v;
        v.x = fmaf(-kappa, acc[r][c].x, p[c].x);
        v.y = fmaf(-kappa, acc[r][c].y, p[c].y);
        if (tmu != 0.f) {
          const float mm = c < 6 ? tmu : -tmu;
          v.x = fmaf(-mm, p[c].y, v.x);
          v.y = fmaf(mm, p[c].x, v.y);
        }
        o[c] = v;
      }
      st_h(out.v + (long long)q * 3 * V, out.n + (long long)q * V, V, s, o);
      if (EPI == EPI_DOT) {
        float2 a[12];
        ld_f(aux + (long long)q * 6 * V, V, s, a);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          red[r][0] = fmaf(a[c].x, o[c].x, fmaf(a[c].y, o[c].y, red[r][0]));
          red[r][1] = fmaf(a[c].x, o[c].y, fmaf(-a[c].y, o[c].x, red[r][1]));
          red[r][2] = fmaf(o[c].x, o[c].x, fmaf(o[c].y, o[c].y, red[r][2]));
        }
      } else if (EPI == EPI_TSTT) {
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          red[r][0] = fmaf(o[c].x, p[c].x, fmaf(o[c].y, p[c].y, red[r][0]));
          red[r][1] = fmaf(o[c].x, p[c].y, fmaf(-o[c].y, p[c].x, red[r][1]));
          red[r][2] = fmaf(o[c].x, o[c].x, fmaf(o[c].y, o[c].y, red[r][2]));
        }
      }
    }
  }
  if (EPI != EPI_NONE) {
    constexpr int NW = TPB / 32;
    __shared__ double sh[R][3][NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float v = red[r][q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[r][q][w] = (double)v;
      }
    __syncthreads();
    if (threadIdx.x < R * 3) {
      const int r = threadIdx.x / 3, q = threadIdx.x % 3;
      if (on[r]) {
        double t = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) t += sh[r][q][w2];
        partial[((long long)(r0 + r) * nsb + sb) * 3 + q] = t;
      }
    }
  }
}

template <int R, int TPB>
static cudaError_t launch_w16(const wd_context *h, const uint2 *links, Half16 in, const float4 *r32,
                              Half16 out, int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, unsigned long long *sites, cudaStream_t s) {
  const LatticeGeom g = geom_of(h);
  const long long nblk = (h->V + TPB - 1) / TPB * ((nrhs + R - 1) / R);
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk);
  const float kap = (float)h->kappa, mu = (float)h->mu;
  if (epi == EPI_DOT)
    wilson_f16_kernel<R, TPB, false, EPI_DOT, false><<<grid, TPB, 0, s>>>(links, in, r32, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, sites);
  else if (epi == EPI_TSTT)
    wilson_f16_kernel<R, TPB, false, EPI_TSTT, true><<<grid, TPB, 0, s>>>(links, in, r32, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, sites);
  else if (dagger)
    wilson_f16_kernel<R, TPB, true, EPI_NONE, false><<<grid, TPB, 0, s>>>(links, in, r32, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, sites);
  else
    wilson_f16_kernel<R, TPB, false, EPI_NONE, false><<<grid, TPB, 0, s>>>(links, in, r32, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, sites);
  return cudaGetLastError();
}

static int tune_key16(int nrhs) { return nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1; }

// Launch shape for nrhs systems: the tuned one if any, else one right-hand
// side per thread and 128 threads per block.
void wilson16_shape(const wd_context *h, int nrhs, int *R, int *T) {
  const int key = tune_key16(nrhs);
  if (h->tune16_R[key] != 0) {
    *R = h->tune16_R[key];
    *T = h->tune16_T[key];
    return;
  }
  *R = 1;
  *T = 128;
}

int wilson16_blocks(const wd_context *h, int nrhs) {
  int R, T;
  wilson16_shape(h, nrhs, &R, &T);
  return (int)((h->V + T - 1) / T);
}

static cudaError_t launch_w16_shape(const wd_context *h, int R, int T, const uint2 *links,
                                    Half16 in, const float4 *r32, Half16 out, int nrhs, int dagger,
                                    int epi, const BicgScalars *sc, const float4 *aux,
                                    double *partial, const int *status, unsigned mask,
                                    unsigned long long *sites, cudaStream_t s) {
#define W16(RR, TT)                                                                           \
  if (R == RR && T == TT)                                                                     \
    return launch_w16<RR, TT>(h, links, in, r32, out, nrhs, dagger, epi, sc, aux, partial, \
                              status, mask, sites, s);
  W16(1, 64) W16(1, 128) W16(1, 256)
  W16(2, 64) W16(2, 128) W16(2, 256)
  W16(4, 64) W16(4, 128) W16(4, 256)
#undef W16
  return cudaErrorInvalidValue;
}

cudaError_t launch_wilson_f16(const wd_context *h, const uint2 *links, Half16 in, const float4 *r32,
                              Half16 out, int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s) {
  ProfLaunch prof(PC_DSLASH_LOW, s);
  int R, T;
  wilson16_shape(h, nrhs, &R, &T);
  return launch_w16_shape(h, R, T, links, in, r32, out, nrhs, dagger, epi, sc, aux, partial,
                          status, mask, prof_site_counter_low(), s);
}

// Times every launch shape on (in -> out) and keeps the fastest for nrhs.
cudaError_t tune_wilson_f16(wd_context *h, const uint2 *links, int nrhs, Half16 in, Half16 out,
                            cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bR = 1, bT = 128;
  const int Rs[3] = {1, 2, 4}, Ts[3] = {64, 128, 256};
  cudaError_t err = cudaSuccess;
  for (int R : Rs) {
    if (R > nrhs && R > 1) continue;
    for (int T : Ts) {
      for (int w = 0; w < 2 && err == cudaSuccess; ++w)
        err = launch_w16_shape(h, R, T, links, in, nullptr, out, nrhs, 0, EPI_NONE, nullptr,
                               nullptr, nullptr, nullptr, M_ALL, nullptr, s);
      float t_best = 1e30f;
      for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        err = launch_w16_shape(h, R, T, links, in, nullptr, out, nrhs, 0, EPI_NONE, nullptr,
                               nullptr, nullptr, nullptr, M_ALL, nullptr, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t_best = ms < t_best ? ms : t_best;
      }
      if (err == cudaSuccess && t_best < best) {
        best = t_best;
        bR = R;
        bT = T;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  const int key = tune_key16(nrhs);
  h->tune16_R[key] = bR;
  h->tune16_T[key] = bT;
  h->tune16_ms[key] = best;
  return cudaSuccess;
}

// ----------------------------------------------------------------- conversions

__global__ void links_to_f16_kernel(const double2 *__restrict__ U, uint2 *__restrict__ L,
                                    long long V) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const double2 *u = U + (s * 4 + mu) * 9;
#pragma unroll
      for (int q = 0; q < LINK16_Q; ++q) {
        uint2 w;
        w.x = f2h(f2of(u[2 * q]));
        w.y = 2 * q + 1 < 9 ? f2h(f2of(u[2 * q + 1])) : 0u;
        L[(mu * LINK16_Q + q) * V + s] = w;
      }
    }
  }
}

cudaError_t launch_links_to_f16(const wd_context *h, uint2 *L, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  links_to_f16_kernel<<<608, 256, 0, s>>>(h->links, L, h->V);
  return cudaGetLastError();
}

// FP64 boundary [rhs][V][12] -> half vector (used by wd_apply_f16)
__global__ void f64_to_f16_kernel(const double2 *__restrict__ in, Half16 out, long long V) {
  const int r = blockIdx.y;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    float2 p[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = f2of(in[((long long)r * V + s) * 12 + c]);
    st_h(out.v + (long long)r * 3 * V, out.n + (long long)r * V, V, s, p);
  }
}

__global__ void f16_to_f64_kernel(Half16 in, double2 *__restrict__ out, long long V) {
  const int r = blockIdx.y;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    float2 p[12];
    ld_h(in.v + (long long)r * 3 * V, in.n + (long long)r * V, V, s, p);
#pragma unroll
    for (int c = 0; c < 12; ++c)
      out[((long long)r * V + s) * 12 + c] = make_double2((double)p[c].x, (double)p[c].y);
  }
}

static unsigned site_blocks(long long V) {
  long long b = (V + 255) / 256;
  return (unsigned)(b > 608 ? 608 : (b < 1 ? 1 : b));
}

cudaError_t launch_f64_to_f16(const double2 *in, Half16 out, long long V, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  f64_to_f16_kernel<<<dim3(site_blocks(V), nrhs), 256, 0, s>>>(in, out, V);
  return cudaGetLastError();
}

cudaError_t launch_f16_to_f64(Half16 in, double2 *out, long long V, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  f16_to_f64_kernel<<<dim3(site_blocks(V), nrhs), 256, 0, s>>>(in, out, V);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- BiCGStab updates (per site)

__device__ __forceinline__ bool on16(const int *status, unsigned mask, int r) {
  return status == nullptr || ((mask >> status[r]) & 1u);
}

// p (half) = r + beta (p - omega v)
__global__ void __launch_bounds__(256)
bicg16_update_p_kernel(Half16 p, const float4 *__restrict__ r, Half16 v,
                       const BicgScalars *__restrict__ sc, const int *__restrict__ status,
                       long long V) {
  const int q = blockIdx.y;
  if (!on16(status, M_ACTIVE, q)) return;  // uniform per block
  // beta in FP64 once per block (as in bicg_update_p_kernel)
  __shared__ float2 s_bm[2];
  if (threadIdx.x == 0) {
    const BicgScalars S = sc[q];
    s_bm[0] = f2of(cmul(cdiv(S.rho, S.rho_old), cdiv(S.alpha, S.omega)));
    s_bm[1] = make_float2(-(float)S.omega.x, -(float)S.omega.y);
  }
  __syncthreads();
  const float2 beta = s_bm[0], mom = s_bm[1];
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    float2 rv[12], pv[12], vv[12];
    ld_f(r + (long long)q * 6 * V, V, s, rv);
    ld_h(p.v + (long long)q * 3 * V, p.n + (long long)q * V, V, s, pv);
    ld_h(v.v + (long long)q * 3 * V, v.n + (long long)q * V, V, s, vv);
#pragma unroll
    for (int c = 0; c < 12; ++c) pv[c] = fcfma16(beta, fcfma16(mom, vv[c], pv[c]), rv[c]);
    st_h(p.v + (long long)q * 3 * V, p.n + (long long)q * V, V, s, pv);
  }
}

// s = r - alpha v; xs += alpha p + omega s; r = s - omega t; partial <rhat, r>, ||r||^2
__global__ void __launch_bounds__(256)
bicg16_update_xr_kernel(float4 *__restrict__ xs, float4 *__restrict__ r, Half16 p, Half16 v,
                        Half16 t, const float4 *__restrict__ rhat,
                        const BicgScalars *__restrict__ sc, const int *__restrict__ status,
                        double *__restrict__ partial, long long V) {
  const int q = blockIdx.y;
  if (!on16(status, M_ACTIVE, q)) return;
  const float2 al = f2of(sc[q].alpha), om = f2of(sc[q].omega);
  const float2 mal = make_float2(-al.x, -al.y), mom = make_float2(-om.x, -om.y);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    float2 rv[12], vv[12], pv[12], tv[12], xv[12], hv[12];
    ld_f(r + (long long)q * 6 * V, V, s, rv);
    ld_h(v.v + (long long)q * 3 * V, v.n + (long long)q * V, V, s, vv);
    ld_h(p.v + (long long)q * 3 * V, p.n + (long long)q * V, V, s, pv);
    ld_h(t.v + (long long)q * 3 * V, t.n + (long long)q * V, V, s, tv);
    ld_f(xs + (long long)q * 6 * V, V, s, xv);
    ld_f(rhat + (long long)q * 6 * V, V, s, hv);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const float2 sv = fcfma16(mal, vv[c], rv[c]);
      xv[c] = fcfma16(om, sv, fcfma16(al, pv[c], xv[c]));
      const float2 rn = fcfma16(mom, tv[c], sv);
      rv[c] = rn;
      a0 = fmaf(hv[c].x, rn.x, fmaf(hv[c].y, rn.y, a0));
      a1 = fmaf(hv[c].x, rn.y, fmaf(-hv[c].y, rn.x, a1));
      a2 = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, a2));
    }
    st_f(xs + (long long)q * 6 * V, V, s, xv);
    st_f(r + (long long)q * 6 * V, V, s, rv);
  }
  __shared__ double sh[3][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float vals[3] = {a0, a1, a2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float vv2 = vals[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vv2 += __shfl_down_sync(0xffffffffu, vv2, off);
    if (lane == 0) sh[k][w] = (double)vv2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double tot = 0.0;
    for (int w2 = 0; w2 < 8; ++w2) tot += sh[threadIdx.x][w2];
    partial[((long long)q * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = tot;
  }
}

// rhat = r (FP32), p = v = 0 (half)
__global__ void __launch_bounds__(256)
bicg16_restart_kernel(float4 *__restrict__ rhat, const float4 *__restrict__ r, Half16 p, Half16 v,
                      const int *__restrict__ status, unsigned mask, long long V) {
  const int q = blockIdx.y;
  if (!on16(status, mask, q)) return;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int g = 0; g < 6; ++g) rhat[(long long)q * 6 * V + g * V + s] = r[(long long)q * 6 * V + g * V + s];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      p.v[(long long)q * 3 * V + g * V + s] = z;
      v.v[(long long)q * 3 * V + g * V + s] = z;
    }
    p.n[(long long)q * V + s] = 0.f;
    v.n[(long long)q * V + s] = 0.f;
  }
}

int stream16_blocks(long long V) { return (int)site_blocks(V); }

cudaError_t launch_bicg16_update_p(Half16 p, const float4 *r, Half16 v, const BicgScalars *sc,
                                   const int *status, long long V, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM_LOW, s);
  bicg16_update_p_kernel<<<dim3(site_blocks(V), nrhs), 256, 0, s>>>(p, r, v, sc, status, V);
  return cudaGetLastError();
}

cudaError_t launch_bicg16_update_xr(float4 *xs, float4 *r, Half16 p, Half16 v, Half16 t,
                                    const float4 *rhat, const BicgScalars *sc, const int *status,
                                    double *partial, long long V, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM_LOW, s);
  bicg16_update_xr_kernel<<<dim3(site_blocks(V), nrhs), 256, 0, s>>>(xs, r, p, v, t, rhat, sc,
                                                                     status, partial, V);
  return cudaGetLastError();
}

cudaError_t launch_bicg16_restart(float4 *rhat, const float4 *r, Half16 p, Half16 v,
                                  const int *status, unsigned mask, long long V, int nrhs,
                                  cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  bicg16_restart_kernel<<<dim3(site_blocks(V), nrhs), 256, 0, s>>>(rhat, r, p, v, status, mask, V);
  return cudaGetLastError();
}

}  // namespace wd
