// FP32-storage kernels of the mixed-precision BiCGStab (reliable updates in
// FP64 are done with the kernels of dslash.cu and blas.cu).
//
// Layouts (device, internal):
//  * spinor  float4 [rhs][g][V], g = 0..5: complex components 2g, 2g+1 of a
//    site (c = 3*sigma + a), 96 bytes per site, unit stride over sites.
//  * links   float4 [mu][q][V], q = 0..2: rows 0 and 1 of U_mu (12 reals,
//    48 bytes per link); row 2 = conj(row0 x row1), exact for SU(3).
// The dslash handles R right-hand sides per thread so every link it loads
// serves R spinors.  Reductions: FP32 within a thread and a warp, FP64
// across warps and blocks, fixed order.
#include "cplx.cuh"
#include "kernels.cuh"
#include "mixed.h"
#include "spin.cuh"
#include "wd_internal.h"

namespace wd {

__device__ __forceinline__ float2 f2(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ float2 fcfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcfmac(float2 a, float2 b, float2 c) {  // c + conj(a) b
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void ld_spinor32(const float4 *__restrict__ base, long long V,
                                            long long s, float2 (&p)[12]) {
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    const float4 f = __ldg(base + g * V + s);
    p[2 * g] = make_float2(f.x, f.y);
    p[2 * g + 1] = make_float2(f.z, f.w);
  }
}

__device__ __forceinline__ void st_spinor32(float4 *__restrict__ base, long long V, long long s,
                                            const float2 (&p)[12]) {
#pragma unroll
  for (int g = 0; g < 6; ++g)
    base[g * V + s] = make_float4(p[2 * g].x, p[2 * g].y, p[2 * g + 1].x, p[2 * g + 1].y);
}

__device__ __forceinline__ void ld_link32(const float4 *__restrict__ L, long long V, int mu,
                                          long long s, float2 (&u)[9]) {
  const float4 f0 = __ldg(L + (mu * 3 + 0) * V + s);
  const float4 f1 = __ldg(L + (mu * 3 + 1) * V + s);
  const float4 f2v = __ldg(L + (mu * 3 + 2) * V + s);
  u[0] = make_float2(f0.x, f0.y);
  u[1] = make_float2(f0.z, f0.w);
  u[2] = make_float2(f1.x, f1.y);
  u[3] = make_float2(f1.z, f1.w);
  u[4] = make_float2(f2v.x, f2v.y);
  u[5] = make_float2(f2v.z, f2v.w);
  // row 2 = conj(row0 x row1)
  float2 t;
  t = ssub(fcmul(u[1], u[5]), fcmul(u[2], u[4]));
  u[6] = make_float2(t.x, -t.y);
  t = ssub(fcmul(u[2], u[3]), fcmul(u[0], u[5]));
  u[7] = make_float2(t.x, -t.y);
  t = ssub(fcmul(u[0], u[4]), fcmul(u[1], u[3]));
  u[8] = make_float2(t.x, -t.y);
}

template <bool ADJ>
__device__ __forceinline__ void su3_mul32(const float2 (&m)[9], const float2 (&h)[6],
                                          float2 (&c)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        acc = ADJ ? fcfmac(m[3 * b + a], h[3 * sp + b], acc) : fcfma(m[3 * a + b], h[3 * sp + b], acc);
      c[3 * sp + a] = acc;
    }
}

// Input spinor of the hop: `in` itself (FUSED = false) or in - alpha * in2
// (FUSED: s = r - alpha v without materialising s).
template <bool FUSED>
__device__ __forceinline__ void ld_input(const float4 *__restrict__ in, const float4 *__restrict__ in2,
                                         float2 alpha, long long V, long long s, float2 (&p)[12]) {
  ld_spinor32(in, V, s, p);
  if (FUSED) {
    float2 q[12];
    ld_spinor32(in2, V, s, q);
    const float2 ma = make_float2(-alpha.x, -alpha.y);
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = fcfma(ma, q[c], p[c]);
  }
}

template <int MU, int S, bool ADJ, int R, bool FUSED>
__device__ __forceinline__ void hop32(const float4 *__restrict__ links, const float4 *__restrict__ in,
                                      const float4 *__restrict__ in2, const float2 (&alpha)[R],
                                      const bool (&on)[R], long long V, long long q, long long ql,
                                      float2 (&acc)[R][12]) {
  float2 u[9];
  ld_link32(links, V, MU, ql, u);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!on[r]) continue;
    float2 p[12], h[6], c[6];
    ld_input<FUSED>(in + (long long)r * 6 * V, FUSED ? in2 + (long long)r * 6 * V : nullptr,
                    alpha[r], V, q, p);
    project<MU, S>(p, h);
    su3_mul32<ADJ>(u, h, c);
    reconstruct<MU, S>(acc[r], c);
  }
}

// EPI_NONE: out = A in.   EPI_DOT: out = A in, partial <aux, out>, ||out||^2.
// EPI_TSTT (FUSED): out = A s with s = in - alpha in2, partial <out, s>, ||out||^2.
// R = 1 shapes are held to 80 registers (768 threads per SM, 6 blocks of 128):
// the kernel waits on gathers, and the sixth block's warps hide more of that
// latency than the few spilled words cost (0.778 -> 0.692 ms at 24^3 x 48
// with 16 systems).
template <int R, int TPB, bool DAG, int EPI, bool FUSED>
__global__ void __launch_bounds__(TPB, R == 1 ? 768 / TPB : 1)
wilson_f32_kernel(const float4 *__restrict__ links, const float4 *__restrict__ in,
                  const float4 *__restrict__ in2, float4 *__restrict__ out, LatticeGeom g,
                  float kappa, float mu, int nrhs, const BicgScalars *__restrict__ sc,
                  const float4 *__restrict__ aux, double *__restrict__ partial,
                  const int *__restrict__ status, unsigned mask,
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
  if (!any) return;  // uniform over the block
  if (sites != nullptr && sb == 0 && threadIdx.x == 0) {
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) cnt += on[r] ? 1 : 0;
    atomicAdd(sites, (unsigned long long)V * cnt);  // work accounting for the profiler
  }
  float2 alpha[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    alpha[r] = (FUSED && on[r]) ? f2(sc[r0 + r].alpha) : make_float2(0.f, 0.f);
  const long long s = sb * TPB + threadIdx.x;
  float red[R][3];
#pragma unroll
  for (int r = 0; r < R; ++r) red[r][0] = red[r][1] = red[r][2] = 0.f;
  const float4 *inb = in + (long long)r0 * 6 * V;
  const float4 *in2b = FUSED ? in2 + (long long)r0 * 6 * V : nullptr;
  if (s < V) {
    const Nbrs32 nb = neighbours32((unsigned)s, g);
    float2 acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[r][c] = make_float2(0.f, 0.f);
    constexpr int F = DAG ? +1 : -1;
    constexpr int B = -F;
    hop32<0, F, false, R, FUSED>(links, inb, in2b, alpha, on, V, nb.up[0], s, acc);
    hop32<0, B, true, R, FUSED>(links, inb, in2b, alpha, on, V, nb.dn[0], nb.dn[0], acc);
    hop32<1, F, false, R, FUSED>(links, inb, in2b, alpha, on, V, nb.up[1], s, acc);
    hop32<1, B, true, R, FUSED>(links, inb, in2b, alpha, on, V, nb.dn[1], nb.dn[1], acc);
    hop32<2, F, false, R, FUSED>(links, inb, in2b, alpha, on, V, nb.up[2], s, acc);
    hop32<2, B, true, R, FUSED>(links, inb, in2b, alpha, on, V, nb.dn[2], nb.dn[2], acc);
    hop32<3, F, false, R, FUSED>(links, inb, in2b, alpha, on, V, nb.up[3], s, acc);
    hop32<3, B, true, R, FUSED>(links, inb, in2b, alpha, on, V, nb.dn[3], nb.dn[3], acc);
    const float tmu = DAG ? -mu : mu;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!on[r]) continue;
      float2 p[12];
      ld_input<FUSED>(inb + (long long)r * 6 * V, FUSED ? in2b + (long long)r * 6 * V : nullptr,
                      alpha[r], V, s, p);
      float2 o[12];
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
      st_spinor32(out + (long long)(r0 + r) * 6 * V, V, s, o);
      if (EPI == EPI_DOT) {
        float2 a[12];
        ld_spinor32(aux + (long long)(r0 + r) * 6 * V, V, s, a);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          red[r][0] = fmaf(a[c].x, o[c].x, fmaf(a[c].y, o[c].y, red[r][0]));
          red[r][1] = fmaf(a[c].x, o[c].y, fmaf(-a[c].y, o[c].x, red[r][1]));
          red[r][2] = fmaf(o[c].x, o[c].x, fmaf(o[c].y, o[c].y, red[r][2]));
        }
      } else if (EPI == EPI_TSTT) {  // <t, s>, ||t||^2 with s = p
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
static cudaError_t launch_w32(const Mixed32 &m, const float4 *in, const float4 *in2, float4 *out,
                              int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s) {
  const wd_context *h = m.h;
  LatticeGeom g = geom_of(h);
  const long long nblk = (h->V + TPB - 1) / TPB * ((nrhs + R - 1) / R);
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk);
  const float kap = (float)h->kappa, mu = (float)h->mu;
  if (epi == EPI_DOT)
    wilson_f32_kernel<R, TPB, false, EPI_DOT, false><<<grid, TPB, 0, s>>>(m.links, in, nullptr, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, m.sites);
  else if (epi == EPI_TSTT)
    wilson_f32_kernel<R, TPB, false, EPI_TSTT, true><<<grid, TPB, 0, s>>>(m.links, in, in2, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, m.sites);
  else if (dagger)
    wilson_f32_kernel<R, TPB, true, EPI_NONE, false><<<grid, TPB, 0, s>>>(m.links, in, nullptr, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, m.sites);
  else
    wilson_f32_kernel<R, TPB, false, EPI_NONE, false><<<grid, TPB, 0, s>>>(m.links, in, nullptr, out, g, kap, mu, nrhs, sc, aux, partial, status, mask, m.sites);
  return cudaGetLastError();
}

// Launch shape of the FP32 kernel for nrhs right-hand sides: the autotuned
// (R, threads per block) of the handle when there is one, else R = 1 and 128
// threads (the tuner's choice on 16^4 and 20^3 x 32 for 1 to 12 systems:
// R > 1 saves link loads from L2 but its registers cost more occupancy).
void wilson32_shape(const wd_context *h, int nrhs, int *R, int *T) {
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  if (h->tune_R[key] > 0) {
    *R = h->tune_R[key];
    *T = h->tune_T[key];
    return;
  }
  *R = 1;
  *T = 128;
}

cudaError_t launch_wilson_f32_shape(const Mixed32 &m, int R, int T, const float4 *in,
                                    const float4 *in2, float4 *out, int nrhs, int dagger, int epi,
                                    const BicgScalars *sc, const float4 *aux, double *partial,
                                    const int *status, unsigned mask, cudaStream_t s) {
#define W32(RR, TT) \
  if (R == RR && T == TT) return launch_w32<RR, TT>(m, in, in2, out, nrhs, dagger, epi, sc, aux, partial, status, mask, s);
  W32(1, 64) W32(1, 128) W32(1, 256)
  W32(2, 64) W32(2, 128) W32(2, 256)
  W32(4, 64) W32(4, 128) W32(4, 256)
#undef W32
  return cudaErrorInvalidValue;
}

cudaError_t launch_wilson_f32(const Mixed32 &m, const float4 *in, const float4 *in2, float4 *out,
                              int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s) {
  ProfLaunch prof(PC_DSLASH_LOW, s);
  int R, T;
  wilson32_shape(m.h, nrhs, &R, &T);
  Mixed32 mc = m;
  mc.sites = prof_site_counter_low();
  return launch_wilson_f32_shape(mc, R, T, in, in2, out, nrhs, dagger, epi, sc, aux, partial, status,
                                 mask, s);
}

int wilson32_blocks(const wd_context *h, int nrhs) {
  int R, T;
  wilson32_shape(h, nrhs, &R, &T);
  return (int)((h->V + T - 1) / T);
}

// Autotuner: time every (R, threads per block) on this lattice with nrhs
// right-hand sides (plain apply, CUDA events, best of 3 after a warm-up)
// and keep the fastest for the handle.  in and out: scratch FP32 vectors of
// nrhs * 6 V float4 each.
cudaError_t tune_wilson_f32(wd_context *h, const float4 *links, int nrhs, const float4 *in,
                            float4 *out, cudaStream_t s) {
  const Mixed32 m{h, links};
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
        err = launch_wilson_f32_shape(m, R, T, in, nullptr, out, nrhs, 0, EPI_NONE, nullptr, nullptr,
                                      nullptr, nullptr, M_ALL, s);
      float t_best = 1e30f;
      for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        err = launch_wilson_f32_shape(m, R, T, in, nullptr, out, nrhs, 0, EPI_NONE, nullptr, nullptr,
                                      nullptr, nullptr, M_ALL, s);
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
  const int key = nrhs < WD_TUNE_SLOTS ? nrhs : WD_TUNE_SLOTS - 1;
  h->tune_R[key] = bR;
  h->tune_T[key] = bT;
  h->tune_ms[key] = best;
  return cudaSuccess;
}

// ----------------------------------------------------------------- conversions

// FP64 links [V][4][3][3] -> FP32 rows 0, 1 in [mu][q][V] float4
__global__ void links_to_f32_kernel(const double2 *__restrict__ U, float4 *__restrict__ L,
                                    long long V) {
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const double2 *u = U + (s * 4 + mu) * 9;
      L[(mu * 3 + 0) * V + s] = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
      L[(mu * 3 + 1) * V + s] = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
      L[(mu * 3 + 2) * V + s] = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
    }
  }
}

cudaError_t launch_links_to_f32(const wd_context *h, float4 *L, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  links_to_f32_kernel<<<608, 256, 0, s>>>(h->links, L, h->V);
  return cudaGetLastError();
}

// boundary FP64 [rhs][V][12] -> FP32 [rhs][6][V]; optional partial <aux, out>
// (aux FP32) and ||in||^2 (FP64 input) for systems in mask.
__global__ void __launch_bounds__(256)
f64_to_f32_kernel(const double2 *__restrict__ in, float4 *__restrict__ out, long long V,
                  const float4 *__restrict__ aux, double *__restrict__ partial,
                  const int *__restrict__ status, unsigned mask) {
  const int r = blockIdx.y;
  if (status != nullptr && !((mask >> status[r]) & 1u)) return;
  double red[3] = {0.0, 0.0, 0.0};
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    const double2 *p = in + ((long long)r * V + s) * 12;
    float2 o[12];
    float2 a[12];
    if (aux) ld_spinor32(aux + (long long)r * 6 * V, V, s, a);
    float d0 = 0.f, d1 = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 v = p[c];
      o[c] = make_float2((float)v.x, (float)v.y);
      red[2] = fma(v.x, v.x, fma(v.y, v.y, red[2]));
      if (aux) {
        d0 = fmaf(a[c].x, o[c].x, fmaf(a[c].y, o[c].y, d0));
        d1 = fmaf(a[c].x, o[c].y, fmaf(-a[c].y, o[c].x, d1));
      }
    }
    red[0] += (double)d0;
    red[1] += (double)d1;
    st_spinor32(out + (long long)r * 6 * V, V, s, o);
  }
  if (partial != nullptr) {
    block_sum<3>(red);
    if (threadIdx.x == 0) {
      double *d = partial + ((long long)r * gridDim.x + blockIdx.x) * 3;
      d[0] = red[0];
      d[1] = red[1];
      d[2] = red[2];
    }
  }
}

// x64 += (double) xs (FP32), then xs = 0, for systems in mask
__global__ void __launch_bounds__(256)
add_f32_to_f64_kernel(double2 *__restrict__ x, float4 *__restrict__ xs, long long V,
                      const int *__restrict__ status, unsigned mask) {
  const int r = blockIdx.y;
  if (status != nullptr && !((mask >> status[r]) & 1u)) return;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    double2 *p = x + ((long long)r * V + s) * 12;
    float4 *q = xs + (long long)r * 6 * V;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const float4 f = q[g * V + s];
      p[2 * g] = make_double2(p[2 * g].x + (double)f.x, p[2 * g].y + (double)f.y);
      p[2 * g + 1] = make_double2(p[2 * g + 1].x + (double)f.z, p[2 * g + 1].y + (double)f.w);
      q[g * V + s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// FP32 [rhs][6][V] -> boundary FP64 [rhs][V][12]
__global__ void __launch_bounds__(256)
f32_to_f64_kernel(const float4 *__restrict__ in, double2 *__restrict__ out, long long V) {
  const int r = blockIdx.y;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V;
       s += (long long)gridDim.x * blockDim.x) {
    double2 *p = out + ((long long)r * V + s) * 12;
#pragma unroll
    for (int g = 0; g < 6; ++g) {
      const float4 f = __ldg(in + (long long)r * 6 * V + g * V + s);
      p[2 * g] = make_double2((double)f.x, (double)f.y);
      p[2 * g + 1] = make_double2((double)f.z, (double)f.w);
    }
  }
}

static unsigned conv_blocks(long long V) {
  long long b = (V + 255) / 256;
  return (unsigned)(b > 608 ? 608 : (b < 1 ? 1 : b));
}

int conv_blocks_count(long long V) { return (int)conv_blocks(V); }

cudaError_t launch_f64_to_f32(const double2 *in, float4 *out, long long V, int nrhs,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  f64_to_f32_kernel<<<dim3(conv_blocks(V), nrhs), 256, 0, s>>>(in, out, V, aux, partial, status, mask);
  return cudaGetLastError();
}

cudaError_t launch_add_f32_to_f64(double2 *x, float4 *xs, long long V, int nrhs,
                                  const int *status, unsigned mask, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  add_f32_to_f64_kernel<<<dim3(conv_blocks(V), nrhs), 256, 0, s>>>(x, xs, V, status, mask);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float4 *in, double2 *out, long long V, int nrhs,
                              cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  f32_to_f64_kernel<<<dim3(conv_blocks(V), nrhs), 256, 0, s>>>(in, out, V);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- BiCGStab (FP32 vectors)

__device__ __forceinline__ bool on32(const int *status, unsigned mask, int r) {
  return status == nullptr || ((mask >> status[r]) & 1u);
}

__device__ __forceinline__ float4 c2fma(float2 a, float4 b, float4 c) {  // c + a*b, b = 2 complex
  c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
  c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
  c.z = fmaf(a.x, b.z, fmaf(-a.y, b.w, c.z));
  c.w = fmaf(a.x, b.w, fmaf(a.y, b.z, c.w));
  return c;
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(256)
bicg32_update_p_kernel(float4 *__restrict__ p, const float4 *__restrict__ r,
                       const float4 *__restrict__ v, const BicgScalars *__restrict__ sc,
                       const int *__restrict__ status, long long n4) {
  const int q = blockIdx.y;
  if (!on32(status, M_ACTIVE, q)) return;  // uniform per block
  // beta in FP64 once per block (as in bicg_update_p_kernel)
  __shared__ float2 s_bm[2];
  if (threadIdx.x == 0) {
    const BicgScalars S = sc[q];
    s_bm[0] = f2(cmul(cdiv(S.rho, S.rho_old), cdiv(S.alpha, S.omega)));
    s_bm[1] = make_float2(-(float)S.omega.x, -(float)S.omega.y);
  }
  __syncthreads();
  const float2 beta = s_bm[0], mom = s_bm[1];
  const long long off = (long long)q * n4;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 t = c2fma(mom, v[off + i], p[off + i]);
    p[off + i] = c2fma(beta, t, r[off + i]);
  }
}

// s = r - alpha v; xs += alpha p + omega s; r = s - omega t; partial <rhat, r>, ||r||^2
__global__ void __launch_bounds__(256)
bicg32_update_xr_kernel(float4 *__restrict__ xs, float4 *__restrict__ r,
                        const float4 *__restrict__ p, const float4 *__restrict__ v,
                        const float4 *__restrict__ t, const float4 *__restrict__ rhat,
                        const BicgScalars *__restrict__ sc, const int *__restrict__ status,
                        double *__restrict__ partial, long long n4) {
  const int q = blockIdx.y;
  if (!on32(status, M_ACTIVE, q)) return;
  const float2 al = f2(sc[q].alpha), om = f2(sc[q].omega);
  const float2 mal = make_float2(-al.x, -al.y), mom = make_float2(-om.x, -om.y);
  const long long off = (long long)q * n4;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 sv = c2fma(mal, v[off + i], r[off + i]);
    float4 x = xs[off + i];
    x = c2fma(al, p[off + i], x);
    x = c2fma(om, sv, x);
    xs[off + i] = x;
    const float4 rn = c2fma(mom, t[off + i], sv);
    r[off + i] = rn;
    const float4 h = rhat[off + i];
    a0 = fmaf(h.x, rn.x, fmaf(h.y, rn.y, fmaf(h.z, rn.z, fmaf(h.w, rn.w, a0))));
    a1 = fmaf(h.x, rn.y, fmaf(-h.y, rn.x, fmaf(h.z, rn.w, fmaf(-h.w, rn.z, a1))));
    a2 = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, fmaf(rn.z, rn.z, fmaf(rn.w, rn.w, a2))));
  }
  __shared__ double sh[3][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float vals[3] = {a0, a1, a2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float vv = vals[k];
#pragma unroll
    for (int off2 = 16; off2 > 0; off2 >>= 1) vv += __shfl_down_sync(0xffffffffu, vv, off2);
    if (lane == 0) sh[k][w] = (double)vv;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double tot = 0.0;
    for (int w2 = 0; w2 < 8; ++w2) tot += sh[threadIdx.x][w2];
    partial[((long long)q * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = tot;
  }
}

// rhat = r, p = 0, v = 0, xs untouched
__global__ void __launch_bounds__(256)
bicg32_restart_kernel(float4 *__restrict__ rhat, const float4 *__restrict__ r,
                      float4 *__restrict__ p, float4 *__restrict__ v,
                      const int *__restrict__ status, unsigned mask, long long n4) {
  const int q = blockIdx.y;
  if (!on32(status, mask, q)) return;
  const long long off = (long long)q * n4;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    rhat[off + i] = r[off + i];
    p[off + i] = z;
    v[off + i] = z;
  }
}

int stream32_blocks(long long n4) {
  long long b = (n4 + 1023) / 1024;
  return (int)(b > 608 ? 608 : (b < 1 ? 1 : b));
}

cudaError_t launch_bicg32_update_p(float4 *p, const float4 *r, const float4 *v,
                                   const BicgScalars *sc, const int *status, long long n4,
                                   int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM_LOW, s);
  bicg32_update_p_kernel<<<dim3(stream32_blocks(n4), nrhs), 256, 0, s>>>(p, r, v, sc, status, n4);
  return cudaGetLastError();
}

cudaError_t launch_bicg32_update_xr(float4 *xs, float4 *r, const float4 *p, const float4 *v,
                                    const float4 *t, const float4 *rhat, const BicgScalars *sc,
                                    const int *status, double *partial, long long n4, int nrhs,
                                    cudaStream_t s) {
  ProfLaunch prof(PC_STREAM_LOW, s);
  bicg32_update_xr_kernel<<<dim3(stream32_blocks(n4), nrhs), 256, 0, s>>>(xs, r, p, v, t, rhat, sc,
                                                                         status, partial, n4);
  return cudaGetLastError();
}

cudaError_t launch_bicg32_restart(float4 *rhat, const float4 *r, float4 *p, float4 *v,
                                  const int *status, unsigned mask, long long n4, int nrhs,
                                  cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  bicg32_restart_kernel<<<dim3(stream32_blocks(n4), nrhs), 256, 0, s>>>(rhat, r, p, v, status, mask,
                                                                       n4);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- reliable update finalizer
// partial (NQ = 3): <rhat32, r32>, (unused), ||r64||^2 from f64_to_f32_kernel.
// A system is done when its FP64 residual meets tol_outer.  Otherwise, with
// restarted refinement (delta > 0), a system whose recursion reached its
// inner target, or every system when `force` is set, restarts the recurrence
// from the FP64 residual with the next inner target; the others continue
// with the replaced residual (reliable update).
__global__ void reliable_finalize_kernel(const double *__restrict__ partial, int nb,
                                         BicgScalars *sc, int *status, unsigned mask, int force) {
  const int r = blockIdx.x;
  const int st = status[r];
  if (!((mask >> st) & 1u)) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double *src = partial + ((long long)r * nb + b) * 3;
    v[0] += src[0];
    v[1] += src[1];
    v[2] += src[2];
  }
  block_sum<3>(v);
  if (threadIdx.x != 0) return;
  BicgScalars &S = sc[r];
  S.mvp_extra += 1;
  S.rnorm = sqrt(v[2]);
  S.true_rel = S.rnorm / S.bnorm;
  S.rho = make_double2(v[0], v[1]);  // <rhat, r> with the replaced residual
  if (st == ST_BREAKDOWN || st == ST_MAXITER) return;  // final: record only
  if (S.true_rel <= S.tol_outer) {
    status[r] = ST_DONE;
  } else if (S.delta > 0.0 && (st == ST_RECURSIVE || force)) {
    S.tol = fmax(S.tol_outer, S.delta * S.true_rel);
    S.rho = make_double2(v[2], 0.0);  // r_hat = r after the restart
    S.rho_old = make_double2(1.0, 0.0);
    S.alpha = make_double2(1.0, 0.0);
    S.omega = make_double2(1.0, 0.0);
    S.rhat_norm = S.rnorm;
    S.restarts += 1;
    status[r] = ST_RESTART;
  } else {
    status[r] = ST_ACTIVE;
  }
}

cudaError_t launch_reliable_finalize(const double *partial, int nb, BicgScalars *sc, int *status,
                                     unsigned mask, int nrhs, cudaStream_t s, int force) {
  ProfLaunch prof(PC_STREAM, s);
  reliable_finalize_kernel<<<nrhs, 256, 0, s>>>(partial, nb, sc, status, mask, force);
  return cudaGetLastError();
}

// First inner target of restarted refinement: delta x the initial residual.
__global__ void mixed_inner_tol_kernel(BicgScalars *sc, const int *status, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || status[r] != ST_ACTIVE) return;
  BicgScalars &S = sc[r];
  if (S.delta > 0.0) S.tol = fmax(S.tol_outer, S.delta * S.rnorm / S.bnorm);
}

cudaError_t launch_mixed_inner_tol(BicgScalars *sc, const int *status, int nrhs, cudaStream_t s) {
  ProfLaunch prof(PC_STREAM, s);
  mixed_inner_tol_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(sc, status, nrhs);
  return cudaGetLastError();
}

}  // namespace wd
