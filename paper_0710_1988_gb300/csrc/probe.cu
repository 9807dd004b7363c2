// FP64 fused multiply-add throughput probe: the measured denominator of the
// FP64 kernels' roofline (every FP64 kernel of the solver path is bound by
// the FP64 pipe on this GPU, not by HBM).
//
// Each thread runs kChains independent chains acc = fma(acc, a, b) for
// `iters` steps (a < 1, so every chain converges to b / (1 - a) and no value
// overflows or becomes subnormal); a result that can never occur is stored to
// keep the chains live.  2 flops per FMA.
#include "wd_internal.h"

namespace wd {

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;
__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1e-3 * threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == -1.0) g_probe_sink = s;  // never true: every chain stays positive
}
}  // namespace

}  // namespace wd

using namespace wd;

extern "C" int wd_probe_fp64_peak(int iters, int reps, double *tflops, double *ms,
                                  wd_stream stream) {
  if (iters < 1 || iters > (1 << 24) || reps < 1 || reps > 1000 || tflops == nullptr) {
    set_error("wd_probe_fp64_peak: iters in [1, 2^24], reps in [1, 1000], tflops not NULL");
    return WD_BAD_ARG;
  }
  int dev = 0, sms = 0;
  WD_CK(cudaGetDevice(&dev));
  WD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * sms;  // 4 blocks of 256 threads per SM: 32 warps
  cudaStream_t s = (cudaStream_t)stream;
  dfma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7);  // warm-up
  WD_CK_LAUNCH("dfma_probe_kernel");
  cudaEvent_t e0, e1;
  WD_CK(cudaEventCreate(&e0));
  WD_CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    dfma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters, 0.999999, 1e-7);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "wd_probe_fp64_peak");
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads * reps;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t / reps;
  return WD_OK;
}

// ----------------------------------------------------------------- BF16 MMA throughput
//
// tcgen05 BF16 MMAs with FP32 accumulation, M = 128, N = 256, K = 16, one
// CTA per SM issuing `iters` MMAs into one tensor-memory accumulator from
// operands resident in shared memory (K-major, no swizzle): the tensor-core
// rate the exact-split contraction draws on.  The completion wait is bounded
// (one second) and sets the error flag instead of spinning on.
namespace wd {
namespace {
__device__ int g_mma_probe_err;

__device__ __forceinline__ uint32_t probe_smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t probe_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128) bf16_mma_probe_kernel(int iters, float *sink) {
  __shared__ __align__(128) unsigned short sa[128 * 16];
  __shared__ __align__(128) unsigned short sb[256 * 16];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase;
  const int t = threadIdx.x;
  for (int i = t; i < 128 * 16; i += 128) sa[i] = 0x3C80;   // 1/64 in BF16
  for (int i = t; i < 256 * 16; i += 128) sb[i] = 0x3C80;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(probe_smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;"
                 ::"r"(probe_smem_u32(&tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tm = tbase;
  if (t == 0) {
    const uint64_t da = probe_desc(probe_smem_u32(sa)), db = probe_desc(probe_smem_u32(sb));
    const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                        ((uint32_t)(128 >> 4) << 24);
    for (int i = 0; i < iters; ++i)
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
          ::"r"(tm), "l"(da), "l"(db), "r"(id), "r"(i > 0 ? 1 : 0));
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(probe_smem_u32(&bar)));
  }
  unsigned long long t0, tn;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (int i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(probe_smem_u32(&bar)));
    if (ok) break;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(tn));
    if (tn - t0 > 1000000000ull) {
      atomicExch(&g_mma_probe_err, 1);
      break;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  uint32_t v;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
               : "=r"(v)
               : "r"(tm + ((uint32_t)(32 * (t / 32)) << 16)));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
  if (__uint_as_float(v) == -1.0f) sink[t] = 1.0f;   // never: keeps the accumulator live
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tm));
}
}  // namespace
}  // namespace wd

extern "C" int wd_probe_bf16_mma_peak(int iters, int reps, double *tflops, double *ms,
                                      wd_stream stream) {
  if (iters < 1 || iters > (1 << 20) || reps < 1 || reps > 100 || tflops == nullptr) {
    set_error("wd_probe_bf16_mma_peak: iters in [1, 2^20], reps in [1, 100], tflops not NULL");
    return WD_BAD_ARG;
  }
  int dev = 0, sms = 0;
  WD_CK(cudaGetDevice(&dev));
  WD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  float *sink = nullptr;
  WD_CK(cudaMallocAsync(&sink, 128 * sizeof(float), s));
  const int zero = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_mma_probe_err, &zero, sizeof(int), 0,
                                          cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    bf16_mma_probe_kernel<<<sms, 128, 0, s>>>(iters, sink);   // warm-up
    e = cudaGetLastError();
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    bf16_mma_probe_kernel<<<sms, 128, 0, s>>>(iters, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float tms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&tms, e0, e1);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&herr, g_mma_probe_err, sizeof(int));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (e != cudaSuccess) return cuda_fail(e, "wd_probe_bf16_mma_peak");
  if (herr) {
    set_error("wd_probe_bf16_mma_peak: an MMA completion wait gave up");
    return WD_TIMEOUT;
  }
  *tflops = 2.0 * 128 * 256 * 16 * (double)iters * sms * reps / (tms * 1e-3) / 1e12;
  if (ms) *ms = tms / reps;
  return WD_OK;
}
