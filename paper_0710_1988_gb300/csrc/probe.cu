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
