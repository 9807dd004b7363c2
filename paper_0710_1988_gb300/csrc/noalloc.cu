// wd_apply_f32_noalloc: the FP32 Wilson apply of wd_apply_f32 for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need the operator:
// a process that has handed all of its device memory to another allocator
// up front (a framework's caching allocator, a fixed memory budget), and
// code that must not synchronise the device (cudaMalloc and cudaFree may).
// wd_apply_f32 needs two FP32 staging vectors and the FP32 copy of the
// links, which it takes from the handle's pool; this variant keeps all three
// in one file-scope __device__ array instead, so a call allocates nothing.
// The array is WD_NOALLOC_SCRATCH_BYTES (64 MiB) on every GPU that loads the
// library, held until the process exits.
//
// A call needs V * (12 + 12 * nrhs) float4 of it (FP32 links, then the input
// and output vectors); larger requests are rejected with WD_BAD_ARG.  Every
// region a call reads is written earlier in the same call, so nothing has to
// start at zero.  Because the array is shared, the FP32 links are rebuilt
// from the handle's FP64 links on every call (about 768 bytes of traffic per
// site), so at small nrhs a call costs more than wd_apply_f32, which keeps
// its FP32 links.  All calls share the array: calls whose GPU work overlaps
// (other streams, other handles, other threads) race and must be ordered by
// the caller.  The first call on each device looks up the array's device
// address (cudaGetSymbolAddress, with that device current) and keeps it for
// the rest of the process; make that first call before any stream capture.
// The address belongs to the device's primary context, the one the CUDA
// runtime uses: a caller that resets the device (cudaDeviceReset) or runs
// under another context it created must not call this entry point afterwards.
#include <mutex>

#include "kernels.cuh"
#include "mixed.h"
#include "wd_internal.h"

namespace wd {

constexpr size_t kNoallocFloat4 = WD_NOALLOC_SCRATCH_BYTES / sizeof(float4);

static __device__ __align__(256) float4 g_noalloc_scratch[kNoallocFloat4];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float4 *g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device (set-up once).
static int noalloc_scratch(int device, float4 **out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("wd_apply_f32_noalloc: device ordinal out of range");
    return WD_BAD_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[device] == nullptr) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "wd_apply_f32_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[device] = static_cast<float4 *>(p);
  }
  *out = g_scratch_ptr[device];
  return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_apply_f32_noalloc(wd_handle h, const void *in, void *out, int nrhs,
                                    int dagger, wd_stream stream) {
  ProfScope prof_scope_(h ? &h->prof : nullptr);
  if (h == nullptr || in == nullptr || out == nullptr) {
    set_error("wd_apply_f32_noalloc: NULL argument");
    return WD_BAD_ARG;
  }
  if (h->eo) {
    set_error("wd_apply_f32_noalloc: the FP32 kernel acts on the full operator");
    return WD_BAD_ARG;
  }
  if (nrhs < 1 || nrhs > 65535) {
    set_error("wd_apply_f32_noalloc: nrhs must be in [1, 65535]");
    return WD_BAD_ARG;
  }
  const size_t need = (size_t)h->V * (12 + 12 * (size_t)nrhs);
  if (need > kNoallocFloat4) {
    set_error("wd_apply_f32_noalloc: V * (12 + 12 * nrhs) = " + std::to_string(need) +
              " float4 exceeds the static scratch of " + std::to_string(kNoallocFloat4) +
              " float4 (64 MiB); use wd_apply_f32");
    return WD_BAD_ARG;
  }
  if (!is_device_pointer(in) || !is_device_pointer(out)) {
    set_error("wd_apply_f32_noalloc: in and out must be device pointers");
    return WD_BAD_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "wd_apply_f32_noalloc: cudaGetDevice");
  if (dev != h->device) {
    set_error("wd_apply_f32_noalloc: the handle's device must be current");
    return WD_BAD_ARG;
  }
  float4 *scratch = nullptr;
  int rc = noalloc_scratch(dev, &scratch);
  if (rc != WD_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float4 *links32 = scratch;                              // 12 V
  float4 *a = links32 + 12 * (size_t)h->V;                // 6 V nrhs
  float4 *b = a + 6 * (size_t)h->V * nrhs;                // 6 V nrhs
  const Mixed32 m{h, links32};
  e = launch_links_to_f32(h, links32, s);
  if (e == cudaSuccess)
    e = launch_f64_to_f32(static_cast<const double2 *>(in), a, h->V, nrhs, nullptr, nullptr,
                          nullptr, M_ALL, s);
  if (e == cudaSuccess)
    e = launch_wilson_f32(m, a, nullptr, b, nrhs, dagger ? 1 : 0, EPI_NONE, nullptr, nullptr,
                          nullptr, nullptr, M_ALL, s);
  if (e == cudaSuccess) e = launch_f32_to_f64(b, static_cast<double2 *>(out), h->V, nrhs, s);
  if (e != cudaSuccess) return cuda_fail(e, "wd_apply_f32_noalloc");
  return WD_OK;
}
