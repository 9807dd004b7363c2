// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wd.h"
#include "profile.h"

namespace wd {

// ----------------------------------------------------------------- errors

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define WD_CK(call)                                                      \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::wd::cuda_fail(e_, #call);           \
  } while (0)

#define WD_CK_LAUNCH(what)                                               \
  do {                                                                   \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) return ::wd::cuda_fail(e_, what);            \
  } while (0)

// ----------------------------------------------------------------- memory

// Stream-ordered device scratch: every take() is a cudaMallocFromPoolAsync on
// the handle's own memory pool (release threshold = unlimited, so freed
// blocks stay cached for the next call), and release() frees them all on
// the same stream.  A failed take() returns nullptr and sets `failed`.
struct Arena {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<void *> ptrs;
  bool failed = false;
  template <class T> T *take(size_t count) {
    void *p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes < 256) bytes = 256;
    if (failed || cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return reinterpret_cast<T *>(p);
  }
  void release() {
    for (void *p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
  }
};

inline size_t aligned_bytes(size_t b) { return (b + 255) & ~size_t(255); }

// Pointer classification for "device or host" arguments.
bool is_device_pointer(const void *p);

}  // namespace wd

// Autotuner slots: nrhs = 1..WD_TUNE_SLOTS-2 each, larger nrhs share the last.
#define WD_TUNE_SLOTS 34

// The handle.
struct wd_context {
  int dims[4];
  long long V;      // sites
  long long n;      // 12 V complex numbers per spinor
  double kappa;
  double mu;
  int device;
  double2 *links;   // device, [V][4][3][3] complex128
  cudaMemPool_t pool;  // this handle's scratch pool
  wd::Profiler prof;   // optional kernel timing
  float4 *links32;     // FP32 rows 0, 1 of every link (mixed precision), lazily built
  uint2 *links16;      // FP16 links, all nine entries (5 uint2 per link), lazily built
  int mixed_bits;      // storage of the mixed solver's Krylov vectors: 32 or 16
  double mixed_delta;  // 0: reliable updates; > 0: restarted refinement (inner reduction)
  int mixed_inner_max; // restarted refinement: iterations before a forced restart
  cudaStream_t side;   // non-blocking stream for graph capture when the caller
                       // passes the legacy default stream; lazily created
  cudaEvent_t ev_in, ev_out;
  int tune_R[WD_TUNE_SLOTS];   // autotuned FP32 launch shape per nrhs (0: not tuned)
  int tune_T[WD_TUNE_SLOTS];
  float tune_ms[WD_TUNE_SLOTS];
  int tune16_R[WD_TUNE_SLOTS];  // the same for the FP16-storage kernel
  int tune16_T[WD_TUNE_SLOTS];
  float tune16_ms[WD_TUNE_SLOTS];
  int eo;              // 1: the operator is the even-odd Schur complement on even sites
  double2 *eo_tmp;     // odd half-vector scratch of the Schur operator
  size_t eo_tmp_cap;   // complex numbers
  std::vector<double> gmresdr_hist;  // last GMRES-DR solve: residual / ||r0|| per cycle
  int tc_contract;     // 1: wide V*Y products on the tensor cores (exact-split), 0: FP64
  int eig32;           // 1: harmonic Ritz values from FP32 estimates refined in FP64, 0: FP64 QR
};

// Length (complex numbers) of the vectors the solvers work on.
inline long long op_n(const wd_context *h) { return h->eo ? h->n / 2 : h->n; }

struct wd_deflation_space {
  wd_context *h;
  int k;
  double2 *V;       // [k][n]
  double2 *U;       // [k][n], nullptr means gamma5 V
  double2 *W;       // [k][n] = A V
  double2 *LU;      // [k][k] row-major LU factors of G = U^dagger A V
  int *piv;         // [k]
  double kappa, mu; // operator parameters W and G were built for
};

namespace wd {

// ----------------------------------------------------------------- kernels
// Every launcher enqueues on `s` and returns cudaGetLastError().

// out[r] = A in[r] (dagger: A^dagger), r < nrhs; n-vectors in boundary layout.
cudaError_t launch_wilson_f64(const wd_context *h, const double2 *in,
                              double2 *out, int nrhs, int dagger,
                              cudaStream_t s);

}  // namespace wd
