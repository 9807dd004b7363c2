// FP32-storage kernels of the mixed-precision solver (see mixed.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "wd_internal.h"

namespace wd {

struct Mixed32 {
  const wd_context *h;
  const float4 *links;  // [mu][3][V] float4, rows 0 and 1 of every link
  unsigned long long *sites = nullptr;  // profiler's work counter (or nullptr)
};

// launch shape (right-hand sides per thread, threads per block) and grid
void wilson32_shape(const wd_context *h, int nrhs, int *R, int *T);
int wilson32_blocks(const wd_context *h, int nrhs);
cudaError_t tune_wilson_f32(wd_context *h, const float4 *links, int nrhs, const float4 *in,
                            float4 *out, cudaStream_t s);
int stream32_blocks(long long n4);
int conv_blocks_count(long long V);

// out = A in (FP32 [rhs][6][V]); epi as for the FP64 kernel; EPI_TSTT applies
// A to s = in - alpha in2 (alpha from sc) and reduces <out, s>, ||out||^2.
cudaError_t launch_wilson_f32(const Mixed32 &m, const float4 *in, const float4 *in2, float4 *out,
                              int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s);
cudaError_t launch_links_to_f32(const wd_context *h, float4 *L, cudaStream_t s);
// boundary FP64 -> FP32; partial (3 per block): <aux, out>, 0, ||in||^2 when
// partial != nullptr (conv_blocks_count(V) blocks per system).
cudaError_t launch_f64_to_f32(const double2 *in, float4 *out, long long V, int nrhs,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s);
cudaError_t launch_add_f32_to_f64(double2 *x, float4 *xs, long long V, int nrhs,
                                  const int *status, unsigned mask, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float4 *in, double2 *out, long long V, int nrhs,
                              cudaStream_t s);
cudaError_t launch_bicg32_update_p(float4 *p, const float4 *r, const float4 *v,
                                   const BicgScalars *sc, const int *status, long long n4,
                                   int nrhs, cudaStream_t s);
cudaError_t launch_bicg32_update_xr(float4 *xs, float4 *r, const float4 *p, const float4 *v,
                                    const float4 *t, const float4 *rhat, const BicgScalars *sc,
                                    const int *status, double *partial, long long n4, int nrhs,
                                    cudaStream_t s);
cudaError_t launch_bicg32_restart(float4 *rhat, const float4 *r, float4 *p, float4 *v,
                                  const int *status, unsigned mask, long long n4, int nrhs,
                                  cudaStream_t s);
// ----------------------------------------------------------------- FP16 storage (mixed16.cu)
// Half vector: uint4 [rhs][3][V] of __half2 (re, im) scaled by a per-site
// norm float [rhs][V]; 52 bytes per site.
struct Half16 {
  uint4 *v;
  float *n;
};
void wilson16_shape(const wd_context *h, int nrhs, int *R, int *T);
int wilson16_blocks(const wd_context *h, int nrhs);
cudaError_t tune_wilson_f16(wd_context *h, const uint2 *links, int nrhs, Half16 in, Half16 out,
                            cudaStream_t s);
int stream16_blocks(long long V);
// out = A in (half), epi as launch_wilson_f32; EPI_TSTT applies A to
// s = r32 - alpha in and reduces <out, s>, ||out||^2.
cudaError_t launch_wilson_f16(const wd_context *h, const uint2 *links, Half16 in, const float4 *r32,
                              Half16 out, int nrhs, int dagger, int epi, const BicgScalars *sc,
                              const float4 *aux, double *partial, const int *status,
                              unsigned mask, cudaStream_t s);
cudaError_t launch_links_to_f16(const wd_context *h, uint2 *L, cudaStream_t s);
cudaError_t launch_f64_to_f16(const double2 *in, Half16 out, long long V, int nrhs, cudaStream_t s);
cudaError_t launch_f16_to_f64(Half16 in, double2 *out, long long V, int nrhs, cudaStream_t s);
cudaError_t launch_bicg16_update_p(Half16 p, const float4 *r, Half16 v, const BicgScalars *sc,
                                   const int *status, long long V, int nrhs, cudaStream_t s);
cudaError_t launch_bicg16_update_xr(float4 *xs, float4 *r, Half16 p, Half16 v, Half16 t,
                                    const float4 *rhat, const BicgScalars *sc, const int *status,
                                    double *partial, long long V, int nrhs, cudaStream_t s);
cudaError_t launch_bicg16_restart(float4 *rhat, const float4 *r, Half16 p, Half16 v,
                                  const int *status, unsigned mask, long long V, int nrhs,
                                  cudaStream_t s);

// ----------------------------------------------------------------- FP32 Schur operator (mixed_eo.cu)
// out = A_hat in on even half vectors (float4 [rhs][6][V/2]); tmp: an odd
// half vector per system; epi / FUSED as launch_wilson_f32.
int schur32_blocks(const wd_context *h);
cudaError_t launch_schur_f32(const Mixed32 &m, const float4 *in, const float4 *in2, float4 *out,
                             float4 *tmp, int nrhs, int dagger, int epi, const BicgScalars *sc,
                             const float4 *aux, double *partial, const int *status,
                             unsigned mask, cudaStream_t s);

cudaError_t launch_reliable_finalize(const double *partial, int nb, BicgScalars *sc, int *status,
                                     unsigned mask, int nrhs, cudaStream_t s, int force = 0);
cudaError_t launch_mixed_inner_tol(BicgScalars *sc, const int *status, int nrhs, cudaStream_t s);

}  // namespace wd
