// Spin projection and reconstruction of the Wilson hop, for complex128
// (double2) and complex64 (float2) arithmetic.
//
// Chiral basis: gamma_mu = [[0, B], [B^dagger, 0]] with B = -i sigma_k for
// mu = x, y, z and B = 1 for t.  Then
//   (1 - gamma_mu) psi = [h ; -B^dagger h],  h = psi_up - B psi_dn
//   (1 + gamma_mu) psi = [h ; +B^dagger h],  h = psi_up + B psi_dn
// so each hop needs two SU(3) mat-vecs on the half spinor h.  Spinor
// component c = 3*sigma + a (spin sigma, colour a).
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace wd {

__device__ __forceinline__ double2 sadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 ssub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 smuli(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 sadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 ssub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 smuli(float2 a) { return make_float2(-a.y, a.x); }

template <int MU, int S, class T>  // S = -1: (1 - gamma_mu), S = +1: (1 + gamma_mu)
__device__ __forceinline__ void project(const T (&p)[12], T (&h)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T p0 = p[a], p1 = p[3 + a], p2 = p[6 + a], p3 = p[9 + a];
    if (MU == 0) {        // B psi_dn = (-i p3, -i p2)
      h[a] = S < 0 ? sadd(p0, smuli(p3)) : ssub(p0, smuli(p3));
      h[3 + a] = S < 0 ? sadd(p1, smuli(p2)) : ssub(p1, smuli(p2));
    } else if (MU == 1) { // B psi_dn = (-p3, p2)
      h[a] = S < 0 ? sadd(p0, p3) : ssub(p0, p3);
      h[3 + a] = S < 0 ? ssub(p1, p2) : sadd(p1, p2);
    } else if (MU == 2) { // B psi_dn = (-i p2, i p3)
      h[a] = S < 0 ? sadd(p0, smuli(p2)) : ssub(p0, smuli(p2));
      h[3 + a] = S < 0 ? ssub(p1, smuli(p3)) : sadd(p1, smuli(p3));
    } else {              // B psi_dn = (p2, p3)
      h[a] = S < 0 ? ssub(p0, p2) : sadd(p0, p2);
      h[3 + a] = S < 0 ? ssub(p1, p3) : sadd(p1, p3);
    }
  }
}

// acc += [chi ; S * B^dagger chi]
template <int MU, int S, class T>
__device__ __forceinline__ void reconstruct(T (&acc)[12], const T (&c)[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T c0 = c[a], c1 = c[3 + a];
    acc[a] = sadd(acc[a], c0);
    acc[3 + a] = sadd(acc[3 + a], c1);
    if (MU == 0) {        // B^dagger chi = (i c1, i c0)
      acc[6 + a] = S < 0 ? ssub(acc[6 + a], smuli(c1)) : sadd(acc[6 + a], smuli(c1));
      acc[9 + a] = S < 0 ? ssub(acc[9 + a], smuli(c0)) : sadd(acc[9 + a], smuli(c0));
    } else if (MU == 1) { // B^dagger chi = (c1, -c0)
      acc[6 + a] = S < 0 ? ssub(acc[6 + a], c1) : sadd(acc[6 + a], c1);
      acc[9 + a] = S < 0 ? sadd(acc[9 + a], c0) : ssub(acc[9 + a], c0);
    } else if (MU == 2) { // B^dagger chi = (i c0, -i c1)
      acc[6 + a] = S < 0 ? ssub(acc[6 + a], smuli(c0)) : sadd(acc[6 + a], smuli(c0));
      acc[9 + a] = S < 0 ? sadd(acc[9 + a], smuli(c1)) : ssub(acc[9 + a], smuli(c1));
    } else {              // B^dagger chi = (c0, c1)
      acc[6 + a] = S < 0 ? ssub(acc[6 + a], c0) : sadd(acc[6 + a], c0);
      acc[9 + a] = S < 0 ? ssub(acc[9 + a], c1) : sadd(acc[9 + a], c1);
    }
  }
}

// Neighbour sites of s on the periodic lattice L (site = x + Lx(y + Ly(z + Lz t))).
struct Nbrs {
  long long up[4], dn[4];
};

__device__ __forceinline__ Nbrs neighbours(long long s, const int (&L)[4]) {
  Nbrs nb;
  const int x = (int)(s % L[0]);
  long long t1 = s / L[0];
  const int y = (int)(t1 % L[1]);
  t1 /= L[1];
  const int z = (int)(t1 % L[2]);
  const int t = (int)(t1 / L[2]);
  const long long sy = L[0], sz = sy * L[1], st = sz * L[2];
  nb.up[0] = x + 1 == L[0] ? s - (L[0] - 1) : s + 1;
  nb.dn[0] = x == 0 ? s + (L[0] - 1) : s - 1;
  nb.up[1] = y + 1 == L[1] ? s - (L[1] - 1) * sy : s + sy;
  nb.dn[1] = y == 0 ? s + (L[1] - 1) * sy : s - sy;
  nb.up[2] = z + 1 == L[2] ? s - (L[2] - 1) * sz : s + sz;
  nb.dn[2] = z == 0 ? s + (L[2] - 1) * sz : s - sz;
  nb.up[3] = t + 1 == L[3] ? s - (L[3] - 1) * st : s + st;
  nb.dn[3] = t == 0 ? s + (L[3] - 1) * st : s - st;
  return nb;
}

// The same for site indices below 2^31 (the FP32 / FP16 kernels), with
// 32-bit arithmetic and the geometry's multiply-shift divisions.
struct Nbrs32 {
  unsigned up[4], dn[4];
};

__device__ __forceinline__ unsigned fast_div(unsigned n, unsigned long long m, int sh) {
  return (unsigned)(((unsigned long long)n * m) >> sh);
}

__device__ __forceinline__ Nbrs32 neighbours32(unsigned s, const LatticeGeom &g) {
  Nbrs32 nb;
  const unsigned L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
  const unsigned q0 = fast_div(s, g.dm[0], g.dsh[0]);
  const unsigned x = s - q0 * L0;
  const unsigned q1 = fast_div(q0, g.dm[1], g.dsh[1]);
  const unsigned y = q0 - q1 * L1;
  const unsigned t = fast_div(q1, g.dm[2], g.dsh[2]);
  const unsigned z = q1 - t * L2;
  const unsigned sy = L0, sz = sy * L1, st = sz * L2;
  nb.up[0] = x + 1 == L0 ? s - (L0 - 1) : s + 1;
  nb.dn[0] = x == 0 ? s + (L0 - 1) : s - 1;
  nb.up[1] = y + 1 == L1 ? s - (L1 - 1) * sy : s + sy;
  nb.dn[1] = y == 0 ? s + (L1 - 1) * sy : s - sy;
  nb.up[2] = z + 1 == L2 ? s - (L2 - 1) * sz : s + sz;
  nb.dn[2] = z == 0 ? s + (L2 - 1) * sz : s - sz;
  nb.up[3] = t + 1 == L3 ? s - (L3 - 1) * st : s + st;
  nb.dn[3] = t == 0 ? s + (L3 - 1) * st : s - st;
  return nb;
}

}  // namespace wd
