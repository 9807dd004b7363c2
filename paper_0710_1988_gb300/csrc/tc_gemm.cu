// OUT[c] = (beta_one ? IN[c] : 0) + sign * sum_r V[r] * Y[r][c] for complex128
// vectors of length n, on the tensor cores (tcgen05, BF16 inputs, FP32
// accumulation in tensor memory), to FP64 accuracy.
//
// This is the contraction of GMRES-DR's restart, V_{k+1} = V_{m+1} P_{k+1}
// (Sec. 1), and of the projection's updates x0 += V y, r0 -= (A V) y
// (Sec. 2): M = n rows, K = 2 kv real values per row, N = 2 ncol real
// columns.  It is exact-split emulation (Ozaki's scheme): every FP64 value
// of a row of V (or a column of Y) is written as a fixed-point number
// relative to the largest exponent of its row (column) and split into
// eight balanced 7-bit digits, |d| <= 64, each exact in BF16.  Digit pairs
// whose significance levels sum to L <= 7 are accumulated in one FP32
// tensor-memory accumulator per level; every product is an integer of at
// most 2^12, and a level holds at most 8 pairs x 2 * 88 rows of them, so
// each accumulator stays an exact integer below 2^24 and no rounding happens
// before the epilogue combines the eight levels in FP64 (Horner) and
// applies the two exponents.  The pairs with a + b > 7 and the rounding of
// values smaller than their row's maximum to 55 fixed-point bits leave an
// error of a few units of 2^-53 relative to (row maximum) x (column
// maximum), the size of an FP64 product's own rounding.  Inputs must be
// finite; subnormal inputs count as zero.
//
// Layout.  A CTA owns one 128-row tile and one 24-complex-column (48 real)
// tile of OUT at a time (persistent grid, one CTA per SM).  The BF16 digit
// planes live in shared memory in the tensor cores' K-major layout without
// swizzle: 8x8 core matrices of 16-byte rows, the K-adjacent core matrix
// 128 bytes on, the next 8-row group 256 bytes on.  Per K-chunk of 16 the
// A digits (8 planes x 128 rows) are double-buffered; all digit planes of
// Y for the column tile stay resident.  Tensor memory: 8 levels x 48
// columns.
#include <cstdint>

#include "kernels.cuh"
#include "wd_internal.h"

namespace wd {

namespace {

constexpr int TC_ROWS = 128;          // rows of OUT per tile (MMA M)
constexpr int TC_CCOLS = 24;          // complex columns per tile
constexpr int TC_NCOLS = 48;          // real columns per tile (MMA N)
constexpr int TC_DIGITS = 8;          // balanced 7-bit digits per value
constexpr int TC_LEVELS = 8;          // accumulated significance levels
constexpr int TC_MAXKV = 88;          // complex rows of V: K = 2 kv <= 176
constexpr int TC_MAXCH = 2 * TC_MAXKV / 16;   // K-chunks of 16
constexpr int TC_THREADS = 256;
constexpr int A_PLANE = TC_ROWS * 16 * 2;     // bytes of one digit plane, one chunk
constexpr int A_BUF = TC_DIGITS * A_PLANE;    // 32 KB
constexpr int B_BLOCK = TC_NCOLS * 16 * 2;    // one digit plane of Y, one chunk: 1536 B
constexpr int TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1LL << 24;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a K-major no-swizzle operand tile
__device__ __forceinline__ int core_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;       // K-adjacent core matrices
  d |= (uint64_t)(256 >> 4) << 32;       // next 8-row group
  d |= (uint64_t)1 << 46;                // tcgen05 descriptor version
  return d;                              // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((uint32_t)(TC_NCOLS >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}

// true once the phase with this parity has completed; false after the limit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *out) {
  uint32_t v[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 8; ++i) out[i] = __uint_as_float(v[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }

// biased exponent field of a double (0 for zero and subnormals)
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// x as the integer X = x * 2^(1077 - E) (|X| < 2^55), E >= x's exponent field
__device__ __forceinline__ long long fixed_point(double x, int E) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  if (be == 0) return 0;                               // zero or subnormal
  long long M = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
  const int sh = be - E + 2;                           // <= 2
  if (sh >= 0) {
    M <<= sh;
  } else if (sh > -60) {
    M = (M + (1LL << (-sh - 1))) >> (-sh);             // round half up
  } else {
    M = 0;
  }
  return bits < 0 ? -M : M;
}

// BF16 bits of a small integer d, |d| <= 64 (exact: at most 7 significant bits)
__device__ __forceinline__ uint32_t bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// the eight balanced digits of X, most significant first, as BF16 bits
__device__ __forceinline__ void digits_bf16(long long X, uint32_t *d) {
#pragma unroll
  for (int s = 0; s < TC_DIGITS - 1; ++s) {
    const int w = 7 * (TC_DIGITS - 1 - s);             // 49, 42, ..., 7
    const long long q = (X + (1LL << (w - 1))) >> w;   // round half up, |q| <= 64
    X -= q << w;
    d[s] = bf16_of_int((int)q);
  }
  d[TC_DIGITS - 1] = bf16_of_int((int)X);              // |X| <= 64
}

}  // namespace


// ----------------------------------------------------------------- Y digits

// Real column j = 2 c' + o of column tile t (complex column c = 24 t + c',
// o = 0 real part of OUT, 1 imaginary part) against K index k = 2 r + p
// (p = 0 real part of V, 1 imaginary part):
//   o = 0: p = 0 -> Re Y[r][c],  p = 1 -> -Im Y[r][c]
//   o = 1: p = 0 -> Im Y[r][c],  p = 1 ->  Re Y[r][c]
// times `sign`.  One warp per real column: its exponent field (maximum over
// the column), then the digit planes Bd[t][s][q] (q = K-chunk), each in the
// K-major core-matrix layout, and F[j] = the exponent field.
__device__ __forceinline__ double y_value(const double2 *Y, int ldy, int kv, int ncol,
                                          double sign, int j, int k) {
  const int c = (j >> 1), o = j & 1;
  const int r = k >> 1, p = k & 1;
  if (c >= ncol || r >= kv) return 0.0;
  const double2 y = Y[(long long)r * ldy + c];
  double v = o == 0 ? (p == 0 ? y.x : -y.y) : (p == 0 ? y.y : y.x);
  return sign * v;
}

__global__ void __launch_bounds__(256)
tc_prep_y_kernel(const double2 *__restrict__ Y, int ldy, int kv, int ncol, double sign,
                 int nch, unsigned char *__restrict__ Bd, int *__restrict__ F) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int jg = blockIdx.x * 8 + warp;             // global real column
  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  if (jg >= ntile * TC_NCOLS) return;
  const int t = jg / TC_NCOLS, jj = jg % TC_NCOLS;
  const int j = t * TC_NCOLS + jj;                  // real column over all tiles
  const int K = 16 * nch;
  int E = 0;
  for (int k = lane; k < K; k += 32) E = max(E, exp_field(y_value(Y, ldy, kv, ncol, 1.0, j, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xFFFFFFFFu, E, o));
  if (lane == 0) F[jg] = E;
  for (int k = lane; k < K; k += 32) {
    uint32_t d[TC_DIGITS];
    digits_bf16(fixed_point(y_value(Y, ldy, kv, ncol, sign, j, k), E), d);
    const int q = k >> 4, kk = k & 15;
#pragma unroll
    for (int s = 0; s < TC_DIGITS; ++s) {
      unsigned char *blk = Bd + ((long long)(t * TC_DIGITS + s) * nch + q) * B_BLOCK;
      *reinterpret_cast<uint16_t *>(blk + core_off(jj, kk)) = (uint16_t)d[s];
    }
  }
}


// ----------------------------------------------------------------- main kernel

__device__ __forceinline__ double scale_pow2(double h, int e) {
  // h * 2^e through the exponent field when the result stays normal
  const long long b = __double_as_longlong(h);
  const int be = (int)((b >> 52) & 0x7FF);
  if (h == 0.0) return 0.0;
  if (be + e >= 1 && be + e <= 2046 && be != 0) return __longlong_as_double(b + ((long long)e << 52));
  return ldexp(h, e);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_tsgemm_kernel(const double2 *__restrict__ V, int kv, long long n, int nch,
                 const unsigned char *__restrict__ Bd, const int *__restrict__ F, int ncol,
                 const double2 *IN, double2 *OUT, int beta_one, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sB = smem;                                  // 8 x nch x 1536
  unsigned char *sA = smem + TC_DIGITS * nch * B_BLOCK;      // 2 x 32 KB
  int *sE = reinterpret_cast<int *>(sA + 2 * A_BUF);         // [2][128]
  uint64_t *bars = reinterpret_cast<uint64_t *>(sE + 2 * TC_ROWS);
  uint32_t *tbase = reinterpret_cast<uint32_t *>(bars + 2);

  const int t = threadIdx.x;
  const int row = t & (TC_ROWS - 1), half = t >> 7;
  if (t == 0) {
    mbar_init(&bars[0]);
    mbar_init(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tbase)), "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tm = *tbase;

  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  const long long nrt = (n + TC_ROWS - 1) / TC_ROWS;
  const long long ntiles = nrt * ntile;
  int loaded = -1;
  long long committed = 0;      // K-chunks whose MMAs were committed (all tiles)
  bool abort = false;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ct = (int)(tile / nrt);
    const long long i0 = (tile % nrt) * TC_ROWS;
    const long long i = i0 + row;
    const bool valid = i < n;
    // Y digit planes of this column tile (every MMA of the previous tile has
    // completed: waited for below before its epilogue)
    if (ct != loaded) {
      const uint4 *src = reinterpret_cast<const uint4 *>(Bd + (long long)ct * TC_DIGITS * nch * B_BLOCK);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      for (int e = t; e < TC_DIGITS * nch * B_BLOCK / 16; e += TC_THREADS) dst[e] = src[e];
      loaded = ct;
    }
    // exponent field of each row: maximum over its 2 kv values (two halves)
    int E = 0;
    if (valid) {
      for (int q = 0; q < nch; ++q) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 8 * q + 4 * half + u;
          if (r < kv) {
            const double2 v = V[(long long)r * n + i];
            E = max(E, max(exp_field(v.x), exp_field(v.y)));
          }
        }
      }
    }
    sE[half * TC_ROWS + row] = E;
    __syncthreads();
    E = max(sE[row], sE[TC_ROWS + row]);

    // this thread's 8 K values of chunk q: rows r = 8q + 4 half + u, re and im;
    // the next chunk's values are loaded while this chunk's digits are formed
    double2 vcur[4], vnext[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * half + u;
      vcur[u] = (valid && r < kv) ? V[(long long)r * n + i] : make_double2(0.0, 0.0);
    }
    for (int q = 0; q < nch; ++q) {
      const long long g = committed;            // this chunk's global index
      const int b = (int)(g & 1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 8 * (q + 1) + 4 * half + u;
        vnext[u] = (valid && q + 1 < nch && r < kv) ? V[(long long)r * n + i]
                                                    : make_double2(0.0, 0.0);
      }
      bool ok = true;
      if (g >= 2) ok = mbar_wait(&bars[b], (uint32_t)(((g - 2) >> 1) & 1));
      unsigned char *buf = sA + b * A_BUF;
      if (ok) {
        uint32_t d[8][TC_DIGITS];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          digits_bf16(fixed_point(vcur[u].x, E), d[2 * u]);
          digits_bf16(fixed_point(vcur[u].y, E), d[2 * u + 1]);
        }
#pragma unroll
        for (int sl = 0; sl < TC_DIGITS; ++sl) {
          uint4 w;
          w.x = d[0][sl] | (d[1][sl] << 16);
          w.y = d[2][sl] | (d[3][sl] << 16);
          w.z = d[4][sl] | (d[5][sl] << 16);
          w.w = d[6][sl] | (d[7][sl] << 16);
          *reinterpret_cast<uint4 *>(buf + sl * A_PLANE + core_off(row, 8 * half)) = w;
        }
        fence_async_smem();
      }
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
      if (t == 0) {
        fence_after();
        const uint32_t aBase = smem_u32(buf);
        const uint32_t bBase = smem_u32(sB);
#pragma unroll 1
        for (int a = 0; a < TC_DIGITS; ++a) {
          const uint64_t da = smem_desc(aBase + a * A_PLANE);
#pragma unroll 1
          for (int bb = 0; a + bb < TC_LEVELS; ++bb) {
            const uint64_t db = smem_desc(bBase + (bb * nch + q) * B_BLOCK);
            mma_bf16(tm + (uint32_t)((a + bb) * TC_NCOLS), da, db, (q > 0 || a > 0) ? 1u : 0u);
          }
        }
        mma_commit(&bars[b]);
      }
      ++committed;
#pragma unroll
      for (int u = 0; u < 4; ++u) vcur[u] = vnext[u];
    }
    if (abort) break;
    // every MMA of this tile: the last commit tracks all earlier ones
    {
      const long long gl = committed - 1;
      const bool ok = mbar_wait(&bars[gl & 1], (uint32_t)((gl >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        abort = true;
        break;
      }
    }
    fence_after();
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (its rows) and the
    // real columns 24 (w / 4) .. + 23 of the tile, 8 at a time
    const int w = t >> 5;
    const int er = 32 * (w & 3) + (t & 31);
    const long long ie = i0 + er;
    const int Erow = max(sE[er], sE[TC_ROWS + er]);
    const uint32_t lane_addr = (uint32_t)(32 * (w & 3)) << 16;
#pragma unroll 1
    for (int cg = 0; cg < 3; ++cg) {
      const int c0 = 24 * (w >> 2) + 8 * cg;
      float acc[TC_LEVELS][8];
#pragma unroll
      for (int L = 0; L < TC_LEVELS; ++L) tmem_ld8(tm + lane_addr + (uint32_t)(L * TC_NCOLS + c0), acc[L]);
      if (ie < n) {
#pragma unroll
        for (int cc = 0; cc < 8; cc += 2) {
          const int jg = ct * TC_NCOLS + c0 + cc;         // real column (re part)
          const int c = jg >> 1;
          if (c >= ncol) continue;
          double res[2];
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            // the level sums are exact integers below 2^24: combine them in
            // 64-bit integers, levels 0-3 and 4-7 (each below 2^45), and
            // leave one rounding to FP64: sum_L A_L 2^(-7L) = (hi 2^28 + lo) 2^-49
            long long hi = 0, lo = 0;
#pragma unroll
            for (int L = 0; L < 4; ++L) hi = hi * 128 + __float2int_rn(acc[L][cc + o]);
#pragma unroll
            for (int L = 4; L < 8; ++L) lo = lo * 128 + __float2int_rn(acc[L][cc + o]);
            // |hi|, |lo| < 2^51: exact conversion through the 1.5 * 2^52 offset
            const double hd = __longlong_as_double(hi + 0x4338000000000000LL) - 6755399441055744.0;
            const double ld = __longlong_as_double(lo + 0x4338000000000000LL) - 6755399441055744.0;
            const double h = fma(hd, 0x1p28, ld);
            res[o] = scale_pow2(h, Erow + F[jg + o] - 2056 - 49);
          }
          const long long oidx = (long long)c * n + ie;
          double2 out = make_double2(res[0], res[1]);
          if (beta_one) {
            const double2 in = IN[oidx];
            out.x += in.x;
            out.y += in.y;
          }
          OUT[oidx] = out;
        }
      }
    }
    fence_before();
    __syncthreads();     // tensor memory read before the next tile's first MMA
  }

  if (abort) {
    if (t == 0) atomicExch(err, 1);
    if (committed > 0) {   // let the MMAs in flight finish before freeing their memory
      const long long gl = committed - 1;
      mbar_wait(&bars[gl & 1], (uint32_t)((gl >> 1) & 1));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "n"(TMEM_COLS));
}

// ----------------------------------------------------------------- host side

size_t ts_update_tc_scratch_bytes(int kv, int ncol) {
  const int nch = (2 * kv + 15) / 16;
  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  return aligned_bytes((size_t)ntile * TC_DIGITS * nch * B_BLOCK) +
         aligned_bytes((size_t)ntile * TC_NCOLS * sizeof(int));
}

bool ts_update_tc_supported(int kv, int ncol) { return kv >= 1 && kv <= TC_MAXKV && ncol >= 1; }

cudaError_t launch_ts_update_tc(const double2 *V, int kv, const double2 *Y, int ldy, int ncol,
                                const double2 *IN, double2 *OUT, int beta_one, double sign,
                                long long n, void *scratch, int *err, cudaStream_t s) {
  ProfLaunch prof_(PC_TS, s);
  if (!ts_update_tc_supported(kv, ncol) || n < 1 || scratch == nullptr || err == nullptr)
    return cudaErrorInvalidValue;
  const int nch = (2 * kv + 15) / 16;
  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  unsigned char *Bd = static_cast<unsigned char *>(scratch);
  int *F = reinterpret_cast<int *>(Bd + aligned_bytes((size_t)ntile * TC_DIGITS * nch * B_BLOCK));
  const int cols = ntile * TC_NCOLS;
  tc_prep_y_kernel<<<(cols + 7) / 8, 256, 0, s>>>(Y, ldy, kv, ncol, sign, nch, Bd, F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)TC_DIGITS * nch * B_BLOCK + 2 * A_BUF + 2 * TC_ROWS * sizeof(int) + 64;
  static thread_local int attr_device = -1;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(tc_tsgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)TC_DIGITS * TC_MAXCH * B_BLOCK + 2 * A_BUF +
                                   2 * TC_ROWS * sizeof(int) + 64));
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = ((n + TC_ROWS - 1) / TC_ROWS) * ntile;
  const int grid = (int)(tiles < sms ? tiles : sms);
  tc_tsgemm_kernel<<<grid, TC_THREADS, smem, s>>>(V, kv, n, nch, Bd, F, ncol, IN, OUT, beta_one, err);
  return cudaGetLastError();
}

}  // namespace wd
