// OUT[c] = (beta_one ? IN[c] : 0) + sign * sum_r V[r] * Y[r][c] for complex128
// vectors of length n, on the tensor cores (tcgen05, BF16 inputs, FP32
// accumulation in tensor memory), to FP64 accuracy.
//
// This is the contraction of GMRES-DR's restart, V_{k+1} = V_{m+1} P_{k+1}
// (Sec. 1), and of the projection's updates x0 += V y, r0 -= (A V) y
// (Sec. 2): M = n rows, K = 2 kv real values per row, N = 2 ncol real
// columns.  It is exact-split emulation (Ozaki's scheme): every FP64 value
// of a row of V (or a column of Y) is written as a 55-bit fixed-point
// number relative to the largest exponent of its row (column) and split
// into eight balanced 7-bit digits, |d| <= 64, each exact in BF16.  Digit pairs
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
// tile of OUT at a time (persistent grid, one CTA per SM), with three kinds
// of warps: eight producers turn the tile's V values into digit planes,
// one warp issues the MMAs, four read the accumulators and write OUT, so
// that the epilogue of one tile overlaps the digits of the next.  The BF16
// digit planes live in shared memory in the tensor cores' K-major layout
// without swizzle: 8x8 core matrices of 16-byte rows, the K-adjacent core
// matrix 128 bytes on, the next 8-row group 256 bytes on.  Per K-chunk of
// 16 the A digits (8 planes x 128 rows) are double-buffered; all digit
// planes of Y for the column tile stay resident.  Tensor memory: 8 levels x
// 48 columns.  Every wait on an mbarrier gives up after one second and
// sets the error flag; the kernel then lets its MMAs drain and frees its
// tensor memory.
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
constexpr int TC_PRODUCERS = 8;              // warps forming digit planes
constexpr int TC_EPILOGUE = 8;               // warps reading the accumulators
constexpr int TC_MMA_WARP = TC_PRODUCERS + TC_EPILOGUE;
constexpr int TC_THREADS = 32 * (TC_MMA_WARP + 1);
constexpr int A_PLANE = TC_ROWS * 16 * 2;     // bytes of one digit plane, one chunk
constexpr int A_BUF = TC_DIGITS * A_PLANE;    // 32 KB
constexpr int B_BLOCK = TC_NCOLS * 16 * 2;    // one digit plane of Y, one chunk: 1536 B
constexpr int TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 1000000000ull;   // give up a wait after 1 s

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

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major,
// M = 128, N (a multiple of 16 up to 256) given
__device__ __forceinline__ uint32_t idesc_n(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(TC_ROWS >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// true once the phase with this parity has completed; false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (int i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity));
    if (ok) return true;
    if (i == 0) t0 = global_ns();
    else if ((i & 63) == 0 && global_ns() - t0 > WAIT_NS) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}"
               ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)));
}

// eight consecutive 32-bit columns of this warp's 32 lanes (no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// The eight balanced digits of X = sum_s d_s 2^(7 (7 - s)), |X| < 2^55:
// with BIAS = 128 2^49 + 64 sum_{s=1..7} 2^(7 (7 - s)), U = X + BIAS lies in
// [0, 2^57); its top 8-bit field is d_0 + 128 (|d_0| <= 64) and its seven
// 7-bit fields below are d_s + 64 (-64 <= d_s <= 63).  f[s] receives the
// FP32 bit pattern of d_s, whose high half is d_s in BF16 (exact).
constexpr long long DIGIT_BIAS = (1LL << 56) + 64LL * 4432676798593LL;  // 4432676798593 = (2^49 - 1) / 127

__device__ __forceinline__ uint32_t field_f32(int value) {
  // float(value) exactly for |value| <= 128 (at most 8 significant bits)
  return __float_as_uint(__int_as_float(0x4B400000 + value) - 12582912.0f);
}

__device__ __forceinline__ void digits_f32(long long X, uint32_t *f) {
  const unsigned long long U = (unsigned long long)(X + DIGIT_BIAS);
  const uint32_t hi = (uint32_t)(U >> 32), lo = (uint32_t)U;
  f[0] = field_f32((int)((hi >> 17) & 255) - 128);
  f[1] = field_f32((int)((hi >> 10) & 127) - 64);
  f[2] = field_f32((int)((hi >> 3) & 127) - 64);
  f[3] = field_f32((int)(__funnelshift_r(lo, hi, 28) & 127) - 64);
  f[4] = field_f32((int)((lo >> 21) & 127) - 64);
  f[5] = field_f32((int)((lo >> 14) & 127) - 64);
  f[6] = field_f32((int)((lo >> 7) & 127) - 64);
  f[7] = field_f32((int)(lo & 127) - 64);
}

// two BF16 values (the high halves of two FP32 patterns), a in the low half
__device__ __forceinline__ uint32_t pack_bf16(uint32_t a, uint32_t b) {
  return __byte_perm(a, b, 0x7632);
}

}  // namespace


// ----------------------------------------------------------------- Y digits

// Real column j = 2 c' + o of column tile t (complex column c = 24 t + c',
// o = 0 real part of OUT, 1 imaginary part) against K index k = 2 r + p
// (p = 0 real part of V, 1 imaginary part):
//   o = 0: p = 0 -> Re Y[r][c],  p = 1 -> -Im Y[r][c]
//   o = 1: p = 0 -> Im Y[r][c],  p = 1 ->  Re Y[r][c]
// times `sign`.  One warp per real column: its exponent field (maximum over
// the column), then the digit planes Bd[t][q][s] (q = K-chunk), each in the
// K-major core-matrix layout, and F[j] = the exponent field.  For a fixed
// chunk the eight planes follow each other, so that planes b0 .. b1 - 1 read
// as one operand of 48 (b1 - b0) rows.
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
    digits_f32(fixed_point(y_value(Y, ldy, kv, ncol, sign, j, k), E), d);
    const int q = k >> 4, kk = k & 15;
#pragma unroll
    for (int s = 0; s < TC_DIGITS; ++s) {
      unsigned char *blk = Bd + ((long long)(t * nch + q) * TC_DIGITS + s) * B_BLOCK;
      *reinterpret_cast<uint16_t *>(blk + core_off(jj, kk)) = (uint16_t)(d[s] >> 16);
    }
  }
}


// ----------------------------------------------------------------- row exponents

// Erow[i] = the largest exponent field of row i of V (its 2 kv real values).
__global__ void __launch_bounds__(256)
tc_row_exponent_kernel(const double2 *__restrict__ V, int kv, long long n, int *__restrict__ Erow) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int E = 0;
#pragma unroll 8
    for (int r = 0; r < kv; ++r) {
      const double2 v = V[(long long)r * n + i];
      E = max(E, max(exp_field(v.x), exp_field(v.y)));
    }
    Erow[i] = E;
  }
}

// ----------------------------------------------------------------- main kernel

__device__ __forceinline__ double scale_pow2(double h, int e) {
  // h * 2^e (h != 0) through the exponent field when the result stays normal
  const long long b = __double_as_longlong(h);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be + e >= 1 && be + e <= 2046 && be != 0) return __longlong_as_double(b + ((long long)e << 52));
  return ldexp(h, e);
}

// shared memory after the digit planes: row exponents and barriers
struct TcSmemTail {
  uint64_t full[2];                // A buffer b holds digits (producer warps arrive)
  uint64_t empty[2];               // MMAs reading A buffer b completed (commit)
  uint64_t tfull;                  // all MMAs of a tile completed (commit)
  uint64_t tempty;                 // epilogue warps finished reading the accumulators
  uint64_t drain;                  // every MMA issued so far completed (teardown)
  uint32_t tbase;                  // tensor memory base address
};

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_tsgemm_kernel(const double2 *__restrict__ V, int kv, long long n, int nch,
                 const unsigned char *__restrict__ Bd, const int *__restrict__ F, int ncol,
                 const int *__restrict__ Erow, const double2 *IN, double2 *OUT, int beta_one,
                 int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sB = smem;                                  // 8 x nch x 1536
  unsigned char *sA = smem + TC_DIGITS * nch * B_BLOCK;      // 2 x 32 KB
  TcSmemTail &S = *reinterpret_cast<TcSmemTail *>(sA + 2 * A_BUF);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.full[b], TC_PRODUCERS);
      mbar_init(&S.empty[b], 1);
    }
    mbar_init(&S.tfull, 1);
    mbar_init(&S.tempty, TC_EPILOGUE);
    mbar_init(&S.drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&S.tbase)), "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tm = S.tbase;

  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  const long long nrt = (n + TC_ROWS - 1) / TC_ROWS;
  const long long ntiles = nrt * ntile;
  bool failed = false;

  if (warp < TC_PRODUCERS) {
    // ---------------------------------------------------------- producers
    const int row = t & (TC_ROWS - 1), half = t >> 7;
    int loaded = -1;
    long long g = 0;                               // K-chunks produced (all tiles)
    int T = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++T) {
      const int ct = (int)(tile / nrt);
      const long long i = (tile % nrt) * TC_ROWS + row;
      const bool valid = i < n;
      if (ct != loaded) {          // new column tile: the MMAs reading the old Y planes are done
        if (T > 0 && !mbar_wait(&S.tfull, (uint32_t)((T - 1) & 1))) { failed = true; break; }
        const uint4 *src = reinterpret_cast<const uint4 *>(Bd + (long long)ct * TC_DIGITS * nch * B_BLOCK);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        for (int e = t; e < TC_DIGITS * nch * B_BLOCK / 16; e += 32 * TC_PRODUCERS) dst[e] = src[e];
        loaded = ct;
      }
      const int E = valid ? Erow[i] : 0;        // row exponent field (pre-kernel)

      // digit planes, one K-chunk at a time: rows r = 8q + 4 half + u of V;
      // the values of the next two chunks are in flight meanwhile
      double2 v0[4], v1[4], v2[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r0 = 4 * half + u, r1 = 8 + 4 * half + u;
        v0[u] = (valid && r0 < kv) ? V[(long long)r0 * n + i] : make_double2(0.0, 0.0);
        v1[u] = (valid && 1 < nch && r1 < kv) ? V[(long long)r1 * n + i] : make_double2(0.0, 0.0);
      }
      for (int q = 0; q < nch; ++q, ++g) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 8 * (q + 2) + 4 * half + u;
          v2[u] = (valid && q + 2 < nch && r < kv) ? V[(long long)r * n + i]
                                                   : make_double2(0.0, 0.0);
        }
        const int b = (int)(g & 1);
        if (g >= 2 && !mbar_wait(&S.empty[b], (uint32_t)(((g - 2) >> 1) & 1))) {
          failed = true;
          break;
        }
        uint32_t f[8][TC_DIGITS];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          digits_f32(fixed_point(v0[u].x, E), f[2 * u]);
          digits_f32(fixed_point(v0[u].y, E), f[2 * u + 1]);
        }
        unsigned char *buf = sA + b * A_BUF;
#pragma unroll
        for (int sl = 0; sl < TC_DIGITS; ++sl) {
          uint4 w;
          w.x = pack_bf16(f[0][sl], f[1][sl]);
          w.y = pack_bf16(f[2][sl], f[3][sl]);
          w.z = pack_bf16(f[4][sl], f[5][sl]);
          w.w = pack_bf16(f[6][sl], f[7][sl]);
          *reinterpret_cast<uint4 *>(buf + sl * A_PLANE + core_off(row, 8 * half)) = w;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.full[b]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v0[u] = v1[u];
          v1[u] = v2[u];
        }
      }
      if (failed) break;
    }
  } else if (warp == TC_MMA_WARP) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      long long g = 0;
      int T = 0;
      const uint32_t bBase = smem_u32(sB);
      for (long long tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++T) {
        for (int q = 0; q < nch; ++q, ++g) {
          const int b = (int)(g & 1);
          if (!mbar_wait(&S.full[b], (uint32_t)((g >> 1) & 1))) { failed = true; break; }
          if (q == 0 && T > 0 && !mbar_wait(&S.tempty, (uint32_t)((T - 1) & 1))) { failed = true; break; }
          fence_after();
          const uint32_t aBase = smem_u32(sA + b * A_BUF);
          // A plane a against Y planes b = 0 .. 7 - a stacked along N writes
          // the accumulators of levels a .. 7 (adjacent in tensor memory) in
          // one MMA of N = 48 (8 - a), split where N would exceed 240
          const uint32_t qBase = bBase + (uint32_t)(q * TC_DIGITS * B_BLOCK);
#pragma unroll 1
          for (int a = 0; a < TC_DIGITS; ++a) {
            const uint64_t da = smem_desc(aBase + a * A_PLANE);
            for (int b0 = 0; a + b0 < TC_LEVELS;) {
              const int nb = min(TC_LEVELS - a - b0, 5);
              const uint64_t db = smem_desc(qBase + (uint32_t)(b0 * B_BLOCK));
              mma_bf16(tm + (uint32_t)((a + b0) * TC_NCOLS), da, db, idesc_n(TC_NCOLS * nb),
                       (q > 0 || a > 0) ? 1u : 0u);
              b0 += nb;
            }
          }
          mma_commit(&S.empty[b]);
        }
        if (!failed) mma_commit(&S.tfull);
      }
      // teardown: every MMA issued has completed before the memory is freed
      mma_commit(&S.drain);
      if (!mbar_wait(&S.drain, 0)) failed = true;
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    // warp e = warp - 8 reads lanes 32 (warp % 4) .. + 31 (its rows) and the
    // real columns 24 (e / 4) .. + 23 of the tile, 8 at a time
    const int quarter = warp & 3;
    const int chalf = (warp - TC_PRODUCERS) >> 2;
    const int er = 32 * quarter + lane;
    const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
    int T = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++T) {
      const int ct = (int)(tile / nrt);
      const long long ie = (tile % nrt) * TC_ROWS + er;
      const int Er = ie < n ? Erow[ie] : 0;
      if (!mbar_wait(&S.tfull, (uint32_t)(T & 1))) { failed = true; break; }
      fence_after();
#pragma unroll 1
      for (int c0 = 24 * chalf; c0 < 24 * chalf + 24; c0 += 8) {
        uint32_t acc[TC_LEVELS][8];
#pragma unroll
        for (int L = 0; L < TC_LEVELS; ++L)
          tmem_ld8(tm + lane_addr + (uint32_t)(L * TC_NCOLS + c0), acc[L]);
        tmem_wait_ld();
        if (ie >= n) continue;
#pragma unroll
        for (int cc = 0; cc < 8; cc += 2) {
          const int jg = ct * TC_NCOLS + c0 + cc;   // real column of the real part
          const int c = jg >> 1;
          if (c >= ncol) continue;
          double res[2];
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            // the level sums are exact integers below 2^24: combine levels 0-3
            // and 4-7 in 64-bit integers (each below 2^45), leaving one FP64
            // rounding: sum_L A_L 2^(-7L) = (hi 2^28 + lo) 2^-49
            long long hi = 0, lo = 0;
#pragma unroll
            for (int L = 0; L < 4; ++L) hi = hi * 128 + __float2int_rn(__uint_as_float(acc[L][cc + o]));
#pragma unroll
            for (int L = 4; L < 8; ++L) lo = lo * 128 + __float2int_rn(__uint_as_float(acc[L][cc + o]));
            if ((hi | lo) == 0) {
              res[o] = 0.0;
              continue;
            }
            // |hi|, |lo| < 2^51: exact conversion through the 1.5 * 2^52 offset
            const double hd = __longlong_as_double(hi + 0x4338000000000000LL) - 6755399441055744.0;
            const double ld = __longlong_as_double(lo + 0x4338000000000000LL) - 6755399441055744.0;
            res[o] = scale_pow2(fma(hd, 0x1p28, ld), Er + F[jg + o] - 2105);
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
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.tempty);
    }
  }

  if (failed) atomicExch(err, 1);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == TC_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "n"(TMEM_COLS));
}

// ----------------------------------------------------------------- host side

size_t ts_update_tc_scratch_bytes(int kv, int ncol, long long n) {
  const int nch = (2 * kv + 15) / 16;
  const int ntile = (ncol + TC_CCOLS - 1) / TC_CCOLS;
  return aligned_bytes((size_t)ntile * TC_DIGITS * nch * B_BLOCK) +
         aligned_bytes((size_t)ntile * TC_NCOLS * sizeof(int)) + aligned_bytes((size_t)n * sizeof(int));
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
  int *Erow = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(F) +
                                      aligned_bytes((size_t)ntile * TC_NCOLS * sizeof(int)));
  const int cols = ntile * TC_NCOLS;
  tc_prep_y_kernel<<<(cols + 7) / 8, 256, 0, s>>>(Y, ldy, kv, ncol, sign, nch, Bd, F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    tc_row_exponent_kernel<<<(unsigned)blocks, 256, 0, s>>>(V, kv, n, Erow);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)TC_DIGITS * nch * B_BLOCK + 2 * A_BUF + sizeof(TcSmemTail);
  static thread_local int attr_device = -1;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_device != dev) {
    e = cudaFuncSetAttribute(tc_tsgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)TC_DIGITS * TC_MAXCH * B_BLOCK + 2 * A_BUF +
                                   sizeof(TcSmemTail)));
    if (e != cudaSuccess) return e;
    attr_device = dev;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = ((n + TC_ROWS - 1) / TC_ROWS) * ntile;
  const int grid = (int)(tiles < sms ? tiles : sms);
  tc_tsgemm_kernel<<<grid, TC_THREADS, smem, s>>>(V, kv, n, nch, Bd, F, ncol, Erow, IN, OUT,
                                                   beta_one, err);
  return cudaGetLastError();
}

}  // namespace wd
