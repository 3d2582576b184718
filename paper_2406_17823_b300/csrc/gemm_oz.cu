// FP64 products on the BF16 tensor cores by the Ozaki splitting scheme
// (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012): K is taken
// in chunks of 64; in each chunk every row of op(A) and every column of
// op(B) is written as a fixed-point number with a power-of-two scale and
// cut into eight signed 7-bit slices, the products of slice pairs (p, q)
// with p + q <= 7 are exact on the tensor cores and summed exactly, and the
// exact sum is rounded to FP64 once; the chunks' results add up in FP64.
// This is the mixed form's contraction kernel: FP64-level accuracy (the
// dropped pairs and the slicing truncation stay below about
// K 2^-53 2^(eA + eB), eA, eB the operands' scale exponents) at a
// tensor-core rate, on a GPU whose FP64 pipe retires about two FMAs per
// clock per SM.
//
// One CTA of 512 threads per 128 x BN output tile (BN = 16, 32 or 64) of one
// batch entry (or one K slice of it); per K chunk:
//  * Slicing.  Every thread loads its share of the two FP64 operand tiles
//    in batches of four pairs (any strides, transposes and batch offsets;
//    a batch's loads issued before use), the rows' largest magnitudes give
//    the scales, and
//    the slices go as BF16 integers into shared memory in the layout the
//    128-byte-swizzled K-major UMMA descriptor expects (rows of 64 BF16,
//    16-byte chunks XOR-ed with the row index mod 8).  Integer arithmetic
//    on the FP64 bit patterns only.
//  * Products.  One thread issues tcgen05.mma kind::f16 (BF16 x BF16, FP32
//    accumulation, M = 128, K = 16) for the 36 slice pairs, pairs of equal
//    p + q = d into accumulator d of eight in tensor memory (8 BN columns):
//    A_p against the consecutive B slices q = 0 .. 7 - p as one MMA of
//    N = (8 - p) BN (two when that exceeds 256) whose output starts at
//    accumulator p.  A diagonal sums at most 8 x 64 products of magnitude
//    below 2^14, so every partial sum is an integer below 2^23 and the FP32
//    accumulation is exact.
//  * Epilogue.  The sixteen warps read the accumulators (warps w, w + 4,
//    w + 8, w + 12 share TMEM lanes 32 (w mod 4) .. and split the 8-column
//    groups), combine the exact integers as T = sum_d D_d 2^(7 (7 - d)) in
//    64-bit integer arithmetic and round T 2^(eA + eB - 63) to FP64 by
//    integer operations (round to nearest even).  A one-chunk item writes
//    alpha x + beta C straight from the accumulator rows; with several
//    chunks the results are staged in shared memory and C is updated in a
//    coalesced pass: the first chunk stores, later ones add theirs in
//    order, the last applies alpha (beta is not taken there: an unbatched
//    product with beta != 0 and several chunks is split over K slices whose
//    partial products the slice sum combines, in order, with alpha and
//    beta).  The wait for each
// chunk's MMAs is bounded by one second of global time; a wait that gives
// up sets QTT_DEVERR_TIMEOUT, skips the output, frees the tensor memory and
// returns.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kOzThreads = 512;
constexpr int kOzM = 128;          // MMA M (rows of the A-operand tile)
constexpr int kOzSlices = 8;       // slices per operand
constexpr int kOzChunk = 64;       // K elements per chunk: one 128-byte swizzled row
constexpr int kOzTileA = kOzM * 128;  // bytes of one A slice tile
constexpr int kOzBad = 1 << 20;    // scale exponent of a row holding Inf or NaN

// Instruction descriptor of kind::f16 with BF16 operands: D FP32 (bit 4),
// A and B BF16 (1 at bits 7 and 10), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// One operand of the kernel: element (r, k) of batch entry (z1, z2) at
// p[z1 s1 + z2 s2 + r sr + k sk], r < rows, k < K.
struct OzOperand {
  const double* p;
  long long s1, s2, sr, sk;
  int rows;
};

struct OzParams {
  OzOperand a, b;      // a: the 128-row side, b: the BN-row side
  int K, nch, BN;
  int kslice;          // > 0: item z is a K slice [z kslice, (z + 1) kslice)
  int nz;              // batch entries (or K slices)
  int nb2;
  int swap;            // 0: C(r_a, r_b); 1: C(r_b, r_a)
  double* C;
  long long ldc, sC1, sC2;
  double alpha, beta;
  const int* skip;
  int* err;
};

// |x| as the bit pattern of a non-negative double (monotonic in |x|; NaN
// above +Inf)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Scale exponent e of a row from its largest |x| (bits): |x| < 2^e for every
// element; kOzBad for a row holding Inf or NaN.
__device__ __forceinline__ int row_scale(unsigned long long mx) {
  if (mx >= 0x7FF0000000000000ull) return kOzBad;
  const int ex = (int)(mx >> 52);
  return (ex > 1 ? ex : 1) - 1022;
}

// floor(|x| 2^(56 - e)) (< 2^56) and the sign of x
__device__ __forceinline__ unsigned long long fixed56(double x, int e, unsigned& sgn) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  sgn = (unsigned)(b >> 63);
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long mant = ex ? (frac | 0x10000000000000ull) : frac;
  const int sh = (ex ? ex : 1) - 1019 - e;
  if (sh >= 0) return mant << sh;  // sh <= 3 when |x| < 2^e
  return sh > -64 ? (mant >> -sh) : 0ull;
}

// Byte offset of element (r, k), k < 64, in a K-major tile of 128-byte rows
// with the 128-byte swizzle (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7))) << 4) +
                    ((k & 7) << 1));
}

// FP64 value of T 2^scale, T = H 2^28 + L (|H|, |L| < 2^47), rounded once to
// nearest even, in 64-bit integer operations: T is first brought to sign
// and magnitude A 2^28 + R with 0 <= R < 2^28; below 2^53 it is exact,
// otherwise its top 53 bits are A's bits and R's upper bits, rounded by R's
// remaining bits (ldexp only for a subnormal or overflowing result).
__device__ __forceinline__ double assemble(long long H, long long L, int scale) {
  const long long Hn = H + (L >> 28);  // arithmetic shift: floor(L / 2^28)
  const unsigned long long R = (unsigned long long)L & 0xFFFFFFFull;
  unsigned long long A, Rn, sgn;
  if (Hn < 0) {  // -T = (-Hn - 1) 2^28 + (2^28 - R)  (or -Hn 2^28 when R = 0)
    sgn = 1ull;
    A = R ? (unsigned long long)(-Hn - 1) : (unsigned long long)(-Hn);
    Rn = R ? 0x10000000ull - R : 0ull;
  } else {
    sgn = 0ull;
    A = (unsigned long long)Hn;
    Rn = R;
  }
  if ((A | Rn) == 0ull) return 0.0;
  unsigned long long m;
  int sh;
  if (A < (1ull << 25)) {
    const unsigned long long U = (A << 28) | Rn;  // < 2^53: exact
    const int nb = 64 - __clzll((long long)U);
    m = U << (53 - nb);
    sh = nb - 53;
  } else {
    sh = (64 - __clzll((long long)A)) - 25;  // bits of A + 28 - 53, 1 .. 22
    m = (A << (28 - sh)) | (Rn >> sh);
    const unsigned long long rem = Rn & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      m++;
      if (m >> 53) {
        m >>= 1;
        sh++;
      }
    }
  }
  // value = m 2^(sh + scale), 2^52 <= m < 2^53
  const int E = 52 + sh + scale;
  if (E < -1022 || E > 1023) {
    const double v = ldexp((double)m, sh + scale);
    return sgn ? -v : v;
  }
  return __longlong_as_double(
      (long long)((sgn << 63) | ((unsigned long long)(E + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// Digits of a pair (x0, x1) of one row (scale exponent e): eight words, word
// p holding the p-th 7-bit digits of x0 (low half) and x1 (high half) as
// signed BF16 integers.  A digit v < 128 with sign s is exact in FP32 as
// (-1)^s (2^23 + v) - (-1)^s 2^23: the bit pattern s | 2^23 exponent | v
// is one logic operation on the shifted field, and the BF16 is the upper
// half of that FP32.
__device__ __forceinline__ void pair_digits(double x0, double x1, int e, uint32_t (&w)[kOzSlices]) {
  unsigned s0, s1;
  const unsigned long long f0 = fixed56(x0, e, s0), f1 = fixed56(x1, e, s1);
  const uint32_t h0 = (uint32_t)(f0 >> 28), l0 = (uint32_t)f0 & 0xFFFFFFFu;
  const uint32_t h1 = (uint32_t)(f1 >> 28), l1 = (uint32_t)f1 & 0xFFFFFFFu;
  const uint32_t m0 = 0x4B000000u | (s0 << 31), m1 = 0x4B000000u | (s1 << 31);
  const float c0 = s0 ? 8388608.0f : -8388608.0f, c1 = s1 ? 8388608.0f : -8388608.0f;
#pragma unroll
  for (int p = 0; p < kOzSlices; p++) {
    const int sh = 7 * (3 - (p & 3));
    const uint32_t b0 = __float_as_uint(__uint_as_float((((p < 4 ? h0 : l0) >> sh) & 127u) | m0) + c0);
    const uint32_t b1 = __float_as_uint(__uint_as_float((((p < 4 ? h1 : l1) >> sh) & 127u) | m1) + c1);
    w[p] = __byte_perm(b0, b1, 0x7632);  // upper halves: the BF16 values
  }
}

// Where thread t's pair i of a tile of R rows lies (R / 16 pairs per thread,
// kOzThreads = 512).  With k contiguous in memory warp w takes rows w,
// w + 16, ... and lane l the pair (2 l, 2 l + 1).  Otherwise (rows contiguous)
// each warp step covers a block of 8 consecutive rows x 4 consecutive pairs
// (lane l: row l mod 8, pair l / 8): loads are 64-byte row runs and the
// swizzled shared-memory stores of a warp fall in 32 different banks.  Block
// W = 16 i + w takes rows 8 (W mod R/8) .. and pairs 4 (W div R/8) ..; for
// R = 128 a thread keeps one row and its warp holds all of that row's pairs.
template <int R>
__device__ __forceinline__ void pair_at(bool kc, int i, int& r, int& k) {
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  if (kc) {
    r = w + 16 * i;
    k = 2 * l;
  } else {
    constexpr int kRB = R / 8;
    const int W = 16 * i + w;
    r = 8 * (W % kRB) + (l & 7);
    k = 2 * (4 * (W / kRB) + (l >> 3));
  }
}

template <int R>
__device__ __forceinline__ void load_pair(const OzOperand& o, const double* base, int r0,
                                          int klen, int r, int k, double& x0, double& x1) {
  const bool live = r0 + r < o.rows;
  const double* row = base + (long long)(r0 + r) * o.sr;
  if (live && o.sk == 1 && k + 1 < klen && (((uintptr_t)(row + k)) & 15) == 0) {
    const double2 v = *(const double2*)(row + k);  // both elements in one 16-byte load
    x0 = v.x;
    x1 = v.y;
    return;
  }
  x0 = (live && k < klen) ? row[(long long)k * o.sk] : 0.0;
  x1 = (live && k + 1 < klen) ? row[(long long)(k + 1) * o.sk] : 0.0;
}

// One K chunk of a tile of R rows (base already at the chunk's first k):
// the rows' largest magnitudes into mx[] and the eight slices into dst
// (slice p at dst + p R 128 bytes).  Every load of the thread's R / 16 pairs
// is issued before the first use.  With k contiguous a row lives in one warp
// and its maximum is a warp reduction; otherwise over the 4 lanes of the row
// in each warp and, when the row spans several warps (R < 128), shared
// memory.
template <int R>
__device__ void slice_tile(const OzOperand& o, const double* base, int r0, int klen,
                           unsigned long long* mx, uint8_t* dst) {
  constexpr int kPairs = R / 16;
  constexpr uint32_t slice_bytes = (uint32_t)R * 128;
  const bool kc = o.sk == 1;
  const int lane = threadIdx.x & 31;
  double x[2 * kPairs];
#pragma unroll
  for (int i = 0; i < kPairs; i++) {
    int r, k;
    pair_at<R>(kc, i, r, k);
    load_pair<R>(o, base, r0, klen, r, k, x[2 * i], x[2 * i + 1]);
  }
  int e[kPairs];
  if (kc) {
#pragma unroll
    for (int i = 0; i < kPairs; i++) {
      unsigned long long m = max(abs_bits(x[2 * i]), abs_bits(x[2 * i + 1]));
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, s));
      int r, k;
      pair_at<R>(true, i, r, k);
      if (lane == 0) mx[r] = m;
      e[i] = row_scale(m);
    }
  } else {
    // the pairs i of one thread share a row when R = 128; in general pair i
    // lies in row block (16 i + w) mod R/8
    unsigned long long m[kPairs];
#pragma unroll
    for (int i = 0; i < kPairs; i++) {
      m[i] = max(abs_bits(x[2 * i]), abs_bits(x[2 * i + 1]));
      m[i] = max(m[i], __shfl_xor_sync(0xffffffffu, m[i], 8));
      m[i] = max(m[i], __shfl_xor_sync(0xffffffffu, m[i], 16));
    }
    if (R == 128) {
      unsigned long long mm = 0;
#pragma unroll
      for (int i = 0; i < kPairs; i++) mm = max(mm, m[i]);
      int r, k;
      pair_at<R>(false, 0, r, k);
      if (lane < 8) mx[r] = mm;
#pragma unroll
      for (int i = 0; i < kPairs; i++) e[i] = row_scale(mm);
    } else {
#pragma unroll
      for (int i = 0; i < kPairs; i++) {
        int r, k;
        pair_at<R>(false, i, r, k);
        if (lane < 8) atomicMax(&mx[r], m[i]);
      }
    }
  }
  if (!kc && R != 128) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPairs; i++) {
      int r, k;
      pair_at<R>(false, i, r, k);
      e[i] = row_scale(mx[r]);
    }
  }
#pragma unroll
  for (int i = 0; i < kPairs; i++) {
    int r, k;
    pair_at<R>(kc, i, r, k);
    uint32_t w[kOzSlices];
    if (e[i] == kOzBad) x[2 * i] = x[2 * i + 1] = 0.0;  // the row's output is NaN
    pair_digits(x[2 * i], x[2 * i + 1], e[i], w);
    const uint32_t off = sw128_off(r, k);
#pragma unroll
    for (int p = 0; p < kOzSlices; p++) *(uint32_t*)(dst + p * slice_bytes + off) = w[p];
  }
}

// The eight accumulators' columns c0 .. c0 + 7 of this warp's 32 TMEM lanes
// (accumulator d at column offset d * BN), one wait for all eight loads.
template <int BN>
__device__ __forceinline__ void tmem_ld_diagonals(uint32_t taddr, float (&D)[kOzSlices][8]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%65];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%66];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%67];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%68];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40, %41, %42, %43, %44, %45, %46, %47}, [%69];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48, %49, %50, %51, %52, %53, %54, %55}, [%70];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%56, %57, %58, %59, %60, %61, %62, %63}, [%71];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]),
        "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
        "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]),
        "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]),
        "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr), "r"(taddr + BN), "r"(taddr + 2 * BN), "r"(taddr + 3 * BN),
        "r"(taddr + 4 * BN), "r"(taddr + 5 * BN), "r"(taddr + 6 * BN), "r"(taddr + 7 * BN)
      : "memory");
#pragma unroll
  for (int d = 0; d < kOzSlices; d++)
#pragma unroll
    for (int j = 0; j < 8; j++) D[d][j] = __uint_as_float(r[8 * d + j]);
}

// D (an integer-valued FP32 accumulator) as an integer: |D| < 2^22 by the
// FP32 addition of 1.5 2^23 (exact, the sum's low mantissa bits are D),
// larger ones by conversion.
__device__ __forceinline__ int int_small(float D) {
  return __float_as_int(D + 12582912.0f) - 0x4B400000;
}

template <int BN>
__global__ void __launch_bounds__(kOzThreads, 1) k_gemm_oz(OzParams g) {
  static_assert(BN == 16 || BN == 32 || BN == 64, "output tile width");
  if (g.skip && *g.skip) return;  // uniform over the grid
  extern __shared__ uint8_t oz_smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sa = base;                          // 8 slices x 128 rows x 128 B
  uint8_t* sb = base + kOzSlices * kOzTileA;   // 8 slices x BN rows x 128 B
  // a chunk's rounded products, staged for coalesced output once the MMAs
  // have read the A slices (128 rows of BN + 1 doubles)
  double* stage = (double*)sa;
  constexpr int kST = BN + 1;
  __shared__ unsigned long long mxa[kOzM], mxb[BN];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t ncols = 8u * (uint32_t)BN;  // 128, 256 or 512
  const uint32_t mbar = smem_u32(&bar);

  if (tid == 0) {
    s_ok = 1;
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // epilogue geometry: warp w reads TMEM lanes 32 (w & 3) .. (tile rows) and
  // the 8-column groups w >> 2, (w >> 2) + 4, ...
  const int quarter = warp & 3, part = warp >> 2;
  const int r = quarter * 32 + lane;
  const bool plain = g.alpha == 1.0 && g.beta == 0.0;  // C = op(A) op(B)
  const int tiles_b = (g.b.rows + BN - 1) / BN, tiles_a = (g.a.rows + kOzM - 1) / kOzM;
  const int items = tiles_b * tiles_a * g.nz;
  uint32_t phase = 0;  // completed waits on the MMA barrier
  // persistent: each CTA takes a contiguous range of work items (B tile
  // fastest, then A tile, then batch entry or K slice), so that consecutive
  // one-chunk items of one A tile reuse its slices in shared memory
  const int per = (items + (int)gridDim.x - 1) / (int)gridDim.x;
  const int item_end = min(items, ((int)blockIdx.x + 1) * per);
  int held = -1;  // the A tile (by + tiles_a z) whose one-chunk slices are in shared memory
  for (int item = blockIdx.x * per; item < item_end && s_ok; item++) {
    const int bx = item % tiles_b, rest = item / tiles_b;
    const int by = rest % tiles_a, z = rest / tiles_a;
    const int z1 = z / g.nb2, z2 = z % g.nb2;
    const int ra0 = by * kOzM, rb0 = bx * BN;
    // this item's K extent (a K slice: the batch strides step along K)
    const int Kz = g.kslice > 0 ? min(g.kslice, g.K - z * g.kslice) : g.K;
    const int nch = (Kz + kOzChunk - 1) / kOzChunk;
    const double* pa = g.a.p + z1 * g.a.s1 + z2 * g.a.s2;
    const double* pb = g.b.p + z1 * g.b.s1 + z2 * g.b.s2;
    double* cz = g.C + z1 * g.sC1 + z2 * g.sC2;
    // one-chunk items write C directly and leave the A slices intact
    const bool keep_a = nch == 1 && held == rest;
    held = nch == 1 ? rest : -1;
    for (int c = 0; c < nch; c++) {
      const int k0 = c * kOzChunk, klen = min(kOzChunk, Kz - k0);
      if (!keep_a)
        for (int i = tid; i < kOzM; i += kOzThreads) mxa[i] = 0ull;
      if (tid < BN) mxb[tid] = 0ull;
      __syncthreads();  // zeroed row maxima; the previous chunk's output read
      if (!keep_a) slice_tile<kOzM>(g.a, pa + (long long)k0 * g.a.sk, ra0, klen, mxa, sa);
      slice_tile<BN>(g.b, pb + (long long)k0 * g.b.sk, rb0, klen, mxb, sb);
      // the generic-proxy writes become visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint64_t da0 = sw128_desc(smem_u32(sa)), db0 = sw128_desc(smem_u32(sb));
        // the descriptor's address field is the byte address / 16.  The B
        // slices lie one after another, so A_p times B_q0 .. B_q1 is one MMA
        // of N = (q1 - q0 + 1) BN whose output columns start at accumulator
        // p + q0: every pair (p, q) lands on its diagonal p + q.  N <= 256.
        constexpr int kQ = 256 / BN < kOzSlices ? 256 / BN : kOzSlices;  // B slices per MMA
        for (int p = 0; p < kOzSlices; p++)
          for (int q0 = 0; q0 + p < kOzSlices; q0 += kQ) {
            const int nq = min(kQ, kOzSlices - p - q0);
            const uint32_t id = idesc_bf16(kOzM, nq * BN);
            const uint32_t dcol = tmem + (uint32_t)((p + q0) * BN);
#pragma unroll
            for (int kk = 0; kk < kOzChunk / 16; kk++)
              // first write of every accumulator: p = 0, kk = 0
              mma_bf16(dcol, da0 + (uint64_t)(p * (kOzTileA / 16) + kk * 2),
                       db0 + (uint64_t)(q0 * (BN * 128 / 16) + kk * 2), id,
                       (p == 0 && kk == 0) ? 0u : 1u);
          }
        tc_commit(mbar);
      }
      __syncwarp();
      const bool ok = mbar_wait(mbar, phase & 1u);
      phase++;
      if (!ok) atomicExch(&s_ok, 0);
      tc_fence_after();
      __syncthreads();
      if (!s_ok) break;
      // this chunk's exact product, rounded once: a one-chunk item writes it
      // (with alpha and beta) straight from the accumulator rows; otherwise
      // it is staged by row for the coalesced accumulation below
      const bool direct = nch == 1;
      const int ea = row_scale(mxa[r]);
      const int ga = ra0 + r;
      // this thread's output row (or, swapped, column) of C: element
      // (ga, rb0 + col) at cbase + col * cstride
      double* const cbase = cz + (g.swap ? (long long)rb0 * g.ldc + ga : (long long)ga * g.ldc + rb0);
      const long long cstride = g.swap ? g.ldc : 1;
#pragma unroll 1
      for (int cg = part * 8; cg < BN; cg += 32) {
        float D[kOzSlices][8];
        tmem_ld_diagonals<BN>(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cg, D);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int eb = row_scale(mxb[cg + j]);
          double x;
          if (ea == kOzBad || eb == kOzBad) {
            x = __longlong_as_double(0x7FF8000000000000ll);
          } else {
            // D_d sums at most min(d + 1, 8 - ...) x 64 digit products below
            // 2^14: |D_0 .. D_3| < 2^22, |D_4 .. D_7| < 2^23, so the pairs
            // D_d 2^7 + D_(d+1) fit in 32 bits
            const int d01 = int_small(D[0][j]) * 128 + int_small(D[1][j]);
            const int d23 = int_small(D[2][j]) * 128 + int_small(D[3][j]);
            const int d45 = __float2int_rz(D[4][j]) * 128 + __float2int_rz(D[5][j]);
            const int d67 = __float2int_rz(D[6][j]) * 128 + __float2int_rz(D[7][j]);
            const long long H = (long long)d01 * (1ll << 14) + d23;
            const long long L = (long long)d45 * (1ll << 14) + d67;
            x = assemble(H, L, ea + eb - 63);
          }
          if (!direct) {
            stage[r * kST + cg + j] = x;
          } else if (ga < g.a.rows && rb0 + cg + j < g.b.rows) {
            double* cp = cbase + (long long)(cg + j) * cstride;
            if (plain) {
              *cp = x;
            } else {
              double v = g.alpha * x;
              if (g.beta != 0.0) v = fma(g.beta, *cp, v);
              *cp = v;
            }
          }
        }
      }
      // every thread's TMEM reads are done before the next chunk's MMAs
      tc_fence_before();
      __syncthreads();
      if (direct) continue;
      // coalesced output: consecutive threads on consecutive addresses of C
      // (along its rows, or along the A side when the product is swapped);
      // the first chunk stores, later ones add in chunk order; alpha with
      // the last
      const bool last = c == nch - 1;
      // thread tid takes elements tid + 512 i of the tile: along C's rows a
      // fixed column and rows 512 / BN apart; swapped, a fixed A-side row
      // and columns 4 apart
      constexpr int kPer = kOzM * BN / kOzThreads;  // 4, 8 or 16
      const int row0 = g.swap ? tid % kOzM : tid / BN, col0 = g.swap ? tid / kOzM : tid % BN;
      const int drow = g.swap ? 0 : kOzThreads / BN, dcol = g.swap ? kOzThreads / kOzM : 0;
      const long long at0 = g.swap ? (long long)(rb0 + col0) * g.ldc + ra0 + row0
                                   : (long long)(ra0 + row0) * g.ldc + rb0 + col0;
      const long long dat = g.swap ? (long long)dcol * g.ldc : (long long)drow * g.ldc;
      const int st0 = row0 * kST + col0, dst = drow * kST + dcol;
      const bool need_old = c > 0;
      double old[kPer];
#pragma unroll
      for (int i = 0; i < kPer; i++) {
        const bool live = ra0 + row0 + i * drow < g.a.rows && rb0 + col0 + i * dcol < g.b.rows;
        old[i] = (live && need_old) ? cz[at0 + i * dat] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kPer; i++) {
        if (ra0 + row0 + i * drow >= g.a.rows || rb0 + col0 + i * dcol >= g.b.rows) continue;
        const double x = stage[st0 + i * dst];
        double v = c == 0 ? x : old[i] + x;
        if (last && !plain) v = g.alpha * v;  // (beta is 0 here)
        cz[at0 + i * dat] = v;
      }
    }
  }
  if (!s_ok && tid == 0 && g.err) atomicOr(g.err, QTT_DEVERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

int oz_bn(int rows) { return rows > 32 ? 64 : rows > 16 ? 32 : 16; }

size_t oz_smem(int BN) { return 1024 + (size_t)kOzSlices * kOzTileA + (size_t)kOzSlices * BN * 128; }

void oz_attr_once() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    ok = cudaFuncSetAttribute(k_gemm_oz<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)oz_smem(16)) == cudaSuccess &&
         cudaFuncSetAttribute(k_gemm_oz<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)oz_smem(32)) == cudaSuccess &&
         cudaFuncSetAttribute(k_gemm_oz<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)oz_smem(64)) == cudaSuccess;
    cudaGetLastError();
  });
  if (!ok) throw QttError(QTT_ERR_CUDA, "emulated FP64 GEMM: shared-memory opt-in refused");
}

// Launch shape of a product: the 128-row side (the orientation with less
// padding; ties: no swap), the output tile width, and for an unbatched
// product whose tiles cannot fill the GPU a split of K over CTAs (whole
// chunks per slice, at most 16 slices, at most 16 chunks per slice).
struct OzPlan {
  bool swap;
  int BN, tiles, nch, S, kslice;
};

OzPlan oz_plan(const GemmF64& g, int max_s) {
  auto padded = [](int ra, int rb) {
    const int bn = oz_bn(rb);
    return (double)((ra + kOzM - 1) / kOzM) * kOzM * (double)((rb + bn - 1) / bn) * bn;
  };
  OzPlan p{};
  p.swap = padded(g.N, g.M) < padded(g.M, g.N);
  const int ra = p.swap ? g.N : g.M, rb = p.swap ? g.M : g.N;
  p.BN = oz_bn(rb);
  p.tiles = ((ra + kOzM - 1) / kOzM) * ((rb + p.BN - 1) / p.BN);
  p.nch = (g.K + kOzChunk - 1) / kOzChunk;
  p.S = 1;
  if ((long long)g.nb1 * g.nb2 == 1 && p.nch > 1) {
    // (a CTA over several chunks accumulates in its output, so beta != 0
    // takes the slice sum)
    // max_s > 16 (the library's own products, when their scratch allows):
    // as many slices as keep every item on its own SM
    int want;
    if (max_s > 16)
      want = p.tiles < 74 ? std::max(2, 148 / p.tiles) : g.beta != 0.0 ? 16 : 1;
    else
      want = g.beta != 0.0 ? 16 : p.tiles < 74 ? (148 + p.tiles - 1) / p.tiles : 1;
    const int lo = (p.nch + 15) / 16, hi = std::min(std::max(16, max_s), p.nch);
    int S = std::max(lo, std::min(want, hi));
    const int cps = (p.nch + S - 1) / S;
    p.S = (p.nch + cps - 1) / cps;
    p.kslice = p.S > 1 ? cps * kOzChunk : 0;
  }
  return p;
}

}  // namespace

bool gemm_oz_eligible(const GemmF64& g) {
  if (g.K < 16 || g.M < 1 || g.N < 1) return false;
  const long long nb = (long long)g.nb1 * g.nb2;
  if (nb < 1 || nb > 65535) return false;
  if (g.K > (nb == 1 ? 16 * 16 * kOzChunk : 16 * kOzChunk)) return false;
  if (nb > 1 && g.K > kOzChunk && g.beta != 0.0) return false;  // no slice sum for batches
  return std::max(g.M, g.N) >= 32 && (double)g.M * g.N * g.K * (double)nb >= (double)(1 << 21);
}

// The library's own products: the shapes above, with the smallest K and the
// smallest multiply-add count that go to the tensor cores settable for
// measurement (QTT_OZ_MIN_K, default 16; QTT_OZ_MIN_LOG2, default 21).  The
// kernel zero-fills a partial K chunk, so any K >= 1 is exact.
bool gemm_oz_dispatch(const GemmF64& g) {
  static const int min_k = [] {
    const char* e = getenv("QTT_OZ_MIN_K");
    const int v = e ? atoi(e) : 16;
    return v < 1 ? 1 : v;
  }();
  static const int min_log2 = [] {
    const char* e = getenv("QTT_OZ_MIN_LOG2");
    const int v = e ? atoi(e) : 21;
    return v < 10 ? 10 : (v > 40 ? 40 : v);
  }();
  if (g.K < min_k || g.M < 1 || g.N < 1) return false;
  const long long nb = (long long)g.nb1 * g.nb2;
  if (nb < 1 || nb > 65535) return false;
  if (g.K > (nb == 1 ? 16 * 16 * kOzChunk : 16 * kOzChunk)) return false;
  if (nb > 1 && g.K > kOzChunk && g.beta != 0.0) return false;
  return std::max(g.M, g.N) >= 32 &&
         (double)g.M * g.N * g.K * (double)nb >= ldexp(1.0, min_log2);
}

int gemm_oz_splits(const GemmF64& g, int max_s) { return oz_plan(g, max_s).S; }

void launch_gemm_oz(const GemmF64& g, int* err, cudaStream_t s, bool ext, double* scratch,
                    size_t scratch_n, int max_s) {
  if (ext ? !gemm_oz_eligible(g) : !gemm_oz_dispatch(g))
    throw QttError(QTT_ERR_SHAPE, "emulated FP64 GEMM shape");
  {
    const long long zb1 = g.nb1 - 1, zb2 = g.nb2 - 1;
    const long long ea = g.tA ? (long long)(g.K - 1) * g.lda + g.M : (long long)(g.M - 1) * g.lda + g.K;
    const long long eb = g.tB ? (long long)(g.N - 1) * g.ldb + g.K : (long long)(g.K - 1) * g.ldb + g.N;
    const long long ec = (long long)(g.M - 1) * g.ldc + g.N;
    check_range(g.A, zb1 * g.sA1 + zb2 * g.sA2 + ea, sizeof(double), ext ? "ext oz gemm A" : "oz gemm A");
    check_range(g.B, zb1 * g.sB1 + zb2 * g.sB2 + eb, sizeof(double), ext ? "ext oz gemm B" : "oz gemm B");
    check_range(g.C, zb1 * g.sC1 + zb2 * g.sC2 + ec, sizeof(double), ext ? "ext oz gemm C" : "oz gemm C");
  }
  oz_attr_once();
  const OzPlan pl = oz_plan(g, ext ? 16 : max_s);
  // op(A) (M x K): element (m, k); op(B)^T (N x K): element (n, k)
  OzOperand opA{g.A, g.sA1, g.sA2, g.tA ? 1 : (long long)g.lda, g.tA ? (long long)g.lda : 1, g.M};
  OzOperand opB{g.B, g.sB1, g.sB2, g.tB ? (long long)g.ldb : 1, g.tB ? 1 : (long long)g.ldb, g.N};
  OzParams p{};
  p.K = g.K;
  p.nch = pl.nch;
  p.BN = pl.BN;
  p.nb2 = g.nb2;
  p.swap = pl.swap ? 1 : 0;
  p.skip = g.skip;
  p.err = err;
  int nz = g.nb1 * g.nb2;
  if (pl.S > 1) {
    // K slices into S partial products (M x N each), summed in slice order
    const size_t need = (size_t)pl.S * g.M * g.N;
    if (!scratch || scratch_n < need) throw QttError(QTT_ERR_SHAPE, "emulated GEMM: split-K scratch");
    check_range(scratch, (long long)need, sizeof(double), "oz gemm partials");
    opA.s1 = (long long)pl.kslice * opA.sk;
    opB.s1 = (long long)pl.kslice * opB.sk;
    opA.s2 = opB.s2 = 0;
    p.kslice = pl.kslice;
    p.nb2 = 1;
    p.C = scratch;
    p.ldc = g.N;
    p.sC1 = (long long)g.M * g.N;
    p.sC2 = 0;
    p.alpha = 1.0;
    p.beta = 0.0;
    nz = pl.S;
  } else {
    p.C = g.C;
    p.ldc = g.ldc;
    p.sC1 = g.sC1;
    p.sC2 = g.sC2;
    p.alpha = g.alpha;
    p.beta = g.beta;
  }
  p.a = pl.swap ? opB : opA;
  p.b = pl.swap ? opA : opB;
  p.nz = nz;
  // persistent CTAs (one per SM: the shared memory allows no second)
  const long long items =
      (long long)((p.b.rows + p.BN - 1) / p.BN) * ((p.a.rows + kOzM - 1) / kOzM) * nz;
  static const int sms = [] {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  dim3 grid((unsigned)std::min<long long>(items, sms));
  pre_launch(s);
  if (p.BN == 64)
    k_gemm_oz<64><<<grid, kOzThreads, oz_smem(64), s>>>(p);
  else if (p.BN == 32)
    k_gemm_oz<32><<<grid, kOzThreads, oz_smem(32), s>>>(p);
  else
    k_gemm_oz<16><<<grid, kOzThreads, oz_smem(16), s>>>(p);
  const char* name = "k_gemm_oz";
  if (shape_profiling()) {
    char tag[80];
    snprintf(tag, sizeof tag, "%dx%dx%d b%d %d%d%s s%d", g.M, g.N, g.K, g.nb1 * g.nb2, g.tA,
             g.tB, pl.swap ? " sw" : "", pl.S);
    name = shape_name(name, tag);
  }
  post_launch(name, s, 2.0 * g.M * g.N * (double)g.K * g.nb1 * g.nb2);
  if (pl.S > 1)
    launch_sum_slices(scratch, pl.S, g.M, g.N, g.C, g.ldc, g.alpha, g.beta, g.skip, s, ext);
}
