// Tensor-core contractions of the mixed form on sm_103a: a TMA-fed
// tcgen05 GEMM in TF32 with the 3xTF32 split and FP32 accumulation in
// tensor memory, the kernels that prepare its operands, and the randomised
// subspace search built from it.
//
// GEMM (k_tc_gemm): one CTA of 128 threads per 128 x BN output tile (and
// split-K slice).  Thread 0 streams K blocks of 32 elements through a ring
// of shared-memory stages with cp.async.bulk.tensor (four boxes per stage:
// A hi/lo, B hi/lo, 128-byte swizzle), thread 32 issues the tcgen05.mma
// instructions (kind::tf32, M = 128, N = BN, K = 8; per K step lo*hi,
// hi*lo, hi*hi into one FP32 accumulator in TMEM) and returns each stage to
// the producer with tcgen05.commit; after the last commit all four warps
// read the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. output rows) and write it out.  Every wait on an mbarrier is bounded
// (one second of global time); a wait that gives up sets QTT_DEVERR_TIMEOUT
// in the error word, the CTA stops issuing, waits (bounded) for the copies it
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kBM = 128;     // MMA M
constexpr int kBK = 32;      // K elements per stage (128 bytes of FP32)
constexpr uint32_t kAPlane = kBM * kBK * 4;  // bytes of one A plane in a stage

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

struct GemmParams {
  int M, N, KB, kbs, BN, stages;
  TcOut o;
  int* err;
  const int* stop;  // nonzero: the launch does nothing (a search given up)
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              GemmParams g) {
  if (g.stop && *g.stop) return;  // uniform over the grid
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t b_plane = (uint32_t)g.BN * kBK * 4;
  const uint32_t stage_bytes = 2 * kAPlane + 2 * b_plane;
  uint64_t* bars = (uint64_t*)(base + (size_t)g.stages * stage_bytes);  // full, empty, done
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * g.stages + 1);
  __shared__ int s_abort, s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * g.BN;
  const int kb0 = blockIdx.z * g.kbs;
  const int nkb = max(0, min(g.KB, kb0 + g.kbs) - kb0);
  const uint32_t ncols = g.BN <= 32 ? 32u : g.BN <= 64 ? 64u : g.BN <= 128 ? 128u : 256u;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + g.stages),
                 done = smem_u32(bars + 2 * g.stages);
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    for (int i = 0; i < 2 * g.stages + 1; i++) mbar_init(smem_u32(bars + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (nkb > 0 && warp == 0 && lane == 0) {
    // producer: K block i into stage i % stages once the MMAs of block
    // i - stages have released it
    for (int i = 0; i < nkb; i++) {
      const int st = i % g.stages;
      if (i >= g.stages && !mbar_wait(empty0 + 8 * st, ((i / g.stages) & 1) ^ 1)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const uint32_t sb = smem_u32(base + (size_t)st * stage_bytes);
      const uint32_t full = full0 + 8 * st;
      mbar_expect_tx(full, stage_bytes);
      const int kx = (kb0 + i) * kBK;
      tma_load_3d(sb, &tA, kx, m0, 0, full);
      tma_load_3d(sb + kAPlane, &tA, kx, m0, 1, full);
      tma_load_3d(sb + 2 * kAPlane, &tB, kx, n0, 0, full);
      tma_load_3d(sb + 2 * kAPlane + b_plane, &tB, kx, n0, 1, full);
      *(volatile int*)&s_issued = i + 1;
    }
  } else if (nkb > 0 && warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32(kBM, g.BN);
    for (int i = 0; i < nkb; i++) {
      const int st = i % g.stages;
      if (!mbar_wait(full0 + 8 * st, (i / g.stages) & 1)) {
        atomicExch(&s_abort, 1);
        break;
      }
      *(volatile int*)&s_consumed = i + 1;
      tc_fence_after();
      const uint32_t sb = smem_u32(base + (size_t)st * stage_bytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 8; kk++) {
        const uint64_t ah = sw128_desc(sb + kk * 32), al = sw128_desc(sb + kAPlane + kk * 32);
        const uint64_t bh = sw128_desc(sb + 2 * kAPlane + kk * 32),
                       bl = sw128_desc(sb + 2 * kAPlane + b_plane + kk * 32);
        tc_mma(tmem, al, bh, idesc, (i | kk) != 0 ? 1u : 0u);
        tc_mma(tmem, ah, bl, idesc, 1u);
        tc_mma(tmem, ah, bh, idesc, 1u);
      }
      tc_commit(empty0 + 8 * st);
    }
    tc_commit(done);
  }
  __syncwarp();

  // epilogue: warp w holds output rows m0 + 32 w + lane in TMEM lanes 32 w + lane
  bool ok = true;
  if (nkb > 0) ok = mbar_wait(done, 0);
  ok = __all_sync(0xffffffffu, ok) && !*(volatile int*)&s_abort;
  ok = __all_sync(0xffffffffu, ok);
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  const TcOut& o = g.o;
  for (int c = 0; c < g.BN; c += 16) {
    float v[16];
    if (nkb > 0 && ok) {
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; i++) v[i] = 0.0f;
    }
    if (row < g.M) {
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const int col = n0 + c + i;
        if (col >= g.N) continue;
        const long long at = (long long)row * o.ldo + col;
        if (o.mode == 0) {
          o.out[blockIdx.z * o.slice + at] = v[i];
        } else if (o.mode == 1) {
          const float hi = tf32_round(v[i]);
          o.out[at] = hi;
          o.out[o.plane + at] = tf32_round(v[i] - hi);
        } else {
          o.out64[at] = o.alpha * (double)v[i];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_abort) {
    // copies issued but never consumed still land in this CTA's shared
    // memory: wait for them (bounded) before the CTA exits
    for (int i = s_consumed; i < s_issued; i++)
      mbar_wait(full0 + 8 * (i % g.stages), (i / g.stages) & 1);
    if (g.err) atomicOr(g.err, QTT_DEVERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// FP64 -> two TF32 planes, K-major, through a 32 x 32 shared tile (reads are
// coalesced in both orientations).  Zero for K <= k < kpad.
__global__ void __launch_bounds__(256) k_tc_split(const double* __restrict__ src, int ld,
                                                  int trans, int R, int K, float* __restrict__ dst,
                                                  int kpad, long long plane) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (trans) {
    // src[k * ld + r]: consecutive threads along r
    for (int q = ty; q < 32; q += 8) {
      const int k = k0 + q, r = r0 + tx;
      tile[q][tx] = (k < K && r < R) ? src[(long long)k * ld + r] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int r = r0 + q, k = k0 + tx;
      if (r >= R) continue;
      const double x = tile[tx][q];
      const float hi = tf32_round((float)x);
      dst[(long long)r * kpad + k] = hi;
      dst[plane + (long long)r * kpad + k] = tf32_round((float)(x - (double)hi));
    }
  } else {
    for (int q = ty; q < 32; q += 8) {
      const int r = r0 + q, k = k0 + tx;
      if (r >= R) continue;
      const double x = k < K ? src[(long long)r * ld + k] : 0.0;
      const float hi = tf32_round((float)x);
      dst[(long long)r * kpad + k] = hi;
      dst[plane + (long long)r * kpad + k] = tf32_round((float)(x - (double)hi));
    }
  }
}

__global__ void k_tc_reduce(const float* __restrict__ P, int S, long long slice, int ldp, int M,
                            int N, TcOut o, int trans, const int* stop) {
  if (stop && *stop) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const int m = (int)(e / N), n = (int)(e % N);
  float v = 0.0f;
  for (int z = 0; z < S; z++) v += P[z * slice + (long long)m * ldp + n];
  const long long at = trans ? (long long)n * o.ldo + m : (long long)m * o.ldo + n;
  if (o.mode == 0) {
    o.out[at] = v;
  } else if (o.mode == 1) {
    const float hi = tf32_round(v);
    o.out[at] = hi;
    o.out[o.plane + at] = tf32_round(v - hi);
  } else {
    o.out64[at] = o.alpha * (double)v;
  }
}

// SplitMix64 (Steele, Lea and Flood 2014): state += golden gamma, then
// the published finaliser.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Gaussian test matrix Omega^T (p x K), TF32-exact (lo plane zero), by
// Box-Muller on two SplitMix64 uniforms per entry; zero for k >= K.
__global__ void k_tc_omega(float* dst, int p, int K, int kpad, long long plane,
                           unsigned long long key, int* stop) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (stop && e == 0) *stop = 0;  // a new search starts
  if (e >= (long long)p * kpad) return;
  const int i = (int)(e / kpad), k = (int)(e % kpad);
  float v = 0.0f;
  if (k < K) {
    const uint64_t h = splitmix64(key ^ ((uint64_t)i << 32) ^ (uint64_t)k);
    const uint64_t h2 = splitmix64(h);
    const double u1 = ((double)(h >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    v = tf32_round((float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2)));
  }
  dst[e] = v;
  dst[plane + e] = 0.0f;
}

// Orthonormalisation of Y (s x p, FP32, row-major ldy) by classical
// Gram-Schmidt with one reorthogonalisation pass per column (CGS2), one CTA,
// columns in shared memory.  Columns j >= rank = max(1, min(pmax, sact,
// lact * lact2)) are
// zero, as is a column with nothing left after the projections.  Writes
// Q^T planes (p x kpad, TF32 hi/lo) and optionally Q in FP64.
struct OrthArgs {
  const float* Y;
  int ldy, s, p;
  DimRef sact, lact, lact2;
  int pmax;
  float* qt;
  int kpad;
  long long plane;
  double* q64;
  int ld64, q64T;
  int* r_out;
  int keep, iters;
  double rho_max;
  int* accept;
  long long* counts;
  int* stop;   // the search's stop word (read; written by the early test)
  int early;   // run the acceptance test now and stop the search if it fails
};

constexpr int kOrthThreads = 512;

__global__ void __launch_bounds__(kOrthThreads, 1) k_tc_orth(OrthArgs a) {
  extern __shared__ float sq[];  // [p][s], columns kept unnormalised until the end
  __shared__ float h[128];
  __shared__ float inv[128];    // 1 / |column|^2 (0: a dropped column)
  __shared__ float cnorm[128];  // column norms after the projections
  __shared__ float red[kOrthThreads / 32], red0[kOrthThreads / 32];
  if (a.stop && *a.stop) return;  // uniform over the block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = kOrthThreads / 32;
  const int s = a.s, p = a.p;
  const int rank =
      max(1, min(a.pmax, min(dval(a.sact), dval(a.lact) * (a.lact2.p ? dval(a.lact2) : 1))));
  for (int e = tid; e < s * p; e += kOrthThreads) {
    const int r = e / p, j = e % p;
    sq[j * s + r] = a.Y[(long long)r * a.ldy + j];
  }
  // the update phase: two threads per row, each over half of the earlier
  // columns (partners are adjacent lanes)
  const int row = tid >> 1, half = tid & 1;
  __syncthreads();
  for (int j = 0; j < p; j++) {
    float* y = sq + (size_t)j * s;
    if (j >= rank) {
      for (int r = tid; r < s; r += kOrthThreads) y[r] = 0.0f;
      inv[j] = 0.0f;  // every thread writes the same value before it reads it
      cnorm[j] = 0.0f;
      continue;  // uniform over the block
    }
    for (int pass = 0; pass < 2; pass++) {
      // h_i = (q_i . y) / |q_i|^2 for the earlier columns i < j
      for (int i = warp; i < j; i += nw) {
        const float* q = sq + (size_t)i * s;
        float d0 = 0.0f, d1 = 0.0f;
        int r = lane;
        for (; r + 32 < s; r += 64) {
          d0 = fmaf(q[r], y[r], d0);
          d1 = fmaf(q[r + 32], y[r + 32], d1);
        }
        if (r < s) d0 = fmaf(q[r], y[r], d0);
        float d = d0 + d1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) h[i] = d * inv[i];
      }
      __syncthreads();
      // y -= sum_i q_i h_i (and the squared norms before / after)
      float t = 0.0f, c = 0.0f;
      if (row < s) {
        float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
        int i = half;
        for (; i + 6 < j; i += 8) {
          c0 = fmaf(sq[(size_t)i * s + row], h[i], c0);
          c1 = fmaf(sq[(size_t)(i + 2) * s + row], h[i + 2], c1);
          c2 = fmaf(sq[(size_t)(i + 4) * s + row], h[i + 4], c2);
          c3 = fmaf(sq[(size_t)(i + 6) * s + row], h[i + 6], c3);
        }
        for (; i < j; i += 2) c0 = fmaf(sq[(size_t)i * s + row], h[i], c0);
        c = (c0 + c1) + (c2 + c3);
      }
      c += __shfl_xor_sync(0xffffffffu, c, 1);  // the two halves of the row
      if (row < s && half == 0) {  // the row's owner
        const float old = y[row];
        const float nv = old - c;
        t = pass == 0 ? old * old : nv * nv;
        y[row] = nv;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) (pass == 0 ? red0 : red)[warp] = t;
      __syncthreads();
    }
    float nrm2 = 0.0f, nrm0 = 0.0f;
    for (int i = 0; i < nw; i++) {
      nrm2 += red[i];
      nrm0 += red0[i];
    }
    // nothing left beyond rounding of an (almost) dependent column: drop it
    // rather than keep noise of a vanishing vector
    const bool keep = nrm2 > 1e-36f && nrm2 > 1e-24f * nrm0;
    inv[j] = keep ? 1.0f / nrm2 : 0.0f;  // every thread writes the same value
    cnorm[j] = keep ? sqrtf(nrm2) : 0.0f;
  }
  __syncthreads();
  for (int e = tid; e < s * p; e += kOrthThreads) {
    const int j = e / s;
    sq[e] *= sqrtf(inv[j]);
  }
  __syncthreads();
  if ((a.accept || a.early) && tid == 0) {
    // cnorm[j] ~ sigma_j^2 (orthogonal iteration orders the columns)
    const int full = min(dval(a.sact), dval(a.lact) * (a.lact2.p ? dval(a.lact2) : 1));
    const int kk = min(a.keep, rank);
    bool ok;
    if (rank >= full || kk >= rank) {
      ok = rank >= full;  // the basis spans the whole actual space
    } else if (!(cnorm[kk - 1] > 0.0f)) {
      ok = true;  // fewer than keep directions carry weight: nothing to resolve
    } else {
      const double rho = (double)cnorm[rank - 1] / (double)cnorm[kk - 1];
      ok = a.iters >= 1 && rho <= a.rho_max && pow(rho, (double)a.iters) <= 1e-6;
    }
    if (!a.early) {
      *a.accept = ok ? 1 : 0;
      if (a.counts) atomicAdd((unsigned long long*)(a.counts + (ok ? 0 : 1)), 1ull);
    } else if (!ok) {
      // the full iteration count will not reach the bar either: give up now
      // (the remaining launches of this search do nothing)
      *a.stop = 1;
      *a.accept = 0;
      if (a.counts) atomicAdd((unsigned long long*)(a.counts + 1), 1ull);
    }
  }
  if (a.qt) {
    for (long long e = tid; e < (long long)p * a.kpad; e += kOrthThreads) {
      const int j = (int)(e / a.kpad), r = (int)(e % a.kpad);
      const float v = r < s ? sq[(size_t)j * s + r] : 0.0f;
      const float hi = tf32_round(v);
      a.qt[e] = hi;
      a.qt[a.plane + e] = tf32_round(v - hi);
    }
  }
  if (a.q64) {
    for (int e = tid; e < s * p; e += kOrthThreads) {
      const int j = e / s, r = e % s;
      const long long at = a.q64T ? (long long)j * a.ld64 + r : (long long)r * a.ld64 + j;
      a.q64[at] = (double)sq[(size_t)j * s + r];
    }
  }
  if (a.r_out && tid == 0) *a.r_out = rank;
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
    cudaGetLastError();
  });
  if (!fn) throw QttError(QTT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  return fn;
}

// Tensor map of a split operand: dims (kpad, rows, 2 planes), box
// (32, box_rows, 1), 128-byte swizzle, zero fill outside the extents.
CUtensorMap make_tmap(const TcOperand& op, int box_rows) {
  if (((uintptr_t)op.p & 15) || op.kpad % 32 || op.plane % 4 || box_rows < 8 || box_rows > 256)
    throw QttError(QTT_ERR_SHAPE, "tensor-core operand alignment");
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)op.kpad, (cuuint64_t)op.rows, 2};
  const cuuint64_t strides[2] = {(cuuint64_t)op.kpad * 4, (cuuint64_t)op.plane * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)op.p, dims,
                                 strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw QttError(QTT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

size_t gemm_smem(int BN, int stages) {
  return (size_t)stages * (2 * kAPlane + 2 * (size_t)BN * kBK * 4) + 1024 +
         (size_t)(2 * stages + 1) * 8 + 16;
}

int gemm_stages(int BN) {
  const size_t limit = 220 * 1024;  // the opt-in of gemm_attr_once
  for (int st = 4; st >= 2; st--)
    if (gemm_smem(BN, st) <= limit) return st;
  return 2;
}

// Dynamic shared memory opt-in (static shared memory comes on top, within
// the 227 KB a block may hold).
void gemm_attr_once() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    ok = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              220 * 1024) == cudaSuccess &&
         cudaFuncSetAttribute(k_tc_orth, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024) == cudaSuccess;
    cudaGetLastError();
  });
  if (!ok) throw QttError(QTT_ERR_CUDA, "tensor-core kernels: shared-memory opt-in refused");
}

long long planes_extent(const TcOperand& op) { return op.plane + (long long)op.rows * op.kpad; }

}  // namespace

void launch_tc_split(const double* src, int ld, int trans, int R, int K, float* dst, int kpad,
                     long long plane, cudaStream_t s, bool src_ext) {
  if (R <= 0 || kpad <= 0) return;
  if (K > kpad || kpad % 32) throw QttError(QTT_ERR_SHAPE, "tc split shape");
  check_range(src, trans ? (long long)(K - 1) * ld + R : (long long)(R - 1) * ld + K,
              sizeof(double), src_ext ? "ext tc split src" : "tc split src");
  check_range(dst, plane + (long long)R * kpad, sizeof(float), "tc split dst");
  pre_launch(s);
  dim3 grid(kpad / 32, ceil_div(R, 32));
  k_tc_split<<<grid, 256, 0, s>>>(src, ld, trans, R, K, dst, kpad, plane);
  post_launch("k_tc_split", s);
}

void launch_tc_gemm(const TcOperand& A, const TcOperand& B, int M, int N, int BN, int S,
                    const TcOut& o, int* err, cudaStream_t s, const int* stop) {
  if (M <= 0 || N <= 0) return;
  if (A.kpad != B.kpad || BN % 16 || BN < 16 || BN > 256 || S < 1 || (S > 1 && o.mode != 0) ||
      M > A.rows || N > B.rows)
    throw QttError(QTT_ERR_SHAPE, "tc gemm shape");
  check_range(A.p, planes_extent(A), sizeof(float), "tc gemm A");
  check_range(B.p, planes_extent(B), sizeof(float), "tc gemm B");
  if (o.mode == 2)
    check_range(o.out64, (long long)(M - 1) * o.ldo + N, sizeof(double), "tc gemm C");
  else if (o.mode == 1)
    check_range(o.out, o.plane + (long long)(M - 1) * o.ldo + N, sizeof(float), "tc gemm C");
  else
    check_range(o.out, (long long)(S - 1) * o.slice + (long long)(M - 1) * o.ldo + N,
                sizeof(float), "tc gemm C");
  gemm_attr_once();
  const CUtensorMap ta = make_tmap(A, kBM), tb = make_tmap(B, BN);
  GemmParams g{};
  g.M = M;
  g.N = N;
  g.KB = A.kpad / kBK;
  g.kbs = ceil_div(g.KB, S);
  g.BN = BN;
  g.stages = gemm_stages(BN);
  g.o = o;
  g.err = err;
  g.stop = stop;
  dim3 grid(ceil_div(N, BN), ceil_div(M, kBM), S);
  pre_launch(s);
  k_tc_gemm<<<grid, kThreads, gemm_smem(BN, g.stages), s>>>(ta, tb, g);
  post_launch("k_tc_gemm", s, 2.0 * M * N * (double)A.kpad);
}

void launch_tc_reduce(const float* P, int S, long long slice, int ldp, int M, int N,
                      const TcOut& o, int trans, cudaStream_t s, bool out_ext, const int* stop) {
  if (M <= 0 || N <= 0) return;
  check_range(P, (long long)(S - 1) * slice + (long long)(M - 1) * ldp + N, sizeof(float),
              "tc reduce P");
  const long long ext = trans ? (long long)(N - 1) * o.ldo + M : (long long)(M - 1) * o.ldo + N;
  if (o.mode == 2)
    check_range(o.out64, ext, sizeof(double), out_ext ? "ext tc reduce out" : "tc reduce out");
  else
    check_range(o.out, (o.mode == 1 ? o.plane : 0) + ext, sizeof(float), "tc reduce out");
  pre_launch(s);
  k_tc_reduce<<<ceil_div((long long)M * N, 256), 256, 0, s>>>(P, S, slice, ldp, M, N, o, trans,
                                                              stop);
  post_launch("k_tc_reduce", s);
}

// ------------------------------------------------------------ subspace search
bool tc_search_supported(int s, int l, int p) {
  return s >= 16 && s <= 256 && l >= 16 && p >= 1 && p <= 128 && p <= s;
}

namespace {
struct SearchLayout {
  int s, l, p, ks, kl, S;
  size_t xa, xb, zt, qt, part, y, total;
};
SearchLayout search_layout(int s, int l, int p) {
  SearchLayout L{};
  L.s = s;
  L.l = l;
  L.p = p;
  L.ks = tc_kpad(s);
  L.kl = tc_kpad(l);
  // split K of Y = X Z over slices of at least four K blocks, about 128 CTAs
  const int mt = ceil_div(s, kBM);
  const int kb = L.kl / kBK;
  L.S = std::max(1, std::min(kb / 4, 128 / mt));
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += (n + 63) / 64 * 64;  // 256-byte alignment of every piece
    return at;
  };
  L.xa = take(2 * (size_t)s * L.kl);
  L.xb = take(2 * (size_t)l * L.ks);
  L.zt = take(2 * (size_t)p * L.kl);
  L.qt = take(2 * (size_t)p * L.ks);
  L.part = take((size_t)L.S * s * p);
  L.y = take((size_t)s * p);
  L.total = o;
  return L;
}
}  // namespace

size_t tc_search_scratch_floats(int s, int l, int p) { return search_layout(s, l, p).total; }

void tc_search(const TcSearch& a, float* scratch, size_t scratch_floats, int* err,
               cudaStream_t st) {
  const int s = a.small_is_rows ? a.rows : a.cols;
  const int l = a.small_is_rows ? a.cols : a.rows;
  const int p = a.p;
  if (!tc_search_supported(s, l, p)) throw QttError(QTT_ERR_SHAPE, "tc search shape");
  const SearchLayout L = search_layout(s, l, p);
  if (scratch_floats < L.total) throw QttError(QTT_ERR_SHAPE, "tc search scratch");
  gemm_attr_once();
  float* xa = scratch + L.xa;
  float* xb = scratch + L.xb;
  float* zt = scratch + L.zt;
  float* qt = scratch + L.qt;
  float* part = scratch + L.part;
  float* y = scratch + L.y;
  // XA = X_s (s x l, K = l) and XB = X_s^T (l x s, K = s), X_s = X or X^T
  launch_tc_split(a.X, a.ld, a.small_is_rows ? 0 : 1, s, l, xa, L.kl, (long long)s * L.kl, st);
  launch_tc_split(a.X, a.ld, a.small_is_rows ? 1 : 0, l, s, xb, L.ks, (long long)l * L.ks, st);
  {
    pre_launch(st);
    const long long n = (long long)p * L.kl;
    k_tc_omega<<<ceil_div(n, 256), 256, 0, st>>>(zt, p, l, L.kl, n, a.key, a.stop);
    post_launch("k_tc_omega", st);
  }
  const TcOperand XA{xa, s, L.kl, (long long)s * L.kl};
  const TcOperand XB{xb, l, L.ks, (long long)l * L.ks};
  const TcOperand ZT{zt, p, L.kl, (long long)p * L.kl};
  const TcOperand QT{qt, p, L.ks, (long long)p * L.ks};
  const int bnp = ((p + 15) / 16) * 16;
  for (int it = 0; it <= a.iters; it++) {
    // Y = X_s Z  (s x p), K = l split over L.S slices
    TcOut o{};
    o.mode = 0;
    o.out = part;
    o.ldo = p;
    o.slice = (long long)s * p;
    launch_tc_gemm(XA, ZT, s, p, bnp, L.S, o, err, st, a.stop);
    TcOut r{};
    r.mode = 0;
    r.out = y;
    r.ldo = p;
    launch_tc_reduce(part, L.S, (long long)s * p, p, s, p, r, 0, st, false, a.stop);
    // Q = orth(Y); the last pass also writes the FP64 result and the rank
    const bool last = it == a.iters;
    OrthArgs q{};
    q.Y = y;
    q.ldy = p;
    q.s = s;
    q.p = p;
    q.sact = a.sact;
    q.lact = a.lact;
    q.lact2 = a.lact2;
    q.pmax = p;
    q.qt = last ? nullptr : qt;
    q.kpad = L.ks;
    q.plane = (long long)p * L.ks;
    q.q64 = last ? a.out : nullptr;
    q.ld64 = a.ldo;
    q.q64T = a.outT;
    q.r_out = last ? a.r_out : nullptr;
    q.keep = a.keep;
    q.iters = a.iters;
    q.rho_max = a.rho_max;
    q.accept = last ? a.accept : nullptr;
    q.counts = last ? a.counts : nullptr;
    if (last)
      check_range(a.out, a.outT ? (long long)(p - 1) * a.ldo + s : (long long)(s - 1) * a.ldo + p,
                  sizeof(double), "tc search out");
    q.stop = a.stop;
    // the early test after two power iterations (column norms ~ sigma^2)
    q.early = (a.accept && a.stop && a.iters >= 3 && it == 2) ? 1 : 0;
    if (q.early) {
      q.accept = a.accept;
      q.counts = a.counts;
    }
    const size_t smem = (size_t)s * p * sizeof(float);
    pre_launch(st);
    k_tc_orth<<<1, kOrthThreads, smem, st>>>(q);
    post_launch("k_tc_orth", st);
    if (last) break;
    // Z^T = Q^T X_s  (p x l), K = s, written as TF32 planes for the next Y
    TcOut z{};
    z.mode = 1;
    z.out = zt;
    z.ldo = L.kl;
    z.plane = (long long)p * L.kl;
    launch_tc_gemm(QT, XB, p, l, 128, 1, z, err, st, a.stop);
  }
}

// ------------------------------------------------------------ plain products
// scratch floats needed by qtt_gemm_tf32x3 for these sizes
size_t tc_gemm_scratch_floats(int M, int N, int K, int S) {
  return tc_planes_floats(M, K) + tc_planes_floats(N, K) + (size_t)S * M * N + 192;
}

int tc_gemm_splits(int M, int N, int K) {
  const int tiles = ceil_div(M, kBM) * ceil_div(N, 128);
  const int kb = tc_kpad(K) / kBK;
  return std::max(1, std::min(kb / 4, std::max(1, 128 / tiles)));
}

// C (M x N, FP64) = op(A) op(B): both operands split into TF32 planes
// (A as M x K, B as N x K, K-major), one tensor-core product, split K
// reduced in a fixed order.
void tc_gemm_f64(cudaStream_t s, int M, int N, int K, const double* A, int lda, int tA,
                 const double* B, int ldb, int tB, double* C, int ldc, int* err, float* scratch,
                 size_t scratch_floats) {
  const int S = tc_gemm_splits(M, N, K);
  if (scratch_floats < tc_gemm_scratch_floats(M, N, K, S))
    throw QttError(QTT_ERR_SHAPE, "tc gemm scratch");
  const int kp = tc_kpad(K);
  float* pa = scratch;
  float* pb = pa + ((tc_planes_floats(M, kp) + 63) / 64) * 64;
  float* part = pb + ((tc_planes_floats(N, kp) + 63) / 64) * 64;
  launch_tc_split(A, lda, tA, M, K, pa, kp, (long long)M * kp, s, true);
  // B operand rows are the columns of op(B): element (n, k) = op(B)[k][n]
  launch_tc_split(B, ldb, tB ? 0 : 1, N, K, pb, kp, (long long)N * kp, s, true);
  const TcOperand OA{pa, M, kp, (long long)M * kp}, OB{pb, N, kp, (long long)N * kp};
  const int BN = N >= 128 ? 128 : ((N + 15) / 16) * 16;
  TcOut o{};
  o.mode = 0;
  o.out = part;
  o.ldo = N;
  o.slice = (long long)M * N;
  launch_tc_gemm(OA, OB, M, N, BN, S, o, err, s);
  TcOut r{};
  r.mode = 2;
  r.out64 = C;
  r.ldo = ldc;
  r.alpha = 1.0;
  launch_tc_reduce(part, S, (long long)M * N, N, M, N, r, 0, s, true);
}
