// Batched FP64 GEMM used for every dense contraction of the FP64 path:
// C[z] = alpha * op(A[z]) * op(B[z]) + beta * C[z], row-major operands,
// op = optional transpose, batch z = z1 * nb2 + z2 with two stride levels
// (the site contractions of the zip-up batch over (carry row, omega)).
//
// Tiling: 64 x 64 (256 threads), 32 x 32 (64 threads) or 16 x 128 (128
// threads, for outputs of a few rows) output tile per CTA, or (tile 3) a
// small op(A) in shared memory with one output column per thread,
// K staged 16 at a time in shared memory, 4 x 4 register accumulators per
// thread; the host picks the tile and a split of K per product shape.  FP64 on this GPU
// runs on the CUDA-core DFMA pipe (no FP64 tensor-core rate worth using), so
// the kernel is DFMA-bound once tiles are full.
#include <stdio.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int BK = 16;

// TBM x TBN output tile per CTA of (TBM / 4) * (TBN / 4) threads, 4 x 4
// accumulators per thread: 64 x 64 (256 threads) for large outputs, 32 x 32
// (64 threads) to spread small outputs over more SMs.
template <int TBM, int TBN>
__global__ void __launch_bounds__((TBM / 4) * (TBN / 4)) k_gemm_f64(GemmF64 g) {
  constexpr int TX = TBN / 4, TY = TBM / 4, NT = TX * TY;
  if (g.skip && *g.skip) return;
  const int z = blockIdx.z;
  const int z1 = z / g.nb2, z2 = z % g.nb2;
  const double* A = g.A + z1 * g.sA1 + z2 * g.sA2;
  const double* B = g.B + z1 * g.sB1 + z2 * g.sB2;
  double* C = g.C + z1 * g.sC1 + z2 * g.sC2;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  __shared__ double As[BK][TBM + 1];
  __shared__ double Bs[BK][TBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int idx = tid; idx < BK * TBM; idx += NT) {
      int mm, kk;
      if (!g.tA) { mm = idx / BK; kk = idx % BK; } else { kk = idx / TBM; mm = idx % TBM; }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < g.M && gk < g.K) v = g.tA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[kk][mm] = v;
    }
    for (int idx = tid; idx < BK * TBN; idx += NT) {
      int nn, kk;
      if (!g.tB) { kk = idx / TBN; nn = idx % TBN; } else { nn = idx / BK; kk = idx % BK; }
      const int gn = n0 + nn, gk = k0 + kk;
      double w = 0.0;
      if (gn < g.N && gk < g.K) w = g.tB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
      Bs[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + TY * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = m0 + ty + TY * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gn = n0 + tx + TX * j;
      if (gn >= g.N) continue;
      double* c = C + (long long)gm * g.ldc + gn;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
  }
}

// Small-operand products over a large batch (an MPO core applied to every
// slice of a tensor, a few rows by a few columns of K): op(A[z]) (M x K,
// M <= MM, K <= kSmallK) staged in shared memory, one thread per output
// column n of one batch entry z, the M rows of that column in registers.
// Each output is the same chain of fused multiply-adds over k = 0..K-1 as in
// k_gemm_f64, so the two kernels give the same bits.
constexpr int kSmallK = 48;

template <int MM>
__global__ void __launch_bounds__(128) k_gemm_f64_small(GemmF64 g) {
  if (g.skip && *g.skip) return;
  __shared__ double As[MM * kSmallK];
  const int M = g.M, K = g.K, N = g.N;
  const int z = blockIdx.y;
  const int z1 = z / g.nb2, z2 = z % g.nb2;
  const double* A = g.A + z1 * g.sA1 + z2 * g.sA2;
  for (int e = threadIdx.x; e < M * K; e += blockDim.x) {
    const int i = e / K, k = e % K;
    As[e] = g.tA ? A[(long long)k * g.lda + i] : A[(long long)i * g.lda + k];
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* B = g.B + z1 * g.sB1 + z2 * g.sB2 + n;
  double* C = g.C + z1 * g.sC1 + z2 * g.sC2 + n;
  double acc[MM];
#pragma unroll
  for (int i = 0; i < MM; i++) acc[i] = 0.0;
  for (int k = 0; k < K; k++) {
    const double b = B[(long long)k * g.ldb];
#pragma unroll
    for (int i = 0; i < MM; i++)
      if (i < M) acc[i] = fma(As[i * K + k], b, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < MM; i++) {
    if (i >= M) break;
    double* c = C + (long long)i * g.ldc;
    double v = g.alpha * acc[i];
    if (g.beta != 0.0) v = fma(g.beta, *c, v);
    *c = v;
  }
}

}  // namespace

bool gemm_small_eligible(const GemmF64& g) {
  return !g.tB && g.M <= 48 && g.K <= kSmallK && g.nb1 * g.nb2 <= 65535;
}

void launch_gemm_f64(const GemmF64& g, cudaStream_t s) { launch_gemm_f64_tile(g, 0, s); }

void launch_gemm_f64_tile(const GemmF64& g, int tile, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nb1 * g.nb2 <= 0) return;
  {
    const long long zb1 = g.nb1 - 1, zb2 = g.nb2 - 1;
    const long long ea = g.tA ? (long long)(g.K - 1) * g.lda + g.M : (long long)(g.M - 1) * g.lda + g.K;
    const long long eb = g.tB ? (long long)(g.N - 1) * g.ldb + g.K : (long long)(g.K - 1) * g.ldb + g.N;
    const long long ec = (long long)(g.M - 1) * g.ldc + g.N;
    check_range(g.A, zb1 * g.sA1 + zb2 * g.sA2 + ea, sizeof(double), "gemm A");
    check_range(g.B, zb1 * g.sB1 + zb2 * g.sB2 + eb, sizeof(double), "gemm B");
    check_range(g.C, zb1 * g.sC1 + zb2 * g.sC2 + ec, sizeof(double), "gemm C");
  }
  if (g.K <= 0) {
    // C = beta * C (alpha * empty product)
    launch_scale(g, s);
    return;
  }
  if (tile == 3 && !gemm_small_eligible(g)) tile = 0;
  pre_launch(s);
  if (tile == 1) {
    dim3 grid(ceil_div(g.N, 32), ceil_div(g.M, 32), g.nb1 * g.nb2);
    k_gemm_f64<32, 32><<<grid, 64, 0, s>>>(g);
  } else if (tile == 3) {
    const int th = g.N >= 128 ? 128 : ((g.N + 31) / 32) * 32;
    dim3 grid(ceil_div(g.N, th), g.nb1 * g.nb2);
    if (g.M <= 16)
      k_gemm_f64_small<16><<<grid, th, 0, s>>>(g);
    else
      k_gemm_f64_small<48><<<grid, th, 0, s>>>(g);
  } else if (tile == 2) {
    // skinny outputs (a few rows, e.g. an MPO core applied over a batch)
    dim3 grid(ceil_div(g.N, 128), ceil_div(g.M, 16), g.nb1 * g.nb2);
    k_gemm_f64<16, 128><<<grid, 128, 0, s>>>(g);
  } else {
    dim3 grid(ceil_div(g.N, 64), ceil_div(g.M, 64), g.nb1 * g.nb2);
    k_gemm_f64<64, 64><<<grid, 256, 0, s>>>(g);
  }
  const char* name = "k_gemm_f64";
  if (shape_profiling()) {
    char tag[80];
    snprintf(tag, sizeof tag, "%dx%dx%d b%d t%d %d%d", g.M, g.N, g.K, g.nb1 * g.nb2, tile, g.tA,
             g.tB);
    name = shape_name(name, tag);
  }
  post_launch(name, s, 2.0 * g.M * g.N * (double)g.K * g.nb1 * g.nb2);
}
