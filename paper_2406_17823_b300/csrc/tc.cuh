// Tensor-core (tcgen05) contractions of the mixed-precision form.
//
// Operands are FP64 matrices of the QTT path, split into two TF32 planes
// (hi = tf32(x), lo = tf32(x - hi)) laid out K-major ([2][rows][kpad],
// kpad a multiple of 32, zero padded), so that every product
// C = A B^T (A: M x K, B: N x K) runs as three TF32 tensor-core products
// hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory (the "3xTF32"
// split; the dropped lo*lo term is below 2^-22 of |A||B|).
#pragma once

#include "common.cuh"

// One split operand: planes [2][rows][kpad] (plane = rows_alloc * kpad).
struct TcOperand {
  const float* p;
  int rows;
  int kpad;
  long long plane;
};

// Size in floats of a split operand with `rows` rows and K = k.
static inline int tc_kpad(int k) { return ((k + 31) / 32) * 32; }
static inline size_t tc_planes_floats(int rows, int k) { return 2 * (size_t)rows * tc_kpad(k); }

// dst planes (rows R, K columns padded to kpad) from the FP64 matrix
// src(r, k) = trans ? src[k * ld + r] : src[r * ld + k], r < R, k < K.
// (src_ext: src is a caller-owned buffer, outside the library's registry)
void launch_tc_split(const double* src, int ld, int trans, int R, int K, float* dst, int kpad,
                     long long plane, cudaStream_t s, bool src_ext = false);

// Output of a tensor-core product C (M x N):
//   mode 0: FP32, out[z * slice + m * ldo + n] (z = split-K slice)
//   mode 1: TF32 planes, out[m * ldo + n] (hi), out[plane + m * ldo + n] (lo)
//   mode 2: FP64, out64[m * ldo + n] = alpha * C
struct TcOut {
  int mode;
  float* out;
  double* out64;
  int ldo;
  long long slice;
  long long plane;
  double alpha;
};
// C = A B^T over K = A.kpad (= B.kpad) with output tiles 128 x BN (BN a
// multiple of 16, 16..256) and K split over S slices (mode 0 when S > 1).
// (stop: a device word; nonzero makes the launch do nothing)
void launch_tc_gemm(const TcOperand& A, const TcOperand& B, int M, int N, int BN, int S,
                    const TcOut& o, int* err, cudaStream_t s, const int* stop = nullptr);
// C = sum of S FP32 slices P[z * slice + m * ldp + n], written as TcOut
// (modes 0..2; `trans` writes C^T, i.e. element (m, n) at n * ldo + m).
// (out_ext: the output is a caller-owned buffer)
void launch_tc_reduce(const float* P, int S, long long slice, int ldp, int M, int N,
                      const TcOut& o, int trans, cudaStream_t s, bool out_ext = false,
                      const int* stop = nullptr);

// Dominant p-dimensional subspace of one side of an FP64 matrix X
// (row-major, capacity shape rows x cols, zeros outside the actual
// extents) by randomised subspace iteration (Halko, Martinsson and Tropp
// 2011, Alg. 4.4): Y = X Omega, then `iters` times Q = orth(Y),
// Y = X (X^T Q), with every product on the tensor cores (3xTF32) and each
// orthonormalisation by classical Gram-Schmidt with reorthogonalisation
// (CGS2) in FP32 on one CTA.  The subspace lives on the "small" side of
// dimension s (<= 256); p <= 128 directions.  Writes the orthonormal basis
// Q (s x p, ldo; or Q^T, p x s, when outT) in FP64 and the rank
// max(1, min(p, sact, lact * lact2)) to *r_out; columns past that rank are
// zero.
struct TcSearch {
  const double* X;
  int ld, rows, cols;
  int small_is_rows;  // the subspace is on the row side (else the column side)
  DimRef sact, lact;  // actual extents of the small and large side
  DimRef lact2;       // second factor of the large side's extent (p null: 1)
  int p;
  int iters;
  unsigned long long key;
  double* out;
  int ldo;
  int outT;
  int* r_out;
  // Acceptance (optional, needs iters >= 1): with the column norms of the
  // last orthonormalisation, which approximate sigma_j^2 in orthogonal
  // iteration, rho = (sigma_rank / sigma_keep)^2 bounds the per-iteration
  // contraction of the kept directions' error; the search is accepted when
  // rho <= rho_max and rho^iters <= 1e-6 (or when the basis spans the whole
  // actual space).  *accept = 1 / 0, counts[0] / counts[1] += 1.
  int keep;
  double rho_max;
  int* accept;
  long long* counts;
  // With iters >= 3 the test also runs after two power iterations and, if
  // rho^iters would miss the bar, stops the search there (*stop = 1: its
  // remaining launches do nothing; *accept = 0).  *stop is reset when a
  // search starts.  May be null (no early test).
  int* stop;
};
bool tc_search_supported(int s, int l, int p);
size_t tc_search_scratch_floats(int s, int l, int p);
void tc_search(const TcSearch& a, float* scratch, size_t scratch_floats, int* err, cudaStream_t st);

// C (M x N, FP64, ldc) = op(A) op(B) on the tensor cores (3xTF32, FP32
// accumulation), op(A) = A (M x K, lda) or A^T (tA), op(B) = B (K x N, ldb)
// or B^T (tB); K split over slices reduced in a fixed order.  Scratch of
// tc_gemm_scratch_floats(M, N, K, tc_gemm_splits(M, N, K)) floats.
int tc_gemm_splits(int M, int N, int K);
size_t tc_gemm_scratch_floats(int M, int N, int K, int S);
void tc_gemm_f64(cudaStream_t s, int M, int N, int K, const double* A, int lda, int tA,
                 const double* B, int ldb, int tB, double* C, int ldc, int* err, float* scratch,
                 size_t scratch_floats);
