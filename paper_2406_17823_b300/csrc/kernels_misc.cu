// Data-movement kernels of the QTT path: MPO x MPS site expansion
// (Sec. II.B), block-diagonal MPS sums (Sec. II.C), core transposes,
// dense <-> quantics reordering (Sec. II.B), and the CG vector updates
// of the local solves (App. B).  The CG updates run in one CTA: the local
// vectors are at most a few 10^4 doubles, and a single CTA gives a fixed,
// reproducible summation order.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

thread_local int* g_dev_err = nullptr;  // error flag of the context issuing the launch

namespace {

__global__ void k_scale(double* C, int M, int N, int ldc, double beta) {
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    C[(long long)i * ldc + j] *= beta;
  }
}

// out[(a,p), so, (b,q)] = sum_si W[p, so, si, q] * A[a, si, b]
__global__ void k_mpo_expand(const double* __restrict__ W, int wl, int wr,
                             const double* __restrict__ A, int Ca, int Cb, double* out) {
  const long long tot = (long long)Ca * wl * 4 * Cb * wr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long t = e;
    const int q = (int)(t % wr); t /= wr;
    const int b = (int)(t % Cb); t /= Cb;
    const int so = (int)(t % 4); t /= 4;
    const int p = (int)(t % wl); t /= wl;
    const int a = (int)t;
    double acc = 0.0;
#pragma unroll
    for (int si = 0; si < 4; si++) {
      const double w = W[((p * 4 + so) * 4 + si) * wr + q];
      if (w != 0.0) acc = fma(w, A[((long long)a * 4 + si) * Cb + b], acc);
    }
    out[e] = acc;
  }
}

struct AddArgs {
  AddTerm t[8];
  int K;
  int first, last;
  double* out;
  int capl, capr;
};

__global__ void k_add_assemble(AddArgs g, int* err) {
  int loff[9], roff[9];
  loff[0] = roff[0] = 0;
  for (int t = 0; t < g.K; t++) {
    // shape guard: actual extents must fit the term's capacities
    if (*g.t[t].dl > g.t[t].capl || *g.t[t].dr > g.t[t].capr) {
      if (blockIdx.x == 0 && threadIdx.x == 0 && err) atomicOr(err, QTT_DEVERR_SHAPE);
      return;
    }
    loff[t + 1] = loff[t] + (g.first ? 0 : *g.t[t].dl);
    roff[t + 1] = roff[t] + (g.last ? 0 : *g.t[t].dr);
  }
  const long long tot = (long long)g.capl * 4 * g.capr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % g.capr);
    const int s = (int)((e / g.capr) % 4);
    const int i = (int)(e / ((long long)g.capr * 4));
    double v = 0.0;
    for (int t = 0; t < g.K; t++) {
      const int dl = *g.t[t].dl, dr = *g.t[t].dr;
      const int ii = g.first ? i : i - loff[t];
      const int jj = g.last ? j : j - roff[t];
      if (ii >= 0 && ii < dl && jj >= 0 && jj < dr) {
        const double x = g.t[t].core[((long long)ii * 4 + s) * g.t[t].capr + jj];
        if (g.first && g.last) v += g.t[t].coef * x;
        else if (g.first) v = g.t[t].coef * x;
        else v = x;
        if (!(g.first && g.last)) break;
      }
    }
    g.out[e] = v;
  }
}

__global__ void k_core_transpose(const double* __restrict__ in, int Ca, int Cb, double* out) {
  const long long tot = (long long)Ca * 4 * Cb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e % Ca);
    const int s = (int)((e / Ca) % 4);
    const int b = (int)(e / ((long long)Ca * 4));
    out[e] = in[((long long)a * 4 + s) * Cb + b];  // out[b][s][a]
  }
}

struct DimsArgs {
  const int* src[8];
  int mul[8][QTT_MAX_N + 1];
  int K;
  int nb;  // bonds 0..nb-1
  int* out;
};

__global__ void k_dims(DimsArgs g) {
  const int b = threadIdx.x;
  if (b >= g.nb) return;
  int v = 0;
  for (int t = 0; t < g.K; t++) v += g.src[t][b] * g.mul[t][b];
  if (b == 0 || b == g.nb - 1) v = 1;
  g.out[b] = v;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

__global__ void k_fill_int(int* p, int n, int v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = v;
}

__device__ __forceinline__ long long omega_index(int x1, int x2, int n) {
  long long idx = 0;
  for (int k = 0; k < n; k++) {
    const int b1 = (x1 >> (n - 1 - k)) & 1, b2 = (x2 >> (n - 1 - k)) & 1;
    idx = idx * 4 + (2 * b1 + b2);
  }
  return idx;
}

__global__ void k_dense_to_omega(const double* F, double* T, int n) {
  const long long N = 1LL << n, tot = N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    T[omega_index((int)(e / N), (int)(e % N), n)] = F[e];
}

__global__ void k_omega_to_dense(const double* T, double* F, int n) {
  const long long N = 1LL << n, tot = N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    F[e] = T[omega_index((int)(e / N), (int)(e % N), n)];
}

__device__ double cta_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; i++) t += sh[i];
  return t;
}

__global__ void k_check_finite(const double* p, size_t n, int* err) {
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(p[e])) bad = true;
  if (bad) atomicOr(err, QTT_DEVERR_NUMERIC);
}

// scal: [0] rs, [1] bb, [2] tol^2 * bb ; ist: [0] done, [1] iters
__global__ void __launch_bounds__(1024) k_cg_start(CgVec v, const double* b0, const double* b1,
                                                    double* scal, int* ist, double tol, int* err) {
  __shared__ double sh[32];
  double rr = 0.0, bb = 0.0;
  for (int sgm = 0; sgm < 2; sgm++) {
    const double* b = sgm ? b1 : b0;
    for (long long e = threadIdx.x; e < v.len[sgm]; e += blockDim.x) {
      const double be = b[e];
      const double re = be - v.ap[sgm][e];
      v.r[sgm][e] = re;
      v.p[sgm][e] = re;
      rr += re * re;
      bb += be * be;
    }
  }
  rr = cta_sum(rr, sh);
  bb = cta_sum(bb, sh);
  if (bb == 0.0) {
    for (int sgm = 0; sgm < 2; sgm++)
      for (long long e = threadIdx.x; e < v.len[sgm]; e += blockDim.x)
        v.x[sgm][e] = v.r[sgm][e] = v.p[sgm][e] = 0.0;
  }
  if (threadIdx.x == 0) {
    if (!isfinite(rr) || !isfinite(bb)) atomicOr(err, QTT_DEVERR_NUMERIC);
    scal[0] = rr;
    scal[1] = bb;
    scal[2] = tol * tol * bb;
    ist[0] = (bb == 0.0 || rr <= tol * tol * bb || !isfinite(rr)) ? 1 : 0;
    ist[1] = 0;
  }
}

// One CG iteration after ap = A p (App. B: the local system is solved by CG).
__global__ void __launch_bounds__(1024) k_cg_step(CgVec v, double* scal, int* ist, int maxit,
                                                   int* err) {
  __shared__ double sh[32];
  if (ist[0]) return;
  double pap = 0.0;
  for (int sgm = 0; sgm < 2; sgm++)
    for (long long e = threadIdx.x; e < v.len[sgm]; e += blockDim.x) pap += v.p[sgm][e] * v.ap[sgm][e];
  pap = cta_sum(pap, sh);
  const double rs = scal[0];
  if (!(pap > 0.0) || !isfinite(pap)) {
    __syncthreads();
    if (threadIdx.x == 0) {
      ist[0] = 1;
      if (!isfinite(pap)) atomicOr(err, QTT_DEVERR_NUMERIC);
    }
    return;
  }
  const double alpha = rs / pap;
  double rr = 0.0;
  for (int sgm = 0; sgm < 2; sgm++)
    for (long long e = threadIdx.x; e < v.len[sgm]; e += blockDim.x) {
      v.x[sgm][e] = fma(alpha, v.p[sgm][e], v.x[sgm][e]);
      const double re = fma(-alpha, v.ap[sgm][e], v.r[sgm][e]);
      v.r[sgm][e] = re;
      rr += re * re;
    }
  rr = cta_sum(rr, sh);
  const double beta = rr / rs;
  for (int sgm = 0; sgm < 2; sgm++)
    for (long long e = threadIdx.x; e < v.len[sgm]; e += blockDim.x)
      v.p[sgm][e] = fma(beta, v.p[sgm][e], v.r[sgm][e]);
  __syncthreads();
  if (threadIdx.x == 0) {
    scal[0] = rr;
    const int it = ist[1] + 1;
    ist[1] = it;
    if (rr <= scal[2] || it >= maxit || !isfinite(rr)) ist[0] = 1;
    if (!isfinite(rr)) atomicOr(err, QTT_DEVERR_NUMERIC);
  }
}

// C = alpha * (sum over S slices of P) + beta * C (slice z at P + z * M * N,
// row-major M x N), the slices added in order (deterministic); C has ld ldc
// and is not read when beta == 0.
__global__ void k_sum_slices(const double* P, int S, int M, int N, double* C, int ldc,
                             double alpha, double beta, const int* skip) {
  if (skip && *skip) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const int i = (int)(e / N), j = (int)(e % N);
  double v = 0.0;
  for (int z = 0; z < S; z++) v += P[(long long)z * M * N + e];
  double* c = C + (long long)i * ldc + j;
  *c = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *c);
}

__global__ void __launch_bounds__(1024) k_sumsq2(const double* a, long long na, const double* b,
                                                  long long nb, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long e = threadIdx.x; e < na; e += blockDim.x) s += a[e] * a[e];
  for (long long e = threadIdx.x; e < nb; e += blockDim.x) s += b[e] * b[e];
  s = cta_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_fill(double* p, size_t n, double v) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    p[e] = v;
}

int grid_for(long long tot) {
  long long g = (tot + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_scale(const GemmF64& g, cudaStream_t s) {
  if (g.beta == 1.0) return;
  for (int z = 0; z < g.nb1 * g.nb2; z++) {
    const int z1 = z / g.nb2, z2 = z % g.nb2;
    pre_launch(s);
    k_scale<<<grid_for((long long)g.M * g.N), 256, 0, s>>>(g.C + z1 * g.sC1 + z2 * g.sC2, g.M, g.N,
                                                           g.ldc, g.beta);
    post_launch("k_scale", s);
  }
}

void launch_zero(double* p, size_t n, cudaStream_t s) {
  if (n) QTT_CUDA_CHECK(cudaMemsetAsync(p, 0, n * sizeof(double), s));
}
void launch_copy(double* dst, const double* src, size_t n, cudaStream_t s) {
  check_range(dst, (long long)n, sizeof(double), "copy dst");
  check_range(src, (long long)n, sizeof(double), "copy src");
  if (n) QTT_CUDA_CHECK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
}
void launch_fill(double* p, size_t n, double v, cudaStream_t s) {
  check_range(p, (long long)n, sizeof(double), "fill");
  pre_launch(s);
  k_fill<<<grid_for((long long)n), 256, 0, s>>>(p, n, v);
  post_launch("k_fill", s);
}

void launch_mpo_expand(const double* W, int wl, int wr, const double* A, int Ca, int Cb,
                       double* out, cudaStream_t s) {
  const long long tot = (long long)Ca * wl * 4 * Cb * wr;
  check_range(W, (long long)wl * 16 * wr, sizeof(double), "expand W");
  check_range(A, (long long)Ca * 4 * Cb, sizeof(double), "expand A");
  check_range(out, tot, sizeof(double), "expand out");
  pre_launch(s);
  k_mpo_expand<<<grid_for(tot), 256, 0, s>>>(W, wl, wr, A, Ca, Cb, out);
  post_launch("k_mpo_expand", s);
}

void launch_add_assemble_args(const AddTerm* terms, int K, int first, int last, double* out,
                              int capl, int capr, cudaStream_t s) {
  AddArgs g{};
  if (K < 1 || K > 8) throw QttError(QTT_ERR_ARG, "add: 1..8 terms");
  check_range(out, (long long)capl * 4 * capr, sizeof(double), "add out");
  for (int t = 0; t < K; t++) {
    g.t[t] = terms[t];
    check_range(terms[t].core, (long long)terms[t].capl * 4 * terms[t].capr, sizeof(double),
                "add term");
  }
  g.K = K;
  g.first = first;
  g.last = last;
  g.out = out;
  g.capl = capl;
  g.capr = capr;
  pre_launch(s);
  k_add_assemble<<<grid_for((long long)capl * 4 * capr), 256, 0, s>>>(g, g_dev_err);
  post_launch("k_add_assemble", s);
}

void launch_add_assemble(const AddTerm* terms, int K, int first, int last, double* out,
                         int capl_out, int capr_out, cudaStream_t s) {
  launch_add_assemble_args(terms, K, first, last, out, capl_out, capr_out, s);
}

// Core of the MPO product of a Hadamard MPO and an MPO (the paper's
// "nonlinear MPOs"): H_B[c][s][t][c'] = B[c][s][c'] delta(s, t), so
//   order 0: P = H_B W,  P[(c p)][s][t][(c' q)] = B[c][s][c'] W[p][s][t][q]
//   order 1: P = W H_B,  P[(c p)][s][t][(c' q)] = B[c][t][c'] W[p][s][t][q]
// written in the three layouts of an MPO: raw [P][s][t][Q], k2 [(s Q)][(P t)]
// and kr2 [(s P)][(Q t)] with P = c wl + p, Q = c' wr + q (capacities).
__global__ void k_hadamard_mpo(const double* __restrict__ B, int cbl, int cbr,
                               const double* __restrict__ W, int wl, int wr, int order,
                               double* __restrict__ raw, double* __restrict__ k2,
                               double* __restrict__ kr2) {
  const int PL = cbl * wl, PR = cbr * wr;
  const long long tot = (long long)PL * 16 * PR;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long t = e;
    const int Q = (int)(t % PR); t /= PR;
    const int si = (int)(t % 4); t /= 4;
    const int so = (int)(t % 4); t /= 4;
    const int P = (int)t;
    const int c = P / wl, p = P % wl, c1 = Q / wr, q = Q % wr;
    const int x = order == 0 ? so : si;
    const double v = B[((long long)c * 4 + x) * cbr + c1] * W[((p * 4 + so) * 4 + si) * wr + q];
    raw[e] = v;
    k2[(long long)(so * PR + Q) * (PL * 4) + (P * 4 + si)] = v;
    kr2[(long long)(so * PL + P) * (PR * 4) + (Q * 4 + si)] = v;
  }
}

void launch_hadamard_mpo(const double* B, int cbl, int cbr, const double* W, int wl, int wr,
                         int order, double* raw, double* k2, double* kr2, cudaStream_t s) {
  const long long tot = (long long)cbl * wl * 16 * cbr * wr;
  check_range(B, (long long)cbl * 4 * cbr, sizeof(double), "hadamard mpo B");
  check_range(W, (long long)wl * 16 * wr, sizeof(double), "hadamard mpo W");
  check_range(raw, tot, sizeof(double), "hadamard mpo raw");
  check_range(k2, tot, sizeof(double), "hadamard mpo k2");
  check_range(kr2, tot, sizeof(double), "hadamard mpo kr2");
  pre_launch(s);
  k_hadamard_mpo<<<grid_for(tot), 256, 0, s>>>(B, cbl, cbr, W, wl, wr, order, raw, k2, kr2);
  post_launch("k_hadamard_mpo", s);
}

void launch_core_transpose(const double* in, int Ca, int Cb, double* out, cudaStream_t s) {
  check_range(in, (long long)Ca * 4 * Cb, sizeof(double), "transpose in");
  check_range(out, (long long)Ca * 4 * Cb, sizeof(double), "transpose out");
  pre_launch(s);
  k_core_transpose<<<grid_for((long long)Ca * 4 * Cb), 256, 0, s>>>(in, Ca, Cb, out);
  post_launch("k_core_transpose", s);
}

__global__ void k_sparse_rows(const double* __restrict__ B, int ldb, long long sB,
                              double* __restrict__ C, int ldc, long long sC, int N,
                              long long total, const __grid_constant__ SparseRows sp) {
  const long long per = (long long)sp.rows * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long z = e / per;
    const int rem = (int)(e - z * per);
    const int r = rem / N, j = rem - r * N;
    const double* Bz = B + z * sB + j;
    double acc = 0.0;
    for (int q = sp.ptr[r]; q < sp.ptr[r + 1]; q++) acc = fma(sp.val[q], Bz[(long long)sp.col[q] * ldb], acc);
    C[z * sC + (long long)r * ldc + j] = acc;
  }
}

void launch_sparse_rows(const SparseRows& sp, const double* B, int ldb, long long sB, double* C,
                        int ldc, long long sC, int N, int nb, cudaStream_t s) {
  if (sp.nnz < 0 || sp.rows < 1 || sp.rows > kSparseMaxRows || sp.cols < 1 || N < 1 || nb < 1 ||
      ldb < N || ldc < N)
    throw QttError(QTT_ERR_SHAPE, "sparse-row product shape");
  check_range(B, (long long)(nb - 1) * sB + (long long)(sp.cols - 1) * ldb + N, sizeof(double),
              "sparse rows B");
  check_range(C, (long long)(nb - 1) * sC + (long long)(sp.rows - 1) * ldc + N, sizeof(double),
              "sparse rows C");
  const long long total = (long long)nb * sp.rows * N;
  const int blocks = grid_for(total);
  pre_launch(s);
  k_sparse_rows<<<blocks, 256, 0, s>>>(B, ldb, sB, C, ldc, sC, N, total, sp);
  post_launch("k_sparse_rows", s, 2.0 * (double)nb * N * (sp.nnz > 0 ? sp.nnz : 0));
}

void launch_set_int(int* p, int v, cudaStream_t s) {
  pre_launch(s);
  k_set_int<<<1, 1, 0, s>>>(p, v);
  post_launch("k_set_int", s);
}

void launch_fill_int(int* p, int n, int v, cudaStream_t s) {
  pre_launch(s);
  k_fill_int<<<1, 64, 0, s>>>(p, n, v);
  post_launch("k_fill_int", s);
}

void launch_dims(const int* const* src, const int (*mul)[QTT_MAX_N + 1], int K, int nb, int* out,
                 cudaStream_t s) {
  DimsArgs g{};
  for (int t = 0; t < K; t++) {
    g.src[t] = src[t];
    for (int b = 0; b < nb; b++) g.mul[t][b] = mul[t][b];
  }
  g.K = K;
  g.nb = nb;
  g.out = out;
  pre_launch(s);
  k_dims<<<1, 32, 0, s>>>(g);
  post_launch("k_dims", s);
}

void launch_dense_to_omega(const double* F, double* T, int n, cudaStream_t s) {
  check_range(T, 1LL << (2 * n), sizeof(double), "omega out");
  pre_launch(s);
  k_dense_to_omega<<<grid_for(1LL << (2 * n)), 256, 0, s>>>(F, T, n);
  post_launch("k_dense_to_omega", s);
}
void launch_omega_to_dense(const double* T, double* F, int n, cudaStream_t s) {
  check_range(T, 1LL << (2 * n), sizeof(double), "omega in");
  pre_launch(s);
  k_omega_to_dense<<<grid_for(1LL << (2 * n)), 256, 0, s>>>(T, F, n);
  post_launch("k_omega_to_dense", s);
}

void launch_check_finite(const double* p, size_t n, int* err, cudaStream_t s) {
  pre_launch(s);
  k_check_finite<<<grid_for((long long)n), 256, 0, s>>>(p, n, err);
  post_launch("k_check_finite", s);
}

static void check_cg(const CgVec& v) {
  for (int i = 0; i < 2; i++) {
    check_range(v.x[i], v.len[i], sizeof(double), "cg x");
    check_range(v.r[i], v.len[i], sizeof(double), "cg r");
    check_range(v.p[i], v.len[i], sizeof(double), "cg p");
    check_range(v.ap[i], v.len[i], sizeof(double), "cg ap");
  }
}

void launch_cg_start(const CgVec& v, const double* b0, const double* b1, double* scal, int* ist,
                     double tol, int* err, cudaStream_t s) {
  check_cg(v);
  check_range(b0, v.len[0], sizeof(double), "cg b0");
  check_range(b1, v.len[1], sizeof(double), "cg b1");
  pre_launch(s);
  k_cg_start<<<1, 1024, 0, s>>>(v, b0, b1, scal, ist, tol, err);
  post_launch("k_cg_start", s);
}
void launch_cg_step(const CgVec& v, double* scal, int* ist, int maxit, int* err, cudaStream_t s) {
  check_cg(v);
  pre_launch(s);
  k_cg_step<<<1, 1024, 0, s>>>(v, scal, ist, maxit, err);
  post_launch("k_cg_step", s);
}
// ---- device-driven loops of a captured step (WHILE graph nodes)
// The loop condition of a WHILE node: iteration `counter` (0 on the first
// call) continues while counter < cap and *stop == 0.  The counter makes
// every loop end after at most cap iterations whatever the stop word holds.
// At the end of each pass (first == 0) `body_launches` kernels of the body
// have run; they are added to *launched (the step's launch count).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int* counter, const int* stop, int cap,
                            int first, long long body_launches, long long* launched) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int c = first ? 0 : *counter + 1;
  *counter = c;
  if (!first && launched) *launched += body_launches;
  cudaGraphSetConditional(h, (c < cap && !(stop && *stop)) ? 1u : 0u);
}
void launch_loop_cond(cudaGraphConditionalHandle h, int* counter, const int* stop, int cap,
                      int first, cudaStream_t s, long long body_launches, long long* launched) {
  pre_launch(s);
  k_loop_cond<<<1, 32, 0, s>>>(h, counter, stop, cap, first, body_launches, launched);
  post_launch("k_loop_cond", s);
}

// After a device-driven CG solve: stats[0] += iterations; a solve that hit
// the iteration cap marks the step not converged (stats[2]).
__global__ void k_cg_account(const int* ist, long long* stats, int maxit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  stats[0] += ist[1];
  if (ist[1] >= maxit) stats[2] = 1;
}
void launch_cg_account(const int* ist, long long* stats, int maxit, cudaStream_t s) {
  pre_launch(s);
  k_cg_account<<<1, 32, 0, s>>>(ist, stats, maxit);
  post_launch("k_cg_account", s);
}

// Sweep convergence on the device, the host rule restated: with N = scal[6]
// (sum of <v_i|v_i> after the sweep) and N_prev = scal[7], stop when N == 0
// or |N - N_prev| <= tol N; N_prev <- N; stats[1] counts sweeps.  init: only
// N_prev <- N and stop <- 0 (before the first sweep).
__global__ void k_sweep_check(double* scal, int* stop, long long* stats, double tol, int init) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double nn = scal[6];
  if (!init) {
    const double np = scal[7];
    *stop = (nn == 0.0 || fabs(nn - np) <= tol * nn) ? 1 : 0;
    stats[1] += 1;
  } else {
    *stop = 0;
  }
  scal[7] = nn;
}
void launch_sweep_check(double* scal, int* stop, long long* stats, double tol, int init,
                        cudaStream_t s) {
  pre_launch(s);
  k_sweep_check<<<1, 32, 0, s>>>(scal, stop, stats, tol, init);
  post_launch("k_sweep_check", s);
}
// After the sweep loop: a loop that ended without the stop word set ran into
// its cap (stats[2] = 1).
__global__ void k_sweep_final(const int* stop, long long* stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!*stop) stats[2] = 1;
}
void launch_sweep_final(const int* stop, long long* stats, cudaStream_t s) {
  pre_launch(s);
  k_sweep_final<<<1, 32, 0, s>>>(stop, stats);
  post_launch("k_sweep_final", s);
}

void launch_sum_slices(const double* P, int S, int M, int N, double* C, int ldc, double alpha,
                       double beta, const int* skip, cudaStream_t s, bool c_ext) {
  if (M <= 0 || N <= 0 || S <= 0) return;
  check_range(P, (long long)S * M * N, sizeof(double), "sum_slices P");
  check_range(C, (long long)(M - 1) * ldc + N, sizeof(double),
              c_ext ? "ext sum_slices C" : "sum_slices C");
  const long long tot = (long long)M * N;
  pre_launch(s);
  k_sum_slices<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, S, M, N, C, ldc, alpha, beta,
                                                                skip);
  post_launch("k_sum_slices", s);
}

void launch_sumsq2(const double* a, long long na, const double* b, long long nb, double* out,
                   cudaStream_t s) {
  check_range(a, na, sizeof(double), "sumsq a");
  check_range(b, nb, sizeof(double), "sumsq b");
  pre_launch(s);
  k_sumsq2<<<1, 1024, 0, s>>>(a, na, b, nb, out);
  post_launch("k_sumsq2", s);
}
