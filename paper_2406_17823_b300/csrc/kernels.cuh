// Kernel argument structs and launchers (host-callable), FP64 path.
#pragma once

#include "common.cuh"

// ---------------------------------------------------------------- GEMM
struct GemmF64 {
  const double* A;
  const double* B;
  double* C;
  int M, N, K;
  int lda, ldb, ldc;
  long long sA1, sA2, sB1, sB2, sC1, sC2;  // batch strides, z = z1 * nb2 + z2
  int nb1, nb2;
  int tA, tB;  // op(A) = A^T when tA (A stored K x M), likewise B
  double alpha, beta;
  const int* skip;  // if non-null and *skip != 0 the launch does nothing
};
static inline GemmF64 gemm_plain(const double* A, const double* B, double* C, int M, int N,
                                 int K, int lda, int ldb, int ldc) {
  GemmF64 g{};
  g.A = A; g.B = B; g.C = C;
  g.M = M; g.N = N; g.K = K;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.nb1 = 1; g.nb2 = 1;
  g.alpha = 1.0; g.beta = 0.0;
  return g;
}
void launch_gemm_f64(const GemmF64& g, cudaStream_t s);
// tile 0: 64 x 64 per CTA, tile 1: 32 x 32 per CTA, tile 2: 16 x 128 per CTA,
// tile 3: op(A) in shared memory, one output column per thread (for
// gemm_small_eligible shapes; others run tile 0).  All tiles give the same bits.
void launch_gemm_f64_tile(const GemmF64& g, int tile, cudaStream_t s);
bool gemm_small_eligible(const GemmF64& g);  // M <= 48, K <= 48, B not transposed
// The mixed form's FP64 product on the BF16 tensor cores (Ozaki splitting,
// gemm_oz.cu): same GemmF64 semantics, FP64-level accuracy, different
// rounding from launch_gemm_f64.  Eligible shapes: K >= 16, at most 65535
// batch entries, max(M, N) >= 32, at least 2^21 multiply-adds, and
// K <= 1024 (batched) or K <= 16384 (unbatched).  An unbatched product
// whose output tiles cannot fill the GPU is split over gemm_oz_splits(g)
// K slices: `scratch` must then hold that many M x N partial products
// (summed in slice order into C).
bool gemm_oz_eligible(const GemmF64& g);
bool gemm_oz_dispatch(const GemmF64& g);
// max_s: the most K slices the plan may take (16, and always 16 for the
// public entry point; the library's own products up to 64 when their
// scratch holds that many partial products).
int gemm_oz_splits(const GemmF64& g, int max_s = 16);
constexpr long long kOzWideSplitMN = 1 << 16;  // outputs that may take up to 64 slices
void launch_gemm_oz(const GemmF64& g, int* err, cudaStream_t s, bool ext = false,
                    double* scratch = nullptr, size_t scratch_n = 0, int max_s = 16);
void launch_scale(const GemmF64& g, cudaStream_t s);  // C = beta C
void launch_sum_slices(const double* P, int S, int M, int N, double* C, int ldc, double alpha,
                       double beta, const int* skip, cudaStream_t s, bool c_ext = false);

// ---------------------------------------------------------------- QR
// Householder QR of F = A (or A^T when inT): F = Q R, Q (m x r) with
// orthonormal columns, R (r x c) upper triangular, r = min(m, c).
struct QrArgs {
  MatView A;
  int inT;
  MatView Q;   // m x r  (or r x m when qT)
  int qT;
  MatView R;   // r x c  (or c x r when rT)
  int rT;
  int* r_out;  // receives r (may be null)
  double* work;
  long long work_len;  // doubles available at work
  const int* skip;
  int* err;
};
size_t qr_work_doubles(int mcap, int ccap);
void launch_qr_f64(const QrArgs& a, int mcap, int ccap, cudaStream_t s);

// ---------------------------------------------------------------- SVD
// SVD of M (m x N): Householder QR of the tall orientation, one-sided
// Jacobi on the square factor, descending order, rank by the truncation
// rule (eps >= 0) or by the cap alone (eps < 0).  Writes U*S (m x r) and
// V^T (r x N) of F = M (or M^T when inT), each optionally transposed.
struct SvdArgs {
  MatView M;
  int inT;     // factor M^T instead of M
  MatView US;
  int usT;     // write (U S)^T
  MatView VT;
  int vtT;     // write (V^T)^T
  double eps;
  int chi;
  DimRef rank_limit;
  int* r_out;
  double* sv_out;   // optional, receives the c singular values
  // optional: the squared Frobenius norm of a larger matrix of which M is
  // a projection; the weight M lacks counts as discarded in the eps rule
  const double* total_weight;
  double* work;
  long long work_len;  // doubles available at work
  const int* skip;
  int* err;
  int no_us;  // US is not wanted (cluster kernels skip the work only it needs)
  int gram;   // M is a Gram matrix B^T B: its singular values are the weights
};
size_t svd_work_doubles(int mcap, int ncap);
// FLOPs performed by the cluster SVDs since the last reset ([0] FP64, [1] FP32)
void svd_work_reset();
void svd_work_read(unsigned long long out[2]);
void launch_svd_f64(const SvdArgs& a, int mcap, int ncap, cudaStream_t s);
bool launch_svd_subspace_f32(const SvdArgs& a, int mcap, int ncap, cudaStream_t s);

// ---------------------------------------------------------------- misc
void launch_zero(double* p, size_t n, cudaStream_t s);
void launch_copy(double* dst, const double* src, size_t n, cudaStream_t s);
void launch_fill(double* p, size_t n, double v, cudaStream_t s);
// out[(a,p), so, (b,q)] = sum_si W[p,so,si,q] A[a,si,b], capacities a<Ca, b<Cb
void launch_mpo_expand(const double* W, int wl, int wr, const double* A, int Ca, int Cb,
                       double* out, cudaStream_t s);
// Block-diagonal placement of up to 8 cores (actual dims read on the device).
struct AddTerm {
  const double* core;
  int capl, capr;
  const int* dl;  // actual left dim (device)
  const int* dr;  // actual right dim (device)
  double coef;    // applied on the first site
};
void launch_add_assemble(const AddTerm* terms, int K, int first, int last, double* out,
                         int capl_out, int capr_out, cudaStream_t s);
// Cores of P = H_B W (order 0) or W H_B (order 1), H_B the Hadamard MPO of
// the MPS core B (cbl x 4 x cbr), W an MPO core (wl x 4 x 4 x wr), in the raw,
// k2 and kr2 layouts (each cbl wl x 16 x cbr wr doubles).
void launch_hadamard_mpo(const double* B, int cbl, int cbr, const double* W, int wl, int wr,
                         int order, double* raw, double* k2, double* kr2, cudaStream_t s);
// out[b][s][a] = in[a][s][b]   (capacities)
void launch_core_transpose(const double* in, int Ca, int Cb, double* out, cudaStream_t s);

// A small constant matrix with few non-zeros (an MPO core reshaped as
// [(s q)][(p t)] or [(s p)][(q t)]), rows in compressed form; host-built.
constexpr int kSparseMaxRows = 64;
constexpr int kSparseMaxNnz = 96;
struct SparseRows {
  int rows = 0, cols = 0, nnz = -1;  // nnz < 0: not stored (too many entries)
  int ptr[kSparseMaxRows + 1];
  int col[kSparseMaxNnz];
  double val[kSparseMaxNnz];
};
// C_z = A B_z for z < nb (A rows x cols as `sp`; B_z cols x N with row
// stride ldb, batch stride sB; C_z rows x N, ldc, sC): each output element
// the FMA chain over A's non-zeros of its row in column order, which is
// the dense product's chain without its exact zero terms.
void launch_sparse_rows(const SparseRows& sp, const double* B, int ldb, long long sB, double* C,
                        int ldc, long long sC, int N, int nb, cudaStream_t s);
void launch_set_int(int* p, int v, cudaStream_t s);
void launch_fill_int(int* p, int n, int v, cudaStream_t s);
// out[b] = sum_t src[t][b] * mul[t][b] for 0 < b < nb-1, out[0] = out[nb-1] = 1
void launch_dims(const int* const* src, const int (*mul)[QTT_MAX_N + 1], int K, int nb, int* out,
                 cudaStream_t s);
void launch_dense_to_omega(const double* F, double* T, int n, cudaStream_t s);
void launch_omega_to_dense(const double* T, double* F, int n, cudaStream_t s);
void launch_check_finite(const double* p, size_t n, int* err, cudaStream_t s);

// CG on the two-component local vector (App. B).
struct CgVec {
  double* x[2];
  double* r[2];
  double* p[2];
  double* ap[2];
  long long len[2];
};
// scal: [0] r.r, [1] b.b, [2] tol^2 b.b ; ist: [0] done, [1] iterations
void launch_cg_start(const CgVec& v, const double* b0, const double* b1, double* scal, int* ist,
                     double tol, int* err, cudaStream_t s);
void launch_cg_step(const CgVec& v, double* scal, int* ist, int maxit, int* err, cudaStream_t s);
// device-driven loops of a captured step (see kernels_misc.cu)
void launch_loop_cond(cudaGraphConditionalHandle h, int* counter, const int* stop, int cap,
                      int first, cudaStream_t s, long long body_launches = 0,
                      long long* launched = nullptr);
void launch_cg_account(const int* ist, long long* stats, int maxit, cudaStream_t s);
void launch_sweep_check(double* scal, int* stop, long long* stats, double tol, int init,
                        cudaStream_t s);
void launch_sweep_final(const int* stop, long long* stats, cudaStream_t s);
void launch_sumsq2(const double* a, long long na, const double* b, long long nb, double* out,
                   cudaStream_t s);

// ---------------------------------------------------------------- learned truncation
void launch_rf_omega(double* O, int Dcap, const int* Dact, int wcap, const int* wact,
                     unsigned long long key, cudaStream_t s);
void launch_mlp_forward(const float* P, const float* X, int N, float* out, cudaStream_t s);
void launch_mlp_grad(const float* P, const float* X, const float* y, int N, float* Z, float* dout,
                     float* G, float* loss, cudaStream_t s);
void launch_adam(float* P, const float* G, float* m, float* v, int t, float lr, cudaStream_t s);
void launch_rf_predict(const float* P, const float* feat, const int* valid, int chi, int over,
                       int wcap, const int* Dact, const int* Nact4, int* w_out, int* use_rf,
                       cudaStream_t s);
void launch_rf_decide(const double* nM, const double* nB, double eps, const int* use_rf,
                      int* skip_full, double* total, long long* counters, cudaStream_t s);
void launch_rf_features(const double* sv, const int* skip_full, const int* w, const int* Dact,
                        const int* Nact4, const int* r, int bond, int n, float* feat, int* rank,
                        int* valid, cudaStream_t s);

// ---------------------------------------------------------------- diagnostics
// TKE spectrum of two dense N x N components (N = 2^logn <= 4096), see
// spectrum.cu; C1, C2: N * N double2 scratch, P: N * N, E: kmax + 1.
void launch_tke_spectrum(const double* u1, const double* u2, int logn, double2* C1, double2* C2,
                         double* P, double* E, int kmax, cudaStream_t s);
// Exact spectral projection of the dense pair (F1, F2) in place (N = 2^logn
// <= 8192), see spectrum.cu; c: nw <= 4 central-difference weights;
// C1, C2: N * N double2 scratch, sig: N doubles of scratch.
void launch_spectral_project(double* F1, double* F2, int logn, const double* c, int nw, double dx,
                             double2* C1, double2* C2, double* sig, cudaStream_t s);
