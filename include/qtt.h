/*
 * qtt.h -- C ABI of the QTT / MPS Navier-Stokes time step on one B300 GPU.
 *
 * The operations follow the problem statement of arXiv 2406.17823
 * ("quantum-inspired" incompressible 2-D Navier-Stokes): velocity
 * components are quantics tensor trains (MPS with interleaved x1/x2 bits,
 * Sec. II.B), derivatives are MPOs (App. A), the convection term uses
 * Hadamard products (Sec. II.B), and one time step is RK4 written as four
 * penalised Euler minimisations solved by DMRG-like sweeps (Sec. II.C,
 * App. B).  Every call below enqueues work on the context's CUDA stream
 * and returns without waiting, except where stated.
 *
 * Conventions shared by all calls
 *   - Grid: periodic, N = 2^n points per side over [0, L)^2, dx = L / N.
 *     A dense field is N*N doubles, row-major, F[x1 * N + x2] (x1 slow).
 *   - Site k = 1..n carries omega_k = 2 * x1^k + x2^k, site 1 the most
 *     significant bits (Sec. II.B).
 *   - An MPS with bond dimensions D_0 = 1, D_1, ..., D_n = 1 has cores of
 *     shape (D_{k-1}, 4, D_k).  The "packed" layout is the n cores one
 *     after the other, each contiguous and row-major.
 *   - qtt_mps / qtt_mpo objects are owned by the library: every `out`
 *     is newly allocated and must be released with qtt_free_mps /
 *     qtt_free_mpo.  Device buffers passed in (d_*) belong to the caller
 *     and are only read (or written, for outputs) by work on the context
 *     stream; they must stay valid until that work has completed.
 *   - Errors: every call returns a qtt_status.  Argument and shape errors
 *     are reported at once.  Errors found on the device (a non-finite
 *     value, a CG that did not converge) are recorded in the context and
 *     returned by the next call that synchronises (qtt_sync,
 *     qtt_to_dense, qtt_mps_info, qtt_mps_to_packed) or by
 *     qtt_project / qtt_rk4_step, which synchronise internally.
 *     qtt_last_error() gives a one-line description.
 */
#ifndef QTT_H_
#define QTT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtt_ctx_s* qtt_ctx;
typedef struct qtt_mps_s* qtt_mps;
typedef struct qtt_mpo_s* qtt_mpo;

typedef enum {
  QTT_OK = 0,
  QTT_ERR_ARG = 1,            /* invalid argument                         */
  QTT_ERR_SHAPE = 2,          /* incompatible n / bond dimensions         */
  QTT_ERR_ALLOC = 3,          /* device or host allocation failed         */
  QTT_ERR_CUDA = 4,           /* a CUDA runtime call failed               */
  QTT_ERR_NOT_CONVERGED = 5,  /* CG or sweep limit reached (result kept)  */
  QTT_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up       */
  QTT_ERR_NUMERIC = 7         /* NaN / Inf met on the device              */
} qtt_status;

typedef enum {
  QTT_PREC_FP64 = 0,   /* every contraction and factorisation in FP64      */
  QTT_PREC_MIXED = 1   /* FP32 subspace search refined by one FP64
                          subspace iteration; FP64 projection, truncation
                          weights and projection residual                    */
} qtt_precision;

/* Form of each Euler minimisation's right-hand side (qtt_params.rhs_form). */
typedef enum {
  QTT_RHS_EXPLICIT = 0,  /* w = a u - h B(b) formed as a compressed MPS
                            (Hadamard products, MPO applications, sums),
                            then projected; initial guess w                  */
  QTT_RHS_IMPLICIT = 1   /* the paper's form (Sec. II.C, App. B): B(b) never
                            formed -- its Hadamard and MPO terms enter the
                            projection's local right-hand sides through their
                            own environments; initial guess a u (the
                            previous time step), whose bonds are kept        */
} qtt_rhs_form;

/* How each Euler minimisation projects onto divergence-free fields
 * (qtt_params.projection). */
typedef enum {
  QTT_PROJ_PENALTY = 0,  /* the paper's penalised minimisation (App. B, cost
                            Theta): DMRG-like sweeps with CG local solves   */
  QTT_PROJ_SPECTRAL = 1  /* exact projection in Fourier space, the
                            alternative the paper's outlook (Sec. IV) points
                            to for periodic boundaries: qtt_project_spectral.
                            Explicit right-hand side only; n <= 13          */
} qtt_projection;

/* Learned truncation modes (qtt_params.learned_trunc). */
typedef enum {
  QTT_LEARNED_OFF = 0,
  QTT_LEARNED_LOG = 1,   /* plain FP64 cuts; log each cut's spectrum features  */
  QTT_LEARNED_ON = 2     /* range-finder cuts of predicted width, plain FP64
                            truncated SVD as the fallback; also logs           */
} qtt_learned_mode;

/* The rank predictor: 33 features -> 64 ReLU units -> 1 output (FP32),
 * parameters packed as W1 (64 x 33, row-major), b1 (64), W2 (64), b2. */
#define QTT_MLP_FEATURES 33
#define QTT_MLP_HIDDEN 64
#define QTT_MLP_PARAMS (QTT_MLP_HIDDEN * QTT_MLP_FEATURES + 2 * QTT_MLP_HIDDEN + 1)
/* Cuts logged per step (one slot per compression call; later calls of a
 * step are neither logged nor predicted). */
#define QTT_LEARNED_SLOTS 512

/* Solver parameters.  Paper defaults (Sec. II.C, App. B): mu = 2.5e5,
 * cg_tol = 1e-5, cg_maxit = 100, sweep_tol = 1e-5. */
typedef struct {
  int n;              /* bits per axis, 1 <= n <= 15                      */
  double L;           /* domain length (dx = L / 2^n)                     */
  double eps;         /* relative truncation per bond (Sec. III.E)        */
  int chi_max;        /* bond cap                                         */
  double mu;          /* penalty of the divergence term (App. B)          */
  double cg_tol;      /* CG stop: |r| <= cg_tol |b|                       */
  int cg_maxit;       /* CG iteration cap per local solve                 */
  double sweep_tol;   /* sweep stop: relative change of sum_i <v_i|v_i>   */
  int max_sweeps;     /* sweep cap per projection                         */
  int precision;      /* qtt_precision                                    */
  int learned_trunc;  /* qtt_learned_mode; LOG needs QTT_PREC_FP64 (ON
                         cuts every compression bond in FP64 either way) */
  int rf_oversample;  /* range-finder width = predicted rank + this (>= 0) */
  int rf_min_width;   /* only cuts whose full factor is at least this wide
                         (capacity) use the range finder (>= 1; 128)      */
  int graphs;         /* 0: every kernel launched from the host.
                         1: a stage's right-hand side w = a u - h B(b) runs
                         as a replayed CUDA graph (key: input capacities,
                         h, nu, a); the projection from the host.
                         2: as 1, and a whole RK4 step runs as one replayed
                         graph (key: capacities of u_1, u_2 and dt, nu), the
                         projection's CG and sweep loops as device-driven
                         WHILE nodes capped at cg_maxit / max_sweeps passes.
                         A key is captured at its second occurrence and
                         replayed from its third; inputs and outputs pass
                         through graph-owned buffers.  The kernels and their
                         per-stream order are those of the eager run, so
                         results are identical.  Ignored while profiling or
                         with learned truncation. */
  int fd_order;       /* order of the central differences: 0 or 2 the
                         paper's (App. A's carry table); 4, 6, 8 the
                         higher-order stencils of Sec. II.B / App. D.  D_1,
                         D_2, the Laplacian and the projection blocks are
                         all built with it.  Fixed at creation. */
  int rhs_form;       /* qtt_rhs_form (RK4, Euler and RK2 steps)          */
  int projection;     /* qtt_projection (RK4, Euler and RK2 steps); 0 the
                         paper's penalty                                    */
} qtt_params;

/* Create a context on `device`, enqueuing on `cuda_stream` (a cudaStream_t,
 * NULL = the legacy default stream).  Builds the MPOs D_1, D_2, the
 * Laplacian D_1 D_1 + D_2 D_2 and the projection blocks D_i^T D_j for
 * dx = L / 2^n (App. A).  Returns QTT_ERR_ARG for invalid parameters. */
qtt_status qtt_create(qtt_ctx* out, int device, void* cuda_stream, const qtt_params* params);
qtt_status qtt_destroy(qtt_ctx ctx);
/* Replace the solver parameters (n and L must not change). */
qtt_status qtt_set_params(qtt_ctx ctx, const qtt_params* params);
/* Wait for all work on the context stream; returns a deferred error. */
qtt_status qtt_sync(qtt_ctx ctx);
const char* qtt_last_error(qtt_ctx ctx);

/* Dense field (device, N*N doubles) -> QTT by a right-to-left TT-SVD with
 * per-bond truncation (eps, chi_max) (Sec. II.B, Sec. III.E). */
qtt_status qtt_from_dense(qtt_ctx ctx, const double* d_field, double eps, int chi_max,
                          qtt_mps* out);
/* QTT -> dense field (device, N*N doubles).  Synchronises. */
qtt_status qtt_to_dense(qtt_ctx ctx, qtt_mps mps, double* d_field_out);

/* Build an MPS from packed cores (see conventions).  `cores_are_device`
 * selects whether `cores` is a device or a host pointer; bonds[0..n]. */
qtt_status qtt_mps_from_packed(qtt_ctx ctx, const double* cores, int cores_are_device,
                               const int* bonds, qtt_mps* out);
/* Overwrite an existing MPS with packed cores (see conventions), keeping its
 * storage and capacities, so that a stepped state can be refreshed from the
 * host without new shapes (a stage graph keyed on those capacities stays
 * valid).  Requires bonds[0] = bonds[n] = 1 and 1 <= bonds[b] <= the MPS's
 * capacity at bond b (QTT_ERR_SHAPE otherwise); the padding is zeroed.
 * `cores_are_device` as in qtt_mps_from_packed.  Synchronises. */
qtt_status qtt_mps_upload_packed(qtt_ctx ctx, qtt_mps dst, const double* cores,
                                 int cores_are_device, const int* bonds);
/* <a|b> = sum over the grid of a(x) b(x) (the MPS inner product, used by
 * the paper's fidelity and kinetic-energy diagnostics, Sec. III): left
 * transfer matrices in FP64 on the context stream; synchronises and writes
 * the value to *out (host). */
qtt_status qtt_inner(qtt_ctx ctx, qtt_mps a, qtt_mps b, double* out);
/* Copy an MPS out in packed layout.  Synchronises; writes bonds[0..n] and
 * at most `capacity` doubles to `cores` (device or host). */
qtt_status qtt_mps_to_packed(qtt_ctx ctx, qtt_mps mps, double* cores, int cores_are_device,
                             size_t capacity, int* bonds);
/* n and the current bonds[0..n].  Synchronises. */
qtt_status qtt_mps_info(qtt_mps mps, int* n, int* bonds);
void qtt_free_mps(qtt_mps mps);

/* A new derivative MPO (App. A; Sec. II.B for higher orders): the central
 * difference of the context's fd_order along `axis` (1: x1, 2: x2) with
 * spacing dx, to the power `power` (1: D, 2: D D, the literal square the
 * paper's diffusion term uses).  The caller owns the handle (qtt_free_mpo).
 * QTT_ERR_ARG for an axis or power outside 1..2 or dx <= 0. */
qtt_status qtt_mpo_diff(qtt_ctx ctx, int axis, int power, double dx, qtt_mpo* out);
/* The context's operators: which = 1 (D_1), 2 (D_2), 3 (Laplacian),
 * 4 + 2i + j (the projection block D_i^T D_j, i, j in {0, 1}).  The handle
 * is a new reference owned by the caller. */
qtt_status qtt_mpo_get(qtt_ctx ctx, int which, qtt_mpo* out);
void qtt_free_mpo(qtt_mpo mpo);

/* out = compress(W |in>, eps, chi_max): site-wise MPO x MPS contraction
 * (Sec. II.B) followed by the compression sweep (Sec. II.C). */
qtt_status qtt_apply_mpo(qtt_ctx ctx, qtt_mpo mpo, qtt_mps in, double eps, int chi_max,
                         qtt_mps* out);
/* out = compress(sum_t coef[t] |terms[t]>, eps, chi_max), k >= 1 terms
 * (block-diagonal MPS sum, Sec. II.C "addition step"). */
qtt_status qtt_add(qtt_ctx ctx, int k, const double* coef, const qtt_mps* terms, double eps,
                   int chi_max, qtt_mps* out);
/* out ~ |a> (.) |b>, the element-wise product (Sec. II.B), by a
 * left-to-right zip-up capped at chi_max then compress(eps, chi_max). */
qtt_status qtt_hadamard(qtt_ctx ctx, qtt_mps a, qtt_mps b, double eps, int chi_max,
                        qtt_mps* out);
/* In-place compression sweep: left-to-right QR, right-to-left truncated
 * SVD keeping per bond the smallest rank whose discarded weight is at most
 * eps^2 of the bond's weight, capped at chi_max (Sec. II.C, Sec. III.E). */
qtt_status qtt_compress(qtt_ctx ctx, qtt_mps inout, double eps, int chi_max);
/* (v1, v2) = argmin mu |D_1 v1 + D_2 v2|^2 + |v - w|^2 / h^2 by DMRG-like
 * single-site sweeps with CG local solves (App. B, Eqs. "first", "second",
 * "big_LS"; Sec. II.C).  mu >= 0 is the penalty of this call (the steps use
 * qtt_params.mu); h > 0.  Initial guess w; bonds of w are kept.
 * Synchronises; cg_iters / sweeps may be NULL.  Returns
 * QTT_ERR_NOT_CONVERGED (results still written) when a cap was hit. */
qtt_status qtt_project(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, double h, double mu, qtt_mps* v1,
                       qtt_mps* v2, int* cg_iters, int* sweeps);
/* The exact discrete projection of (w1, w2) onto divergence-free fields:
 * the limit mu -> infinity of qtt_project, i.e. the orthogonal projection
 * onto the kernel of G = [D_1 D_2] (the central differences of the
 * context's fd_order), as the paper's outlook (Sec. IV) suggests for
 * periodic boundaries: both components are read out densely on the device,
 * transformed by 2-D FFTs, per wavevector m the part along sigma(m) is
 * removed (v_hat = w_hat - sigma (sigma . w_hat) / |sigma|^2, where D_j has
 * the Fourier symbol i sigma_j; wavevectors with sigma = 0, the mean and the
 * Nyquist modes, are kept), transformed back and encoded again by TT-SVD to
 * the context's (eps, chi_max).  New handles in *v1, *v2 (caller frees);
 * the inputs are left as they are.  Device scratch: 6 N^2 doubles
 * (N = 2^n).  QTT_ERR_SHAPE for n > 13 or inputs of another n.  Enqueued on
 * the context stream; device errors surface at the next synchronising
 * call. */
qtt_status qtt_project_spectral(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, qtt_mps* v1, qtt_mps* v2);
/* One RK4 step (App. B, Eq. "4euler", Table RK4, Eqs. U1-U4) in place:
 * *u1, *u2 are replaced by new handles (the old ones are released).
 * nu = 1 / Re.  Synchronises (the projections do). */
qtt_status qtt_rk4_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu);
/* The lower-order steps of App. B, in place like qtt_rk4_step (same
 * ownership, synchronisation and status rules): explicit Euler,
 * u^{s+1} = argmin Theta(v, a = u^s, b = u^s, h = dt) (Eq. "euler"), and the
 * midpoint RK2, u^{s+1/2} = argmin Theta(v, u^s, u^s, dt/2) then
 * u^{s+1} = argmin Theta(v, u^s, u^{s+1/2}, dt) (Eqs. "midpoint_calc",
 * "full_calc"). */
qtt_status qtt_euler_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu);
qtt_status qtt_rk2_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu);

/* The mixed form's dense product on the tensor cores (spec precision
 * option; no counterpart in the paper, which contracts in FP64 through
 * cuTensorNet): C = op(A) op(B) with op(A) M x K (A row-major M x K with
 * leading dimension lda, or its transpose when tA: A stored K x M), op(B)
 * K x N (B stored K x N, or N x K when tB), C M x N row-major (ldc), all
 * FP64 device buffers.  Both operands are split into two TF32 planes
 * (hi = tf32(x), lo = tf32(x - hi)) and multiplied by tcgen05 tensor-core
 * instructions as hi*hi + hi*lo + lo*hi with FP32 accumulation ("3xTF32");
 * the error is below about (K + 3) 2^-23 (|op(A)| |op(B)|)_ij.  Enqueued
 * on the context stream; scratch comes from the stream-ordered pool.
 * QTT_ERR_ARG for null pointers, sizes < 1 or leading dimensions below the
 * row length. */
qtt_status qtt_gemm_tf32x3(qtt_ctx ctx, int M, int N, int K, const double* A, int lda, int tA,
                           const double* B, int ldb, int tB, double* C, int ldc);

/* The mixed form's FP64 product on the BF16 tensor cores (north-star
 * precision option; the paper contracts in FP64 through cuTensorNet), by
 * the Ozaki splitting (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59,
 * 2012): for z = 0..batch-1,
 *   C_z = alpha op(A_z) op(B_z) + beta C_z,
 * A_z = A + z sA, B_z = B + z sB, C_z = C + z sC (element strides), op as
 * in qtt_gemm_tf32x3, all FP64 device buffers.  K is taken in chunks of 64;
 * in each chunk every row of op(A_z) and every column of op(B_z) is scaled
 * by a power of two 2^e (e the smallest with every |x| < 2^e) and cut into
 * eight signed 7-bit slices, the slice pairs (p, q) with p + q <= 7 are
 * multiplied exactly on the tensor cores (tcgen05 kind::f16, BF16
 * operands, exact FP32 accumulation) and their exact sum is rounded to FP64
 * once; the chunks' results are summed in order in FP64.  Error below
 * K 2^-53 2^(eA_i + eB_j) per element plus the FP64 rounding of the chunk
 * sums.  An unbatched product whose output tiles cannot fill the GPU has
 * its K chunks dealt over up to 16 slices computed side by side, whose
 * partial products (scratch from the stream-ordered pool) are summed in
 * slice order.  Sizes the kernel takes: K >= 16, K <= 1024 when
 * batch > 1 and K <= 16384 when batch = 1, 1 <= batch <= 65535,
 * max(M, N) >= 32, M N K batch >= 2^21; other sizes return QTT_ERR_SHAPE
 * (the library's FP64 GEMM serves them).  Enqueued on the context stream.
 * QTT_ERR_ARG for null pointers, sizes < 1 or leading dimensions below the
 * row length. */
qtt_status qtt_gemm_ozaki(qtt_ctx ctx, int M, int N, int K, const double* A, int lda, int tA,
                          long long sA, const double* B, int ldb, int tB, long long sB,
                          double* C, int ldc, long long sC, int batch, double alpha,
                          double beta);

/* Turbulent kinetic energy spectrum of the velocity (u1, u2) (the paper's
 * TKE spectra, Sec. III.A), computed on the device: the dense fields, their
 * 2-D DFTs, and E(k) = sum over wavevectors m with round(|m|) = k of
 * (|u1_hat(m)|^2 + |u2_hat(m)|^2) / (2 N^4) for k = 0..kmax (shells in units
 * of 2 pi / L; wavevectors beyond kmax are left out; with kmax >=
 * ceil(N / sqrt 2) the shells sum to the mean kinetic energy
 * 1/2 mean(u1^2 + u2^2)).  Writes kmax + 1 doubles to h_E (host) and
 * synchronises.  QTT_ERR_SHAPE for n > 12 or components on different grids. */
qtt_status qtt_tke_spectrum(qtt_ctx ctx, qtt_mps u1, qtt_mps u2, int kmax, double* h_E);

/* Subspace searches of the mixed form (QTT_PREC_MIXED) served by the
 * tensor cores since creation, and those whose acceptance test failed so
 * that the FP32 cluster SVD recomputed the subspace.  Synchronises. */
qtt_status qtt_tc_stats(qtt_ctx ctx, long long* accepted, long long* fell_back);

/* Counters of the last qtt_project / qtt_rk4_step: total CG iterations,
 * sweeps, kernel launches enqueued by the library since context creation. */
qtt_status qtt_stats(qtt_ctx ctx, long long* cg_iters, long long* sweeps,
                     long long* launches);

/* Stage and step graphs (qtt_params.graphs): graphs captured and kept by
 * the context (at most 16 of the two kinds together; cleared by
 * qtt_set_params) and replays of either kind since creation.  A key
 * occurring for the second time runs eagerly and is captured; from the
 * third time on it is replayed.  QTT_ERR_ARG for null arguments. */
qtt_status qtt_graph_stats(qtt_ctx ctx, long long* captured, long long* replays);

/* Per-kernel timing of the work enqueued between qtt_profile_begin and
 * qtt_profile_end: CUDA events are recorded on the context stream around
 * every launch (a few microseconds each).  qtt_profile_end synchronises and
 * writes a JSON object {"<kernel>": {"launches": L, "ms": T, "flops": F}, ...}
 * (F = the algorithmic FLOPs of those launches, from their shapes) into buf
 * (at most cap bytes, NUL-terminated); QTT_ERR_ARG if buf is too small. */
qtt_status qtt_profile_begin(qtt_ctx ctx);
qtt_status qtt_profile_end(qtt_ctx ctx, char* buf, size_t cap);

/* Dense readout that allocates nothing (the paper has no counterpart): for
 * callers that cannot allocate device memory when they need the field, such
 * as code running during CUDA graph capture, real-time loops that must not
 * enter an allocator, or hosts whose device memory is owned by another
 * framework's pool.  Same result as qtt_to_dense, but the MPS comes as
 * packed cores in a caller-owned device buffer (d_cores, bonds[0..n] on the
 * host) and the field is written to the caller's d_field_out (N*N doubles,
 * N = 2^n), enqueued on cuda_stream (a cudaStream_t, NULL = legacy default).
 * Intermediates live in a static 4 MiB device array: n <= 9 and every
 * partial contraction 4^k * bonds[k] (k < n) at most 2^18 doubles, else
 * QTT_ERR_SHAPE; QTT_ERR_ARG for null pointers or n outside 1..9.  The
 * array's device address is looked up once per device, with that device
 * current: qtt_create does it for its device, otherwise the first call on a
 * device does, so a caller without a context makes one call before any
 * stream capture.  The cached address assumes the device's primary context
 * lives as long as the process (no cudaDeviceReset).  All calls share the
 * array: calls whose work overlaps on the GPU race and must be ordered by
 * the caller.  Uses no cudaMalloc / cudaFree.  Asynchronous: launch errors
 * are returned (QTT_ERR_CUDA), execution errors surface at the caller's
 * next synchronisation. */
qtt_status qtt_to_dense_noalloc(const double* d_cores, const int* bonds, int n,
                                double* d_field_out, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Learned truncation (no counterpart in the paper's method; a systems
 * extension of its compression, Sec. II.C).  Each compression call of a
 * step gets a slot 0 .. QTT_LEARNED_SLOTS-1 in call order; slots restart at
 * every qtt_rk4_step (or qtt_learned_next_step).  For every right-to-left
 * cut the library records 33 features (the top 32 values of
 * log10(sigma / sigma_1) clipped at -16 and scaled by 1/16, then bond / n)
 * and the rank kept.  In QTT_LEARNED_ON mode the cut of bond b in slot s
 * first runs a randomised range finder (Halko, Martinsson and Tropp 2011,
 * Alg. 4.1) of width min(r + rf_oversample, ...) with r predicted by the
 * perceptron from the PREVIOUS step's features of (s, b); when the weight
 * outside the sketch, |M|^2 - |B|^2, exceeds 0.1 eps^2 |M|^2 (or no
 * features exist yet) the plain truncated SVD overwrites the result.  Only
 * cuts whose full factor is at least rf_min_width wide (capacity) take this
 * path; narrower ones keep the plain SVD.  The test
 * matrix is SplitMix64 / Box-Muller with key (seed << 40) ^ (s << 8) ^ b,
 * seed 0.
 * --------------------------------------------------------------------- */

/* Perceptron parameters (device, QTT_MLP_PARAMS floats) used by
 * QTT_LEARNED_ON; copied, so the caller's buffer may be reused. */
qtt_status qtt_learned_set(qtt_ctx ctx, const float* d_params);
/* Start a new step's slots (qtt_rk4_step does this itself): the current
 * features become the previous step's. */
qtt_status qtt_learned_next_step(qtt_ctx ctx);
/* Copy the current step's log to host memory: h_feat[slot][b][33] and
 * h_rank[slot][b] for slots < max_slots and b = 0..n (entries without a
 * cut have rank 0).  Synchronises; *n_slots = slots used so far. */
qtt_status qtt_learned_log(qtt_ctx ctx, float* h_feat, int* h_rank, int max_slots,
                           int* n_slots);
/* Cuts served by the range finder / cuts that fell back, since creation. */
qtt_status qtt_learned_stats(qtt_ctx ctx, long long* accepted, long long* fell_back);
/* Gaussian test matrix of the range finder (device, 4*D x w doubles,
 * row-major, entry (s*D + b, j)) for `key`; for tests of the generator. */
qtt_status qtt_rf_omega(qtt_ctx ctx, unsigned long long key, int D, int w, double* d_out);

/* Perceptron on device arrays: X (N x 33, row-major), y (N), params
 * (QTT_MLP_PARAMS).  Forward: out (N).  Loss and gradient of the mean
 * squared error: grad (QTT_MLP_PARAMS), loss (1 float); deterministic.
 * Train: `iters` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8) from
 * zero moments, updating params in place; loss_out (may be NULL) receives
 * the loss before each step (iters floats). */
qtt_status qtt_mlp_forward(qtt_ctx ctx, const float* d_params, const float* d_X, int N,
                           float* d_out);
qtt_status qtt_mlp_loss_grad(qtt_ctx ctx, const float* d_params, const float* d_X,
                             const float* d_y, int N, float* d_grad, float* d_loss);
qtt_status qtt_mlp_train(qtt_ctx ctx, float* d_params, const float* d_X, const float* d_y,
                         int N, int iters, float lr, float* d_loss_out);

/* ---------------------------------------------------------------------
 * Batched trajectories (no counterpart in the paper: an ensemble of
 * independent flows stepped together on one GPU).  A batch owns B contexts,
 * each with its own parameters (n, chi_max, ... may differ) and its own
 * non-blocking CUDA stream; qtt_rk4_step_batched runs one RK4 step of every
 * trajectory at once, one host thread per trajectory, so that the
 * factorisations of different trajectories occupy the GPU's SMs together.
 * --------------------------------------------------------------------- */
typedef struct qtt_batch_s* qtt_batch;
qtt_status qtt_batch_create(qtt_batch* out, int device, int B, const qtt_params* per_traj);
qtt_status qtt_batch_destroy(qtt_batch batch);
/* The context of trajectory i (0 <= i < B), for I/O calls; owned by the
 * batch (do not destroy).  NULL for an invalid index. */
qtt_ctx qtt_batch_context(qtt_batch batch, int i);
/* One RK4 step of every trajectory, in place as qtt_rk4_step: u1s[i],
 * u2s[i] belong to context i and are replaced by new handles.  Waits for
 * all trajectories; returns the first status that is not QTT_OK in
 * trajectory order (QTT_ERR_NOT_CONVERGED included), all results kept. */
qtt_status qtt_rk4_step_batched(qtt_batch batch, qtt_mps* u1s, qtt_mps* u2s, const double* dts,
                                const double* nus);

#ifdef __cplusplus
}
#endif
#endif /* QTT_H_ */
