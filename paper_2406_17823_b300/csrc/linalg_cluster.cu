// FP64 QR and SVD spread over a thread-block cluster (8 or 16 CTAs, one
// problem per cluster).  Same algorithms and rounding behaviour as the
// single-CTA kernels in linalg_f64.cu (Householder QR; QR of the tall
// orientation then one-sided Jacobi with round-robin pairs), but:
//
//  * Householder: the columns of the tall matrix are dealt cyclically to
//    the CTAs; the owner of column j forms reflector j, a cluster barrier
//    publishes it, and every CTA applies it to its own columns.
//  * Jacobi: column i of the square factor X and of the rotation
//    accumulator J lives in the shared memory of CTA (i mod CL); in each
//    round every CTA rotates the pairs dealt to it, reading and writing the
//    two columns wherever they live (distributed shared memory), and a
//    cluster barrier ends the round.
//
// On this GPU an SM retires about two FP64 FMAs per clock, so spreading an
// O(c^3) factorisation over the cluster is what makes it affordable.
#include <cooperative_groups.h>
#include <math.h>
#include <stdlib.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

// Arithmetic actually performed by the cluster SVDs (FLOPs: Householder QR,
// Jacobi dot products and rotations counted per visit / per rotation, Q
// application), [0] FP64, [1] FP32; read by the profiler.
__device__ unsigned long long g_svd_work[2];

void svd_work_reset() {
  const unsigned long long z[2] = {0, 0};
  cudaMemcpyToSymbol(g_svd_work, z, sizeof z);
}
void svd_work_read(unsigned long long out[2]) {
  cudaMemcpyFromSymbol(out, g_svd_work, 2 * sizeof(unsigned long long));
}

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum_c(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ T cta_sum_c(T v, double* sh) {
  v = warp_sum_c(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = (double)v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; i++) t += sh[i];
  return (T)t;
}

// numerical constants per working precision: columns below `tiny` in
// squared norm are not reflected; Jacobi stops rotating below `cos_tol`
template <typename T> struct Prec;
template <> struct Prec<double> {
  static __device__ double tiny() { return 1e-280; }
  static __device__ double cos_tol(int c) { return fmax(1e-15, 1e-16 * (double)c); }
};
template <> struct Prec<float> {
  static __device__ float tiny() { return 1e-30f; }
  static __device__ float cos_tol(int) { return 4e-6f; }
};

__device__ __forceinline__ bool axis_ok_c(const Axis& a) {
  const int h = dval(a.hact), l = dval(a.lact);
  return h >= 0 && h <= a.hcap && l >= 1 && l <= a.lcap;
}
__device__ __forceinline__ bool view_ok_c(const MatView& v) {
  return axis_ok_c(v.rows) && axis_ok_c(v.cols);
}
__device__ __forceinline__ long long voff(const MatView& v, int ic, int jc, int rl, int cl) {
  return (long long)axis_full(v.rows, ic, rl) * v.ld + axis_full(v.cols, jc, cl);
}

// zero the capacity region of a view, rows dealt over the cluster
__device__ void zero_view_cl(const MatView& v, int rank, int CL) {
  const int R = v.rows.hcap * v.rows.lcap, C = v.cols.hcap * v.cols.lcap;
  for (int i = rank; i < R; i += CL)
    for (int j = threadIdx.x; j < C; j += blockDim.x) v.ptr[(long long)i * v.ld + j] = 0.0;
}

// Householder QR of W (m x c, column-major, ld = m) with the columns dealt
// cyclically over the cluster.  tau / diag live in global memory.
template <typename T>
__device__ void householder_cl(cg::cluster_group& cl, T* W, int m, int c, T* tau, T* diag,
                               double* sh, int rank, int CL) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kmax = min(m, c);
  for (int j = 0; j < kmax; j++) {
    T* col = W + (size_t)j * m;
    __syncthreads();  // this CTA's updates of column j (if it owns it) are complete
    if (j % CL == rank) {
      T part = 0;
      for (int i = j + threadIdx.x; i < m; i += blockDim.x) part += col[i] * col[i];
      const T nrm2 = cta_sum_c(part, sh);
      const T x0 = col[j];
      __syncthreads();
      T t = 0, alpha = x0;
      if (nrm2 > Prec<T>::tiny() && isfinite((double)nrm2)) {
        const T nrm = sqrt(nrm2);
        alpha = (x0 >= 0) ? -nrm : nrm;
        t = (T)1 / (nrm * (nrm + fabs(x0)));
        if (threadIdx.x == 0) col[j] = x0 - alpha;
      }
      if (threadIdx.x == 0) {
        tau[j] = t;
        diag[j] = alpha;
      }
    }
    cl.sync();  // reflector j published
    const T t = *(volatile T*)(tau + j);
    if (t != (T)0) {
      // my columns cc > j with cc % CL == rank
      int c0 = j + 1;
      c0 += ((rank - c0) % CL + CL) % CL;
      for (int cc = c0 + warp * CL; cc < c; cc += nw * CL) {
        T* x = W + (size_t)cc * m;
        T s = 0;
        for (int i = j + lane; i < m; i += 32) s += col[i] * x[i];
        s = warp_sum_c(s) * t;
        for (int i = j + lane; i < m; i += 32) x[i] -= s * col[i];
      }
    }
  }
  cl.sync();
}

// Blocked Householder QR of W (m x c, column-major, global memory), same
// output format as householder_cl (R above the diagonal, the reflectors v_j
// below it with v_j[j] = x_j - alpha_j, tau and diag = alpha in global
// memory).  Panels of PB columns: panel p is factored by CTA p mod CL alone
// (its columns in that CTA's shared memory, CTA barriers only), which also
// forms the panel's compact-WY factor Tp (H_0 ... H_{b-1} = I - V Tp V^T,
// upper triangular, Schreiber-Van Loan).  One cluster barrier publishes the
// panel; every CTA then updates its own trailing columns (column j belongs
// to CTA (j / PB) mod CL, so a panel's columns are updated by the CTA that
// will factor them) as C <- C - V Tp^T (V^T C), reading each column once per
// panel instead of once per reflector.  sm: PB * m elements (the panel, then
// V); Tsh: 2 x PB x PB.
template <typename T, int PB>
__device__ void householder_blocked_cl(cg::cluster_group& cl, T* W, int m, int c, T* tau,
                                       T* diag, double* sh, int rank, int CL, T* sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ T Tsh[2][PB * PB];
  __shared__ T Tl[PB * PB];
  const int kmax = min(m, c);
  for (int p0 = 0, pi = 0; p0 < kmax; p0 += PB, pi++) {
    const int bb = min(PB, kmax - p0);
    const int owner = pi % CL;
    const int rows = m - p0;  // panel rows p0 .. m-1
    T* Tp = Tsh[pi & 1];
    __syncthreads();  // this CTA's updates of the previous panel are complete
    if (rank == owner) {
      // panel (rows p0.., columns p0..p0+bb-1) into shared memory, ld = rows
      for (int jj = 0; jj < bb; jj++)
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
          sm[(size_t)jj * rows + i] = W[(size_t)(p0 + jj) * m + p0 + i];
      __syncthreads();
      for (int jj = 0; jj < bb; jj++) {
        const int j = p0 + jj;
        T* x = sm + (size_t)jj * rows;  // x[i - p0] is row i
        T part = 0;
        for (int i = jj + threadIdx.x; i < rows; i += blockDim.x) part += x[i] * x[i];
        const T nrm2 = cta_sum_c(part, sh);
        const T x0 = x[jj];
        __syncthreads();
        T t = 0, alpha = x0;
        if (nrm2 > Prec<T>::tiny() && isfinite((double)nrm2)) {
          const T nrm = sqrt(nrm2);
          alpha = (x0 >= 0) ? -nrm : nrm;
          t = (T)1 / (nrm * (nrm + fabs(x0)));
        }
        if (threadIdx.x == 0) {
          if (t != (T)0) x[jj] = x0 - alpha;
          tau[j] = t;
          diag[j] = alpha;
          Tl[jj * PB + jj] = t;
        }
        __syncthreads();
        if (t != (T)0) {  // apply H_j to the panel's later columns
          for (int kk = jj + 1 + warp; kk < bb; kk += nw) {
            T* y = sm + (size_t)kk * rows;
            T d = 0;
            for (int i = jj + lane; i < rows; i += 32) d += x[i] * y[i];
            d = warp_sum_c(d) * t;
            for (int i = jj + lane; i < rows; i += 32) y[i] -= d * x[i];
          }
        }
        __syncthreads();
      }
      // Tp: column i above the diagonal = -tau_i Tp[0:i, 0:i] (V[:, 0:i]^T v_i)
      // (v_k is zero above row k; a zero tau leaves its row and column zero)
      for (int i = 0; i < bb; i++) {
        for (int k = warp; k < i; k += nw) {
          const T* vk = sm + (size_t)k * rows;
          const T* vi = sm + (size_t)i * rows;
          T d = 0;
          for (int r = i + lane; r < rows; r += 32) d += vk[r] * vi[r];
          d = warp_sum_c(d);
          if (lane == 0) Tl[k * PB + i] = d;  // temporarily V^T v_i
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          const T ti = Tl[i * PB + i];
          T tmp[PB];
          for (int k = 0; k < i; k++) {
            T acc = 0;
            for (int q = k; q < i; q++) acc += Tl[k * PB + q] * Tl[q * PB + i];
            tmp[k] = -ti * acc;
          }
          for (int k = 0; k < i; k++) Tl[k * PB + i] = tmp[k];
          for (int k = i + 1; k < PB; k++) Tl[k * PB + i] = 0;
        }
        __syncthreads();
      }
      for (int e = threadIdx.x; e < PB * PB; e += blockDim.x) {
        const int k = e / PB, i = e % PB;
        Tp[e] = (k < bb && i < bb && k <= i) ? Tl[e] : (T)0;
      }
      // the factored panel back to W (R above the diagonal, v below)
      for (int jj = 0; jj < bb; jj++)
        for (int i = threadIdx.x; i < rows; i += blockDim.x)
          W[(size_t)(p0 + jj) * m + p0 + i] = sm[(size_t)jj * rows + i];
    }
    cl.sync();  // panel pi published: V in W, Tp in the owner's shared memory
    // every CTA: V into its shared memory, Tp from the owner
    for (int jj = 0; jj < bb; jj++)
      for (int i = threadIdx.x; i < rows; i += blockDim.x)
        sm[(size_t)jj * rows + i] = (i >= jj) ? W[(size_t)(p0 + jj) * m + p0 + i] : (T)0;
    {
      const T* Tr = cl.map_shared_rank(Tp, owner);
      for (int e = threadIdx.x; e < PB * PB; e += blockDim.x) Tl[e] = Tr[e];
    }
    __syncthreads();
    // own trailing columns: C <- C - V Tp^T (V^T C), one warp per column
    const int first = p0 + bb;
    // columns cc >= first with (cc / PB) % CL == rank, dealt to the warps
    int idx = 0;
    for (int cc = first; cc < c; cc++) {
      if ((cc / PB) % CL != rank) continue;
      if (idx++ % nw != warp) continue;
      T* x = W + (size_t)cc * m + p0;
      T w[PB];
#pragma unroll
      for (int k = 0; k < PB; k++) w[k] = 0;
      for (int i = lane; i < rows; i += 32) {
        const T xi = x[i];
#pragma unroll
        for (int k = 0; k < PB; k++)
          if (k < bb) w[k] += sm[(size_t)k * rows + i] * xi;
      }
#pragma unroll
      for (int k = 0; k < PB; k++) w[k] = warp_sum_c(w[k]);
      T w2[PB];
#pragma unroll
      for (int i2 = 0; i2 < PB; i2++) {  // w2 = Tp^T w
        T acc = 0;
#pragma unroll
        for (int k = 0; k < PB; k++)
          if (k <= i2) acc += Tl[k * PB + i2] * w[k];
        w2[i2] = acc;
      }
      for (int i = lane; i < rows; i += 32) {
        T acc = x[i];
#pragma unroll
        for (int k = 0; k < PB; k++)
          if (k < bb) acc -= sm[(size_t)k * rows + i] * w2[k];
        x[i] = acc;
      }
    }
  }
  cl.sync();
}

// Householder QR of W with the widest panel the shared-memory scratch
// (sm_elems elements) holds for m rows; the column-at-a-time version when
// not even four columns fit (or QTT_QR_UNBLOCKED is set on the host), and
// always in FP64: a panel factored by one SM at two FP64 FMAs per clock
// stalls the cluster (measured slower than the column-at-a-time form), while
// in FP32 the blocked form reads each trailing column once per panel instead
// of once per reflector (measured 1.7x faster for the 4096-row factors).
template <typename T>
__device__ void householder_any_cl(cg::cluster_group& cl, T* W, int m, int c, T* tau, T* diag,
                                   double* sh, int rank, int CL, T* sm, long long sm_elems) {
  if constexpr (sizeof(T) == 8) {
    householder_cl<T>(cl, W, m, c, tau, diag, sh, rank, CL);
    return;
  }
  if (sm_elems >= 16LL * m) householder_blocked_cl<T, 16>(cl, W, m, c, tau, diag, sh, rank, CL, sm);
  else if (sm_elems >= 8LL * m) householder_blocked_cl<T, 8>(cl, W, m, c, tau, diag, sh, rank, CL, sm);
  else if (sm_elems >= 4LL * m) householder_blocked_cl<T, 4>(cl, W, m, c, tau, diag, sh, rank, CL, sm);
  else householder_cl<T>(cl, W, m, c, tau, diag, sh, rank, CL);
}

// B (m x nb, column-major, ld = m): columns cc % CL == rank get
// B[:, cc] <- H_0 ... H_{k-1} B[:, cc]  (columns are independent).
template <typename T>
__device__ void apply_reflectors_cl(const T* W, int m, int k, const T* tau, T* B, int nb,
                                    bool identity_cols, int rank, int CL) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int cc = rank + warp * CL; cc < nb; cc += nw * CL) {
    T* x = B + (size_t)cc * m;
    const int jtop = identity_cols ? min(cc, k - 1) : k - 1;
    for (int j = jtop; j >= 0; j--) {
      const T t = tau[j];
      if (t == (T)0) continue;
      const T* v = W + (size_t)j * m;
      T s = 0;
      for (int i = j + lane; i < m; i += 32) s += v[i] * x[i];
      s = warp_sum_c(s) * t;
      for (int i = j + lane; i < m; i += 32) x[i] -= s * v[i];
    }
  }
}

__global__ void __launch_bounds__(512) k_qr_cluster(QrArgs a, long long sm_elems) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  __shared__ double sh[32];
  if (a.skip && *a.skip) return;  // uniform over the cluster
  const Axis& fr = a.inT ? a.A.cols : a.A.rows;
  const Axis& fc = a.inT ? a.A.rows : a.A.cols;
  const int m = axis_len(fr), c = axis_len(fc);
  const int arl = dval(a.A.rows.lact), acl = dval(a.A.cols.lact);
  const int r = min(m, c);
  {
    const int fr_cap = fr.hcap * fr.lcap, fc_cap = fc.hcap * fc.lcap;
    const int qr_cap = a.qT ? a.Q.cols.hcap * a.Q.cols.lcap : a.Q.rows.hcap * a.Q.rows.lcap;
    const int qc_cap = a.qT ? a.Q.rows.hcap * a.Q.rows.lcap : a.Q.cols.hcap * a.Q.cols.lcap;
    const int rr_cap = a.rT ? a.R.cols.hcap * a.R.cols.lcap : a.R.rows.hcap * a.R.rows.lcap;
    const int rc_cap = a.rT ? a.R.rows.hcap * a.R.rows.lcap : a.R.cols.hcap * a.R.cols.lcap;
    const bool bad = !view_ok_c(a.A) || !view_ok_c(a.Q) || !view_ok_c(a.R) || m < 1 || c < 1 ||
                     m > fr_cap || c > fc_cap || m > qr_cap || r > qc_cap || r > rr_cap ||
                     c > rc_cap ||
                     (long long)m * c + (long long)m * r + 2LL * c > a.work_len;
    if (bad) {
      if (rank == 0 && threadIdx.x == 0 && a.err) atomicOr(a.err, QTT_DEVERR_SHAPE);
      return;  // every CTA of the cluster takes this branch
    }
  }
  double* W = a.work;
  double* Qw = W + (size_t)m * c;
  double* tau = Qw + (size_t)m * r;
  double* diag = tau + c;
  bool badv = false;
  for (int j = rank; j < c; j += CL)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const long long off = a.inT ? voff(a.A, j, i, arl, acl) : voff(a.A, i, j, arl, acl);
      const double v = a.A.ptr[off];
      badv |= !isfinite(v);
      W[(size_t)j * m + i] = v;
    }
  if (badv && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
  cl.sync();
  extern __shared__ double qr_dyn[];
  householder_any_cl<double>(cl, W, m, c, tau, diag, sh, rank, CL, qr_dyn, sm_elems);
  for (int j = rank; j < r; j += CL)
    for (int i = threadIdx.x; i < m; i += blockDim.x) Qw[(size_t)j * m + i] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  apply_reflectors_cl<double>(W, m, r, tau, Qw, r, true, rank, CL);
  cl.sync();  // all reads of A done before outputs (they may alias A)
  zero_view_cl(a.Q, rank, CL);
  zero_view_cl(a.R, rank, CL);
  cl.sync();
  const int qrl = dval(a.Q.rows.lact), qcl = dval(a.Q.cols.lact);
  for (int j = rank; j < r; j += CL)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const long long off = a.qT ? voff(a.Q, j, i, qrl, qcl) : voff(a.Q, i, j, qrl, qcl);
      a.Q.ptr[off] = Qw[(size_t)j * m + i];
    }
  const int rrl = dval(a.R.rows.lact), rcl = dval(a.R.cols.lact);
  for (int j = rank; j < c; j += CL)
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      double v = 0.0;
      if (j == i) v = diag[i];
      else if (j > i) v = W[(size_t)j * m + i];
      const long long off = a.rT ? voff(a.R, j, i, rrl, rcl) : voff(a.R, i, j, rrl, rcl);
      a.R.ptr[off] = v;
    }
  if (rank == 0 && threadIdx.x == 0 && a.r_out) *a.r_out = r;
}

__device__ __forceinline__ int rr_pos_c(int k, int t, int cp) {
  return k == 0 ? 0 : 1 + (k - 1 + t) % (cp - 1);
}


// Systolic one-sided Jacobi (circle ordering of the round-robin
// tournament).  Pair slot s (0 .. P-1, P = cp/2) is held in REGISTERS by warp
// (s mod spc) of CTA (s / spc): lane l keeps rows l, l+32, ... of the slot's
// two columns of X and of J, so a round needs no shared-memory reads for its
// dot products or rotations.  After rotating, the columns move one place
// along the circle (slot 0 keeps its first column): slot s hands its first
// column (slot 0: its second) to slot s+1 and its second column to slot s-1,
// through mailboxes in the receiver's shared memory (double-buffered by
// round parity, so one cluster barrier per round suffices: a mailbox of
// parity t is rewritten only after every reader of round t-2 has passed
// the barrier of round t-1).  Column ids travel with the columns and fix
// the orientation of each pair (lower id first), as in the scalar kernel.
// The circle has period cp-1, so after each sweep every column is back in
// its starting slot.  Rows at and beyond c are zero in every register.
//
// FP64 (about two FMAs per clock per SM on this GPU) takes three shortcuts
// that keep the arithmetic but cut the instruction count: the squared
// column norms travel with the columns and are updated by the exact Jacobi
// identities |x'|^2 = |x|^2 - t g, |y'|^2 = |y|^2 + t g (recomputed at the
// start of every sweep and whenever an update cancels more than 99%), so a
// round computes one dot product instead of three; the rotation scalars of
// all pairs of a CTA are computed by one warp, one pair per lane, instead
// of redundantly by all 32 lanes of every pair's warp; and the rotations
// are scaled ("fast" Givens, as in LAPACK's one-sided Jacobi): a column is
// held as d * x, a rotation updates x by two FMAs per element pair,
// x_a -= t (d_b / d_a) x_b, x_b += t (d_a / d_b) x_a, and multiplies both
// scales by cos; the scales (at least cos^(c-1) >= 2^-128 within a sweep)
// are folded into the columns at every sweep start.
template <typename T>
__device__ __forceinline__ bool jacobi_angle(T al, T be, T ga, T tol, T& cs, T& sn, T& tt) {
  if (!(ga != (T)0 && fabs(ga) > tol * sqrt(al) * sqrt(be))) return false;
  const T zeta = (be - al) / ((T)2 * ga);
  tt = copysign((T)1, zeta) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
  cs = (T)1 / sqrt((T)1 + tt * tt);
  sn = cs * tt;
  return true;
}

// FP32 (the mixed form's subspace search, latency-bound per round): the
// same angle with the hardware's approximate reciprocal and reciprocal
// square root, measured at about a third of the IEEE divide / square-root
// chain.  The test compares squares (no square roots); one Newton-Raphson
// step on rsqrt restores cos to full precision, so that cos^2 + sin^2 = 1
// to rounding and the rotation stays orthogonal (the angle itself only
// needs to be near the optimum).  Columns below 1e-30 in squared norm, and
// angles whose zeta would overflow, take the IEEE path.
template <>
__device__ __forceinline__ bool jacobi_angle<float>(float al, float be, float ga, float tol,
                                                   float& cs, float& sn, float& tt) {
  if (!(ga != 0.0f)) return false;
  if (al < 1e-30f || be < 1e-30f) {
    if (!(fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return false;
  } else if (!(ga * ga > (tol * tol) * (al * be))) {
    return false;
  }
  const float zeta = __fdividef(be - al, 2.0f * ga);
  const float az = fabsf(zeta);
  if (az > 1e15f) {
    tt = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.0f);
    const float root = q * rsqrtf(q);  // sqrt(1 + zeta^2)
    tt = copysignf(__fdividef(1.0f, az + root), zeta);
  }
  const float x = fmaf(tt, tt, 1.0f);
  float r = rsqrtf(x);
  r = r * fmaf(-0.5f * x * r, r, 1.5f);  // Newton-Raphson step for 1/sqrt(x)
  cs = r;
  sn = r * tt;
  return true;
}

template <typename T, int EPL>
__device__ __forceinline__ T warp_dot(const T (&u)[EPL], const T (&v)[EPL]) {
  T s = 0;
#pragma unroll
  for (int e = 0; e < EPL; e++) s += u[e] * v[e];
  return warp_sum_c(s);
}

template <typename T, int EPL, typename XC, typename JC>
__device__ void jacobi_systolic(cg::cluster_group& cl, XC xcol, JC jcol, int c, T tol, T* box,
                                int spc, int rank, int* flag_local, bool withJ) {
  constexpr bool kTrack = sizeof(T) == 8;  // FP64: tracked norms, shared scalars
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cp = c + (c & 1), P = cp / 2;
  const int s = rank * spc + warp;
  const bool active = warp < spc && s < P;
  const int nact = max(0, min(spc, P - rank * spc));  // active slots of this CTA
  __shared__ int mb_id[2][16][2];
  __shared__ T mb_nrm[2][16][2];
  __shared__ T mb_scl[2][16][2];
  __shared__ T sc_in[16][5];   // (alpha, beta, gamma, d_a, d_b) per slot, FP64 only
  __shared__ T sc_out[16][4];  // (cs, t d_b / d_a, t d_a / d_b, t); t = 0: no rotation
  constexpr int L = 32 * EPL;  // mailbox column length
  // box[buf][lslot][which][xj][L]; which 0 = new first column, 1 = new second
  auto mbox = [&](T* base, int buf, int ls, int which, int xj) -> T* {
    return base + ((((size_t)buf * spc + ls) * 2 + which) * 2 + xj) * L;
  };
  T xa[EPL], xb[EPL], ja[EPL], jb[EPL];
  int ida = 2 * s, idb = 2 * s + 1;
  unsigned long long n_dot = 0, n_rot = 0;  // dot products and rotations done
  T na = -1, nb = -1;  // tracked squared norms (negative: recompute)
  T da = 1, db = 1;    // column scales (FP64: the column is d * x)
  if (active) {
#pragma unroll
    for (int e = 0; e < EPL; e++) {
      const int i = lane + 32 * e;
      const bool ok = i < c;
      xa[e] = (ok && ida < c) ? xcol(ida)[i] : (T)0;
      ja[e] = (withJ && ok && ida < c) ? jcol(ida)[i] : (T)0;
      xb[e] = (ok && idb < c) ? xcol(idb)[i] : (T)0;
      jb[e] = (withJ && ok && idb < c) ? jcol(idb)[i] : (T)0;
    }
  }
  // destinations are fixed per slot: next slot (as its first column) and
  // previous slot (as its second column)
  const int sn_ = s + 1, sp_ = s - 1;
  T* to_next = (active && sn_ < P) ? cl.map_shared_rank(box, sn_ / spc) : nullptr;
  T* to_prev = (active && s >= 1) ? cl.map_shared_rank(box, sp_ / spc) : nullptr;
  int* id_next = (active && sn_ < P) ? cl.map_shared_rank(&mb_id[0][0][0], sn_ / spc) : nullptr;
  int* id_prev = (active && s >= 1) ? cl.map_shared_rank(&mb_id[0][0][0], sp_ / spc) : nullptr;
  T* nr_next = (active && sn_ < P) ? cl.map_shared_rank(&mb_nrm[0][0][0], sn_ / spc) : nullptr;
  T* nr_prev = (active && s >= 1) ? cl.map_shared_rank(&mb_nrm[0][0][0], sp_ / spc) : nullptr;
  T* sc_next = (active && sn_ < P) ? cl.map_shared_rank(&mb_scl[0][0][0], sn_ / spc) : nullptr;
  T* sc_prev = (active && s >= 1) ? cl.map_shared_rank(&mb_scl[0][0][0], sp_ / spc) : nullptr;
  // fold the scales into the columns (FP64)
  auto fold = [&]() {
    if constexpr (kTrack) {
      if (active && (da != (T)1 || db != (T)1)) {
#pragma unroll
        for (int e = 0; e < EPL; e++) {
          xa[e] *= da;
          xb[e] *= db;
          ja[e] *= da;
          jb[e] *= db;
        }
      }
      da = db = (T)1;
    }
  };
  cl.sync();  // every CTA has read its homes before anything is rotated
  for (int sweep = 0; sweep < 80 && c > 1; sweep++) {
    if (threadIdx.x == 0) *flag_local = 0;
    fold();
    na = nb = (T)-1;  // exact norms at the start of every sweep
    __syncthreads();
    for (int t = 0; t < cp - 1; t++) {
      const int buf = t & 1;
      T al = 0, be = 0, ga = 0, cs = 1, sn = 0, tt = 0;
      bool swp = false, rot = false;
      if (active) {
        swp = ida > idb;  // orientation: lower column id is "x"
        if constexpr (kTrack) {
          if (na < (T)0) { na = warp_dot<T, EPL>(xa, xa) * (da * da); n_dot++; }
          if (nb < (T)0) { nb = warp_dot<T, EPL>(xb, xb) * (db * db); n_dot++; }
          ga = warp_dot<T, EPL>(xa, xb) * (da * db);
          n_dot++;
        } else {
          n_dot += 3;
          T saa = 0, sbb = 0, sab = 0;
#pragma unroll
          for (int e = 0; e < EPL; e++) {
            saa += xa[e] * xa[e];
            sbb += xb[e] * xb[e];
            sab += xa[e] * xb[e];
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            saa += __shfl_xor_sync(0xffffffffu, saa, o);
            sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
            sab += __shfl_xor_sync(0xffffffffu, sab, o);
          }
          na = saa;
          nb = sbb;
          ga = sab;
        }
        al = swp ? nb : na;
        be = swp ? na : nb;
      }
      if constexpr (kTrack) {
        if (active && lane == 0) {
          sc_in[warp][0] = al;
          sc_in[warp][1] = be;
          sc_in[warp][2] = ga;
          sc_in[warp][3] = da;
          sc_in[warp][4] = db;
        }
        __syncthreads();
        if (warp == 0 && lane < nact) {
          T c_ = 1, s_ = 0, t_ = 0, r1 = 0, r2 = 0;
          if (!jacobi_angle<T>(sc_in[lane][0], sc_in[lane][1], sc_in[lane][2], tol, c_, s_, t_)) {
            t_ = 0;
          } else {
            const T d_a = sc_in[lane][3], d_b = sc_in[lane][4];
            r1 = t_ * (d_b / d_a);
            r2 = t_ * (d_a / d_b);
          }
          sc_out[lane][0] = c_;
          sc_out[lane][1] = r1;
          sc_out[lane][2] = r2;
          sc_out[lane][3] = t_;
        }
        __syncthreads();
        if (active) {
          cs = sc_out[warp][0];
          sn = sc_out[warp][1];  // t d_b / d_a (FP64 scaled form)
          tt = sc_out[warp][3];
          rot = tt != (T)0;
        }
      } else {
        if (active) rot = jacobi_angle<T>(al, be, ga, tol, cs, sn, tt);
      }
      if (active) {
        if (rot) {
          n_rot++;
          if constexpr (kTrack) {
            // scaled rotation: x_a -= f1 x_b, x_b += f2 x_a (old x_a)
            const T f1 = swp ? -sn : sn;
            const T f2 = swp ? -sc_out[warp][2] : sc_out[warp][2];
#pragma unroll
            for (int e = 0; e < EPL; e++) {
              const T x0 = xa[e], y0 = xb[e];
              xa[e] = fma(-f1, y0, x0);
              xb[e] = fma(f2, x0, y0);
            }
            if (withJ) {
#pragma unroll
              for (int e = 0; e < EPL; e++) {
                const T j0 = ja[e], k0 = jb[e];
                ja[e] = fma(-f1, k0, j0);
                jb[e] = fma(f2, j0, k0);
              }
            }
            da *= cs;
            db *= cs;
          } else {
            if (swp) sn = -sn;
#pragma unroll
            for (int e = 0; e < EPL; e++) {
              const T x0 = xa[e], y0 = xb[e];
              xa[e] = cs * x0 - sn * y0;
              xb[e] = sn * x0 + cs * y0;
            }
            if (withJ) {
#pragma unroll
              for (int e = 0; e < EPL; e++) {
                const T j0 = ja[e], k0 = jb[e];
                ja[e] = cs * j0 - sn * k0;
                jb[e] = sn * j0 + cs * k0;
              }
            }
          }
          if constexpr (kTrack) {
            const T nx = al - tt * ga, ny = be + tt * ga;  // lower-id column, the other
            const T nxa = swp ? ny : nx, nxb = swp ? nx : ny;
            const T oa = na, ob = nb;
            na = (nxa < (T)0.01 * oa) ? (T)-1 : nxa;
            nb = (nxb < (T)0.01 * ob) ? (T)-1 : nxb;
          }
          if (lane == 0) *flag_local = 1;
        }
        if (P > 1) {
          if (to_next) {  // slot 0 sends its second column forward, the others their first
            T* dx = mbox(to_next, buf, sn_ % spc, 0, 0);
            T* dj = mbox(to_next, buf, sn_ % spc, 0, 1);
#pragma unroll
            for (int e = 0; e < EPL; e++) dx[lane + 32 * e] = s == 0 ? xb[e] : xa[e];
            if (withJ) {
#pragma unroll
              for (int e = 0; e < EPL; e++) dj[lane + 32 * e] = s == 0 ? jb[e] : ja[e];
            }
            if (lane == 0) {
              id_next[(buf * 16 + sn_ % spc) * 2 + 0] = s == 0 ? idb : ida;
              nr_next[(buf * 16 + sn_ % spc) * 2 + 0] = s == 0 ? nb : na;
              sc_next[(buf * 16 + sn_ % spc) * 2 + 0] = s == 0 ? db : da;
            }
          }
          if (to_prev) {  // second column backward
            T* dx = mbox(to_prev, buf, sp_ % spc, 1, 0);
            T* dj = mbox(to_prev, buf, sp_ % spc, 1, 1);
#pragma unroll
            for (int e = 0; e < EPL; e++) dx[lane + 32 * e] = xb[e];
            if (withJ) {
#pragma unroll
              for (int e = 0; e < EPL; e++) dj[lane + 32 * e] = jb[e];
            }
            if (lane == 0) {
              id_prev[(buf * 16 + sp_ % spc) * 2 + 1] = idb;
              nr_prev[(buf * 16 + sp_ % spc) * 2 + 1] = nb;
              sc_prev[(buf * 16 + sp_ % spc) * 2 + 1] = db;
            }
          }
        }
      }
      cl.sync();
      if (active && P > 1) {
        const int ls = warp;
        if (s == P - 1) {  // last slot: its first column becomes its second
#pragma unroll
          for (int e = 0; e < EPL; e++) {
            xb[e] = xa[e];
            jb[e] = ja[e];
          }
          idb = ida;
          nb = na;
          db = da;
        }
        if (s >= 1) {  // new first column from slot s-1
          const T* sx = mbox(box, buf, ls, 0, 0);
          const T* sj = mbox(box, buf, ls, 0, 1);
#pragma unroll
          for (int e = 0; e < EPL; e++) xa[e] = sx[lane + 32 * e];
          if (withJ) {
#pragma unroll
            for (int e = 0; e < EPL; e++) ja[e] = sj[lane + 32 * e];
          }
          ida = mb_id[buf][ls][0];
          na = mb_nrm[buf][ls][0];
          da = mb_scl[buf][ls][0];
        }
        if (s < P - 1) {  // new second column from slot s+1
          const T* sx = mbox(box, buf, ls, 1, 0);
          const T* sj = mbox(box, buf, ls, 1, 1);
#pragma unroll
          for (int e = 0; e < EPL; e++) xb[e] = sx[lane + 32 * e];
          if (withJ) {
#pragma unroll
            for (int e = 0; e < EPL; e++) jb[e] = sj[lane + 32 * e];
          }
          idb = mb_id[buf][ls][1];
          nb = mb_nrm[buf][ls][1];
          db = mb_scl[buf][ls][1];
        }
      }
    }
    // the last round ended with a cluster barrier, so every flag is final
    int any = 0;
    for (int rr = 0; rr < (int)cl.num_blocks(); rr++) any |= *cl.map_shared_rank(flag_local, rr);
    cl.sync();  // nobody resets its flag before all have read it
    if (!any) break;
  }
  fold();
  if (active && lane == 0) {
    // per dot 2c; per rotation of X (and J) 4c scaled (FP64) or 6c
    const unsigned long long rotf = (kTrack ? 4ull : 6ull) * (unsigned long long)c * (withJ ? 2 : 1);
    atomicAdd(&g_svd_work[sizeof(T) == 4], n_dot * 2ull * c + n_rot * rotf);
  }
  if (active) {
#pragma unroll
    for (int e = 0; e < EPL; e++) {
      const int i = lane + 32 * e;
      if (i < c) {
        if (ida < c) {
          xcol(ida)[i] = xa[e];
          if (withJ) jcol(ida)[i] = ja[e];
        }
        if (idb < c) {
          xcol(idb)[i] = xb[e];
          if (withJ) jcol(idb)[i] = jb[e];
        }
      }
    }
  }
  cl.sync();
}

// dynamic shared memory: X and J home columns (slots x c each).  T is the
// working precision: double for the FP64 path; float for the mixed path,
// whose callers re-orthonormalise the returned factor in FP64.
template <typename T, int EPL>
__global__ void __launch_bounds__(512, 1) k_svd_cluster_t(SvdArgs a, int use_smem,
                                                          long long dyn_elems) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  extern __shared__ double dsm_raw[];
  T* dsm = (T*)dsm_raw;
  __shared__ double sh[32];
  __shared__ int flag_local;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (a.skip && *a.skip) return;
  const int m = a.inT ? axis_len(a.M.cols) : axis_len(a.M.rows);
  const int N = a.inT ? axis_len(a.M.rows) : axis_len(a.M.cols);
  const int mrl = dval(a.M.rows.lact), mcl = dval(a.M.cols.lact);
  const bool wide = (m <= N);
  const int Rt = wide ? N : m;
  const int c = wide ? m : N;
  const int slots = (c + CL - 1) / CL;
  {
    const Axis& fr = a.inT ? a.M.cols : a.M.rows;
    const Axis& fc = a.inT ? a.M.rows : a.M.cols;
    const int us_r = a.usT ? a.US.cols.hcap * a.US.cols.lcap : a.US.rows.hcap * a.US.rows.lcap;
    const int us_c = a.usT ? a.US.rows.hcap * a.US.rows.lcap : a.US.cols.hcap * a.US.cols.lcap;
    const int vt_r = a.vtT ? a.VT.cols.hcap * a.VT.cols.lcap : a.VT.rows.hcap * a.VT.rows.lcap;
    const int vt_c = a.vtT ? a.VT.rows.hcap * a.VT.rows.lcap : a.VT.cols.hcap * a.VT.cols.lcap;
    const int rmax = min(c, min(a.chi, dval(a.rank_limit)));
    const long long need = (long long)Rt * c * 2 + (long long)c * c * 2 + 4LL * c + 2 + (c + 1) / 2;
    const bool bad = !view_ok_c(a.M) || !view_ok_c(a.US) || !view_ok_c(a.VT) || m < 1 ||
                     N < 1 || m > fr.hcap * fr.lcap || N > fc.hcap * fc.lcap || m > us_r ||
                     max(rmax, 1) > us_c || max(rmax, 1) > vt_r || N > vt_c ||
                     need > a.work_len || (use_smem && slots * c > use_smem);
    if (bad) {
      if (rank == 0 && threadIdx.x == 0 && a.err) atomicOr(a.err, QTT_DEVERR_SHAPE);
      return;
    }
  }
  // work layout (in units of T, then doubles for the FP64 bookkeeping)
  T* Tm = (T*)a.work;                   // Rt x c
  T* Xg = Tm + (size_t)Rt * c;          // c x c   (used when not in shared memory)
  T* Jg = Xg + (size_t)c * c;           // c x c
  T* Bw = Jg + (size_t)c * c;           // Rt x c
  T* tau = Bw + (size_t)Rt * c;
  T* diag = tau + c;
  double* sig = a.work + ((size_t)(2 * Rt * c + 2 * c * c + 2 * c) * sizeof(T) + 7) / 8;
  double* tail = sig + c;
  int* perm = (int*)(tail + c + 1);
  // home of column i: CTA i % CL, slot i / CL
  T* Xs = dsm;
  T* Js = dsm + (size_t)slots * c;
  auto xcol = [&](int i) -> T* {
    if (!use_smem) return Xg + (size_t)i * c;
    return cl.map_shared_rank(Xs, i % CL) + (size_t)(i / CL) * c;
  };
  auto jcol = [&](int i) -> T* {
    if (!use_smem) return Jg + (size_t)i * c;
    return cl.map_shared_rank(Js, i % CL) + (size_t)(i / CL) * c;
  };
  bool badv = false;
  for (int j = rank; j < c; j += CL)
    for (int i = threadIdx.x; i < Rt; i += blockDim.x) {
      const int fi = wide ? j : i, fj = wide ? i : j;
      const long long off = a.inT ? voff(a.M, fj, fi, mrl, mcl) : voff(a.M, fi, fj, mrl, mcl);
      const double v = a.M.ptr[off];
      badv |= !isfinite(v);
      Tm[(size_t)j * Rt + i] = (T)v;
    }
  if (badv && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
  cl.sync();
  // the whole dynamic shared memory is scratch until the Jacobi starts
  householder_any_cl<T>(cl, Tm, Rt, c, tau, diag, sh, rank, CL, dsm, dyn_elems);
  // X = R^T into the home columns (for both orientations: Jacobi on the
  // columns of R^T needs about half the sweeps of Jacobi on R's columns
  // here, the preconditioning effect of the QR); J = I
  for (int i = rank; i < c; i += CL) {
    T* x = xcol(i);
    T* jj = jcol(i);
    for (int e = threadIdx.x; e < c; e += blockDim.x) {
      T rv = 0;  // X(e, i) = R(i, e)
      if (i == e) rv = diag[i];
      else if (i < e) rv = Tm[(size_t)e * Rt + i];
      x[e] = rv;
      jj[e] = (e == i) ? (T)1 : (T)0;
    }
  }
  cl.sync();
  const T tol = Prec<T>::cos_tol(c);
  const int cp = c + (c & 1);
  // J is needed for V = Q J (wide) and for U S = Q J S (tall); a tall
  // factorisation whose U S is not wanted needs neither J nor Q
  const bool needJ = wide || !a.no_us;
  const int spc = ((cp / 2) + CL - 1) / CL;
  bool done = false;
  if constexpr (EPL > 0) {
    if (c <= 32 * EPL && spc <= nw && spc <= 16 && !use_smem) {
      // the homes are in global memory and the whole dynamic shared memory
      // holds the mailboxes (sized by the launcher for the capacity shape)
      jacobi_systolic<T, EPL>(cl, xcol, jcol, c, tol, dsm, spc, rank, &flag_local, needJ);
      done = true;
    }
  }
  if (!done)
  for (int sweep = 0; sweep < 80 && c > 1; sweep++) {
    if (threadIdx.x == 0) flag_local = 0;
    __syncthreads();
    for (int t = 0; t < cp - 1; t++) {
      for (int k = rank + warp * CL; k < cp / 2; k += nw * CL) {
        int p = rr_pos_c(k, t, cp), q = rr_pos_c(cp - 1 - k, t, cp);
        if (p >= c || q >= c) continue;
        if (p > q) { const int s_ = p; p = q; q = s_; }
        T* x = xcol(p);
        T* y = xcol(q);
        T al = 0, be = 0, ga = 0;
#pragma unroll 4
        for (int i = lane; i < c; i += 32) {
          const T xi = x[i], yi = y[i];
          al += xi * xi;
          be += yi * yi;
          ga += xi * yi;
        }
        al = warp_sum_c(al);
        be = warp_sum_c(be);
        ga = warp_sum_c(ga);
        if (ga != (T)0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          // rotation angle in the working precision
          const T zeta = (be - al) / ((T)2 * ga);
          const T tt = copysign((T)1, zeta) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
          const T cs = (T)1 / sqrt((T)1 + tt * tt), sn = cs * tt;
          for (int i = lane; i < c; i += 32) {
            const T xi = x[i], yi = y[i];
            x[i] = cs * xi - sn * yi;
            y[i] = sn * xi + cs * yi;
          }
          T* jx = jcol(p);
          T* jy = jcol(q);
          for (int i = lane; i < c; i += 32) {
            const T xi = jx[i], yi = jy[i];
            jx[i] = cs * xi - sn * yi;
            jy[i] = sn * xi + cs * yi;
          }
          if (lane == 0) flag_local = 1;
        }
      }
      cl.sync();
    }
    // cluster-wide "any rotation in this sweep": read every CTA's flag
    // (the last round ended with a cluster barrier, so the flags are final)
    int any = 0;
    for (int rr = 0; rr < CL; rr++) any |= *cl.map_shared_rank(&flag_local, rr);
    cl.sync();  // nobody resets its flag before all have read it
    if (!any) break;
  }
  // singular values (home columns), order, rank (computed by every CTA alike)
  for (int k = rank + warp * CL; k < c; k += nw * CL) {
    const T* x = xcol(k);
    double s = 0.0;  // FP64 sum of squares: the truncation weights
    for (int i = lane; i < c; i += 32) s += (double)x[i] * (double)x[i];
    s = warp_sum_c(s);
    if (lane == 0) sig[k] = sqrt(s);
  }
  cl.sync();
  if (rank == 0) {
    for (int k = threadIdx.x; k < c; k += blockDim.x) {
      int rk = 0;
      const double sk = isnan(sig[k]) ? -1.0 : sig[k];
      for (int j = 0; j < c; j++) {
        const double sj = isnan(sig[j]) ? -1.0 : sig[j];
        rk += (sj > sk) || (sj == sk && j < k);
      }
      perm[rk] = k;
    }
    bool nan_seen = false;
    for (int k = threadIdx.x; k < c; k += blockDim.x) nan_seen |= !isfinite(sig[k]);
    if (nan_seen && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
    __syncthreads();
    if (threadIdx.x == 0) {
      int r;
      const int lim = dval(a.rank_limit);
      if (a.eps >= 0.0) {
        tail[c] = 0.0;
        for (int j = c - 1; j >= 0; j--) {
          const double s = sig[perm[j]];
          tail[j] = tail[j + 1] + (a.gram ? s : s * s);
        }
        if (a.total_weight) {  // weight outside M's subspace, counted as discarded
          const double extra = fmax(0.0, *a.total_weight - tail[0]);
          for (int j = 0; j <= c; j++) tail[j] += extra;
        }
        const double total = tail[0];
        r = c;
        if (total == 0.0) {
          r = 1;
        } else {
          const double thr = a.eps * a.eps * total;
          for (int cand = 1; cand <= c; cand++)
            if (tail[cand] <= thr) { r = cand; break; }
        }
      } else {
        r = c;
      }
      r = max(1, min(min(r, a.chi), min(lim, c)));
      tail[c] = (double)r;  // publish r
      if (a.r_out) *a.r_out = r;
    }
    if (a.sv_out)
      for (int k = threadIdx.x; k < c; k += blockDim.x) a.sv_out[k] = sig[perm[k]];
  }
  cl.sync();
  const int r = (int)(*(volatile double*)(tail + c));
  // X J = U_x S with X = R^T.  Wide (M = R^T Q^T): U S = X and V = Q J.
  // Tall (M = Q R = (Q J) S U_x^T): U S = Q (J S) and V = U_x = X / S.
  // Bw = [J_perm (times S when tall) ; 0], own columns, then Q applied.
  if (rank == 0 && threadIdx.x == 0) {
    const double R_ = Rt, c_ = c;
    double f = 2.0 * R_ * c_ * c_ - 2.0 / 3.0 * c_ * c_ * c_;  // Householder QR
    if (needJ) f += 4.0 * R_ * c_ * r;                          // Q applied to r columns
    atomicAdd(&g_svd_work[sizeof(T) == 4], (unsigned long long)f);
  }
  if (needJ) {
    for (int k = rank; k < r; k += CL) {
      const T* src = jcol(perm[k]);
      const T sc = wide ? (T)1 : (T)sig[perm[k]];
      for (int i = threadIdx.x; i < Rt; i += blockDim.x)
        Bw[(size_t)k * Rt + i] = (i < c) ? src[i] * sc : (T)0;
    }
    __syncthreads();
    apply_reflectors_cl<T>(Tm, Rt, c, tau, Bw, r, false, rank, CL);
  }
  cl.sync();
  if (!a.no_us) zero_view_cl(a.US, rank, CL);
  zero_view_cl(a.VT, rank, CL);
  cl.sync();
  const int url = dval(a.US.rows.lact), ucl = dval(a.US.cols.lact);
  const int vrl = dval(a.VT.rows.lact), vcl = dval(a.VT.cols.lact);
  for (int k = rank; k < r; k += CL) {
    const T* xs = xcol(perm[k]);
    for (int i = threadIdx.x; i < m && !a.no_us; i += blockDim.x) {
      const double v = wide ? (double)xs[i] : (double)Bw[(size_t)k * Rt + i];
      a.US.ptr[a.usT ? voff(a.US, k, i, url, ucl) : voff(a.US, i, k, url, ucl)] = v;
    }
    // a zero singular value (all-zero input, or a kept rank above the
    // numerical rank) leaves a zero row: its U S column is zero as well
    const double sk = sig[perm[k]];
    const double inv = sk > 0.0 ? 1.0 / sk : 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const double v = wide ? (double)Bw[(size_t)k * Rt + j] : (double)xs[j] * inv;
      a.VT.ptr[a.vtT ? voff(a.VT, j, k, vrl, vcl) : voff(a.VT, k, j, vrl, vcl)] = v;
    }
  }
  cl.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

int g_cluster_size = -1;  // 16, 8 or 0 (no cluster launch)

// every cluster SVD instantiation: <precision, elements per lane> (0 = the
// scalar tournament with homes in distributed shared memory)
template <typename F>
void for_each_svd_kernel(F f) {
  f((const void*)k_svd_cluster_t<double, 0>);
  f((const void*)k_svd_cluster_t<double, 2>);
  f((const void*)k_svd_cluster_t<double, 4>);
  f((const void*)k_svd_cluster_t<double, 8>);
  f((const void*)k_svd_cluster_t<float, 0>);
  f((const void*)k_svd_cluster_t<float, 2>);
  f((const void*)k_svd_cluster_t<float, 4>);
  f((const void*)k_svd_cluster_t<float, 8>);
}

int pick_cluster_size_once();
int pick_cluster_size() {
  static std::once_flag once;
  std::call_once(once, [] { pick_cluster_size_once(); });
  return g_cluster_size;
}

int pick_cluster_size_once() {
  g_cluster_size = 0;
  const int want[2] = {16, 8};
  for (int w : want) {
    if (w == 16) {
      bool ok = cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                     1) == cudaSuccess;
      for_each_svd_kernel([&](const void* k) {
        ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                       cudaSuccess;
      });
      if (!ok) {
        cudaGetLastError();
        continue;
      }
    }
    for_each_svd_kernel([&](const void* k) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(w);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = 200 * 1024;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = w;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)k_svd_cluster_t<double, 8>,
                                       &cfg) == cudaSuccess &&
        nclusters > 0) {
      g_cluster_size = w;
      break;
    }
    cudaGetLastError();
  }
  return g_cluster_size;
}


// shared-memory scratch of the blocked Householder: up to 16 panel columns
// of mcap rows, within the 200 KB the kernels are configured for
long long qr_scratch_elems(int mcap, size_t es) {
  static const bool unblocked = getenv("QTT_QR_UNBLOCKED") != nullptr;
  if (unblocked) return 0;
  const long long cap = (long long)(200 * 1024) / (long long)es;
  const long long want = 16LL * mcap;
  return want < cap ? want : cap;
}

void launch_svd_kernel(const void* kern, int CL, size_t smem, cudaStream_t s, SvdArgs a,
                       int use_smem, int Rcap, size_t es) {
  // room for the blocked Householder's panels as well (scratch before the
  // Jacobi; FP32 only)
  const long long qr_elems = es == sizeof(float) ? qr_scratch_elems(Rcap, es) : 0;
  if ((size_t)qr_elems * es > smem) smem = (size_t)qr_elems * es;
  long long dyn_elems = (long long)(smem / es);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[3] = {(void*)&a, (void*)&use_smem, (void*)&dyn_elems};
  QTT_CUDA_CHECK(cudaLaunchKernelExC(&cfg, kern, args));
}

}  // namespace

bool cluster_linalg_available() { return pick_cluster_size() > 0; }

// Returns false when no cluster launch is possible (the caller falls back).
bool launch_qr_cluster(const QrArgs& a, int mcap, cudaStream_t s) {
  const int CL = pick_cluster_size();
  if (CL <= 0) return false;
  const long long elems = 0;  // the FP64 QR factors column at a time (see householder_any_cl)
  (void)mcap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = (size_t)elems * sizeof(double);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  pre_launch(s);
  QTT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_qr_cluster, a, elems));
  return true;
}

bool launch_svd_cluster(const SvdArgs& a, int mcap, int ncap, cudaStream_t s, bool fp32) {
  const int CL = pick_cluster_size();
  if (CL <= 0) return false;
  const int c = mcap < ncap ? mcap : ncap;  // capacity bound on the square factor
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  const size_t limit = 200 * 1024;
  static const bool scalar_only = getenv("QTT_SCALAR_JACOBI") != nullptr;
  // preferred: the systolic kernel, columns in registers, mailboxes in
  // shared memory (2 parities x slots per CTA x 2 columns x (X, J))
  const int epl = c <= 64 ? 2 : c <= 128 ? 4 : c <= 256 ? 8 : 0;
  const int spc = ((c + 1) / 2 + CL - 1) / CL;
  const size_t need_sys = (size_t)8 * spc * 32 * epl * es;
  if (!scalar_only && epl > 0 && spc <= 16 && need_sys <= limit) {
    pre_launch(s);
    const void* k = nullptr;
    if (fp32) k = epl == 2 ? (const void*)k_svd_cluster_t<float, 2>
                 : epl == 4 ? (const void*)k_svd_cluster_t<float, 4>
                            : (const void*)k_svd_cluster_t<float, 8>;
    else k = epl == 2 ? (const void*)k_svd_cluster_t<double, 2>
           : epl == 4 ? (const void*)k_svd_cluster_t<double, 4>
                      : (const void*)k_svd_cluster_t<double, 8>;
    launch_svd_kernel(k, CL, need_sys, s, a, 0, mcap > ncap ? mcap : ncap, es);
    return true;
  }
  int use_smem = 0;
  size_t smem = 0;
  const int slots = (c + CL - 1) / CL;
  const size_t need = (size_t)2 * slots * c * es + 64;
  if (need <= limit) {
    use_smem = slots * c;
    smem = need;
  }
  pre_launch(s);
  launch_svd_kernel(fp32 ? (const void*)k_svd_cluster_t<float, 0> : (const void*)k_svd_cluster_t<double, 0>,
                    CL, smem, s, a, use_smem, mcap > ncap ? mcap : ncap, es);
  return true;
}
