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

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

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

__global__ void __launch_bounds__(512) k_qr_cluster(QrArgs a) {
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
  householder_cl<double>(cl, W, m, c, tau, diag, sh, rank, CL);
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


// Block one-sided Jacobi across the cluster.  The c columns of X (and of the
// rotation accumulator J) are cut into 2 CL blocks of b columns (zero
// columns pad the last ones).  Tournament position p (0 .. 2CL-1) lives in
// CTA p (p < CL, slot 0) or CTA 2CL-1-p (slot 1), so CTA k pairs positions k
// and 2CL-1-k.  In each outer round a CTA rotates every pair of its 2b
// columns in its own shared memory (an inner round-robin sweep), then all
// blocks advance one position (position 0 stays) by copying into the
// destination CTA's other buffer; one cluster barrier per outer round.
// 2CL-1 outer rounds meet every pair of blocks once (one sweep).  X and J are
// read from and written back to global memory column-major (c x c).
template <typename T>
__device__ void jacobi_blocks(cg::cluster_group& cl, T* Xg, T* Jg, int c, int b, T* sm, T tol,
                              int rank, int CL) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int blk[2][2];
  __shared__ int flag_b;
  const size_t blk_elems = (size_t)b * c;                   // one block, X or J
  auto buf = [&](int which, int slot, int xj) -> T* {       // local pointer
    return sm + (((size_t)which * 2 + slot) * 2 + xj) * blk_elems;
  };
  const int P2 = 2 * CL;
  int cur = 0;
  for (int slot = 0; slot < 2; slot++) {
    const int beta = slot == 0 ? rank : P2 - 1 - rank;
    if (threadIdx.x == 0) blk[0][slot] = beta;
    for (int col = 0; col < b; col++) {
      const int gi = beta * b + col;
      T* x = buf(0, slot, 0) + (size_t)col * c;
      T* jj = buf(0, slot, 1) + (size_t)col * c;
      for (int e = threadIdx.x; e < c; e += blockDim.x) {
        x[e] = gi < c ? Xg[(size_t)gi * c + e] : (T)0;
        jj[e] = gi < c ? Jg[(size_t)gi * c + e] : (T)0;
      }
    }
  }
  cl.sync();
  const int cq = 2 * b;  // local columns, even
  for (int sweep = 0; sweep < 80 && c > 1; sweep++) {
    if (threadIdx.x == 0) flag_b = 0;
    __syncthreads();
    for (int t = 0; t < P2 - 1; t++) {
      for (int it = 0; it < cq - 1; it++) {
        for (int k = warp; k < b; k += nw) {
          int p = rr_pos_c(k, it, cq), q = rr_pos_c(cq - 1 - k, it, cq);
          if (p > q) { const int s_ = p; p = q; q = s_; }
          T* x = buf(cur, p / b, 0) + (size_t)(p % b) * c;
          T* y = buf(cur, q / b, 0) + (size_t)(q % b) * c;
          T al = 0, be = 0, ga = 0;
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
            const double zeta = ((double)be - (double)al) / (2.0 * (double)ga);
            const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double csd = 1.0 / sqrt(1.0 + tt * tt);
            const T cs = (T)csd, sn = (T)(csd * tt);
            for (int i = lane; i < c; i += 32) {
              const T xi = x[i], yi = y[i];
              x[i] = cs * xi - sn * yi;
              y[i] = sn * xi + cs * yi;
            }
            T* jx = buf(cur, p / b, 1) + (size_t)(p % b) * c;
            T* jy = buf(cur, q / b, 1) + (size_t)(q % b) * c;
            for (int i = lane; i < c; i += 32) {
              const T xi = jx[i], yi = jy[i];
              jx[i] = cs * xi - sn * yi;
              jy[i] = sn * xi + cs * yi;
            }
            if (lane == 0) flag_b = 1;
          }
        }
        __syncthreads();
      }
      // advance every block one tournament position (position 0 stays)
      for (int slot = 0; slot < 2; slot++) {
        const int pos = slot == 0 ? rank : P2 - 1 - rank;
        const int np = pos == 0 ? 0 : (pos % (P2 - 1)) + 1;
        const int dcta = np < CL ? np : P2 - 1 - np, dslot = np < CL ? 0 : 1;
        T* dst = cl.map_shared_rank(buf(cur ^ 1, dslot, 0), dcta);
        const T* src = buf(cur, slot, 0);
        for (size_t e = threadIdx.x; e < 2 * blk_elems; e += blockDim.x) dst[e] = src[e];
        if (threadIdx.x == 0) *cl.map_shared_rank(&blk[cur ^ 1][dslot], dcta) = blk[cur][slot];
      }
      cl.sync();
      cur ^= 1;
    }
    int any = 0;
    for (int rr = 0; rr < CL; rr++) any |= *cl.map_shared_rank(&flag_b, rr);
    cl.sync();
    if (!any) break;
  }
  for (int slot = 0; slot < 2; slot++) {
    const int beta = blk[cur][slot];
    for (int col = 0; col < b; col++) {
      const int gi = beta * b + col;
      if (gi >= c) continue;
      const T* x = buf(cur, slot, 0) + (size_t)col * c;
      const T* jj = buf(cur, slot, 1) + (size_t)col * c;
      for (int e = threadIdx.x; e < c; e += blockDim.x) {
        Xg[(size_t)gi * c + e] = x[e];
        Jg[(size_t)gi * c + e] = jj[e];
      }
    }
  }
  cl.sync();
}

// dynamic shared memory: X and J home columns (slots x c each).  T is the
// working precision: double for the FP64 path; float for the mixed path,
// whose callers re-orthonormalise the returned factor in FP64.
template <typename T>
__global__ void __launch_bounds__(512) k_svd_cluster_t(SvdArgs a, int use_smem, int bcols) {
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
                     need > a.work_len || (use_smem && slots * c > use_smem) ||
                     (bcols && 2 * CL * bcols < c);
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
  householder_cl<T>(cl, Tm, Rt, c, tau, diag, sh, rank, CL);
  // X = R^T (wide) or R (tall) into the home columns; J = I
  for (int i = rank; i < c; i += CL) {
    T* x = xcol(i);
    T* jj = jcol(i);
    for (int e = threadIdx.x; e < c; e += blockDim.x) {
      const int p = wide ? i : e, q = wide ? e : i;  // X(e, i) = R(p, q)
      T rv = 0;
      if (p == q) rv = diag[p];
      else if (p < q) rv = Tm[(size_t)q * Rt + p];
      x[e] = rv;
      jj[e] = (e == i) ? (T)1 : (T)0;
    }
  }
  cl.sync();
  const T tol = Prec<T>::cos_tol(c);
  const int cp = c + (c & 1);
  if (bcols) {
    jacobi_blocks<T>(cl, Xg, Jg, c, bcols, dsm, tol, rank, CL);
  } else
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
          tail[j] = tail[j + 1] + s * s;
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
  // Bw = [J_perm ; 0] (wide: V = Q J) or [X_perm ; 0] (tall: U S = Q X), own columns
  for (int k = rank; k < r; k += CL) {
    const T* src = wide ? jcol(perm[k]) : xcol(perm[k]);
    for (int i = threadIdx.x; i < Rt; i += blockDim.x)
      Bw[(size_t)k * Rt + i] = (i < c) ? src[i] : (T)0;
  }
  __syncthreads();
  apply_reflectors_cl<T>(Tm, Rt, c, tau, Bw, r, false, rank, CL);
  cl.sync();
  zero_view_cl(a.US, rank, CL);
  zero_view_cl(a.VT, rank, CL);
  cl.sync();
  const int url = dval(a.US.rows.lact), ucl = dval(a.US.cols.lact);
  const int vrl = dval(a.VT.rows.lact), vcl = dval(a.VT.cols.lact);
  for (int k = rank; k < r; k += CL) {
    const T* xs = xcol(perm[k]);
    const T* js = jcol(perm[k]);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double v = wide ? (double)xs[i] : (double)Bw[(size_t)k * Rt + i];
      a.US.ptr[a.usT ? voff(a.US, k, i, url, ucl) : voff(a.US, i, k, url, ucl)] = v;
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const double v = wide ? (double)Bw[(size_t)k * Rt + j] : (double)js[j];
      a.VT.ptr[a.vtT ? voff(a.VT, j, k, vrl, vcl) : voff(a.VT, k, j, vrl, vcl)] = v;
    }
  }
  cl.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

int g_cluster_size = -1;  // 16, 8 or 0 (no cluster launch)

int pick_cluster_size() {
  if (g_cluster_size >= 0) return g_cluster_size;
  g_cluster_size = 0;
  const int want[2] = {16, 8};
  for (int w : want) {
    if (w == 16) {
      if (cudaFuncSetAttribute(k_svd_cluster_t<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
              cudaSuccess ||
          cudaFuncSetAttribute(k_svd_cluster_t<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
              cudaSuccess ||
          cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
              cudaSuccess) {
        cudaGetLastError();
        continue;
      }
    }
    cudaFuncSetAttribute(k_svd_cluster_t<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_svd_cluster_t<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_svd_cluster_t<double>, &cfg) == cudaSuccess &&
        nclusters > 0) {
      g_cluster_size = w;
      break;
    }
    cudaGetLastError();
  }
  return g_cluster_size;
}

template <typename K, typename Args>
void launch_cluster(K kern, int CL, size_t smem, cudaStream_t s, Args a) {
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
  QTT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, a));
}

template <typename K>
void launch_cluster2(K kern, int CL, size_t smem, cudaStream_t s, SvdArgs a, int use_smem,
                     int bcols) {
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
  QTT_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, a, use_smem, bcols));
}

}  // namespace

bool cluster_linalg_available() { return pick_cluster_size() > 0; }

// Returns false when no cluster launch is possible (the caller falls back).
bool launch_qr_cluster(const QrArgs& a, cudaStream_t s) {
  const int CL = pick_cluster_size();
  if (CL <= 0) return false;
  pre_launch(s);
  launch_cluster(k_qr_cluster, CL, 0, s, a);
  return true;
}

bool launch_svd_cluster(const SvdArgs& a, int mcap, int ncap, cudaStream_t s, bool fp32) {
  const int CL = pick_cluster_size();
  if (CL <= 0) return false;
  const int c = mcap < ncap ? mcap : ncap;  // capacity bound on the square factor
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  const size_t limit = 200 * 1024;
  // block Jacobi measured slower than the scalar tournament on this GPU
  // (intra-block pairs are repeated every outer round); kept behind a switch
  static const bool use_block = getenv("QTT_BLOCK_JACOBI") != nullptr;
  // preferred: block Jacobi, double-buffered blocks in each CTA's memory
  const int b = (c + 2 * CL - 1) / (2 * CL);
  const size_t need_block = (size_t)8 * b * c * es + 64;
  int use_smem = 0, bcols = 0;
  size_t smem = 0;
  if (use_block && need_block <= limit) {
    bcols = b;
    smem = need_block;
  } else {
    const int slots = (c + CL - 1) / CL;
    const size_t need = (size_t)2 * slots * c * es + 64;
    if (need <= limit) {
      use_smem = slots * c;
      smem = need;
    }
  }
  pre_launch(s);
  if (fp32) launch_cluster2(k_svd_cluster_t<float>, CL, smem, s, a, use_smem, bcols);
  else launch_cluster2(k_svd_cluster_t<double>, CL, smem, s, a, use_smem, bcols);
  return true;
}
