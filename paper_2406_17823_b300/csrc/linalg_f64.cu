// FP64 factorisations, one CTA per problem, shapes read from device memory.
//
//  * Householder QR (Golub & Van Loan, Alg. 5.2.1 with explicit Q formed by
//    backward accumulation): the gauge step of every compression sweep
//    (Sec. II.C) and the centre shift of the projection sweep (App. B).
//  * SVD: Householder QR of the tall orientation, then one-sided (Hestenes)
//    Jacobi on the square triangular factor with round-robin pair ordering;
//    singular values sorted descending; rank by the per-bond truncation
//    rule (Sec. III.E) or by a cap alone (zip-up).  One-sided Jacobi gives
//    small singular values to high relative accuracy, which the eps tail
//    sums need at eps = 1e-12.
//
// Matrices are gathered into a column-major work buffer first, so outputs
// may alias the input storage.
#include <stdio.h>
#include <math.h>
#include <stdlib.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; i++) t += sh[i];  // same order in every thread
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place Householder QR of W (m x c, column-major, leading dim ldw).
// Reflector j: v_j in W[j:, j] (v_j[j] at W[j][j]), tau[j]; R[j][j] = diag[j],
// R[i][j] = W[i][j] for i < j.
__device__ void householder(double* W, int ldw, int m, int c, double* tau, double* diag,
                            double* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kmax = min(m, c);
  for (int j = 0; j < kmax; j++) {
    double* col = W + (size_t)j * ldw;
    double part = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) part += col[i] * col[i];
    const double nrm2 = block_sum(part, sh);
    const double x0 = col[j];
    __syncthreads();
    // A column whose squared norm is below 1e-280 is left as it is (no
    // reflection, R[j][j] = x0): its entries are < 1e-140, and forming the
    // reflector from them would overflow tau.
    double t = 0.0, alpha = x0;
    if (nrm2 > 1e-280 && isfinite(nrm2)) {
      const double nrm = sqrt(nrm2);
      alpha = (x0 >= 0.0) ? -nrm : nrm;
      t = 1.0 / (nrm * (nrm + fabs(x0)));
      if (threadIdx.x == 0) col[j] = x0 - alpha;
    }
    if (threadIdx.x == 0) {
      tau[j] = t;
      diag[j] = alpha;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int cc = j + 1 + warp; cc < c; cc += nw) {
        double* x = W + (size_t)cc * ldw;
        double s = 0.0;
        for (int i = j + lane; i < m; i += 32) s += col[i] * x[i];
        s = warp_sum(s) * t;
        for (int i = j + lane; i < m; i += 32) x[i] -= s * col[i];
      }
    }
    __syncthreads();
  }
}

// B (m x nb, column-major) <- H_0 H_1 ... H_{k-1} B.  When `identity_cols`
// the columns of B start as unit vectors e_cc, so H_j only touches cc >= j.
__device__ void apply_reflectors(const double* W, int ldw, int m, int k, const double* tau,
                                 double* B, int ldb, int nb, bool identity_cols) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = k - 1; j >= 0; j--) {
    const double t = tau[j];
    if (t != 0.0) {
      const double* v = W + (size_t)j * ldw;
      const int c0 = identity_cols ? j : 0;
      for (int cc = c0 + warp; cc < nb; cc += nw) {
        double* x = B + (size_t)cc * ldb;
        double s = 0.0;
        for (int i = j + lane; i < m; i += 32) s += v[i] * x[i];
        s = warp_sum(s) * t;
        for (int i = j + lane; i < m; i += 32) x[i] -= s * v[i];
      }
    }
    __syncthreads();
  }
}

// Index maps stay inside their storage only when hact <= hcap and
// 1 <= lact <= lcap on both axes.
__device__ __forceinline__ bool axis_ok(const Axis& a) {
  const int h = dval(a.hact), l = dval(a.lact);
  return h >= 0 && h <= a.hcap && l >= 1 && l <= a.lcap;
}
__device__ __forceinline__ bool view_ok(const MatView& v) {
  return axis_ok(v.rows) && axis_ok(v.cols);
}

__device__ void zero_view(const MatView& v) {
  const int R = v.rows.hcap * v.rows.lcap, C = v.cols.hcap * v.cols.lcap;
  const long long tot = (long long)R * C;
  for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
    const int i = (int)(e / C), j = (int)(e % C);
    v.ptr[(long long)i * v.ld + j] = 0.0;
  }
}

__device__ __forceinline__ long long view_off(const MatView& v, int ic, int jc, int rl, int cl) {
  return (long long)axis_full(v.rows, ic, rl) * v.ld + axis_full(v.cols, jc, cl);
}

__global__ void __launch_bounds__(256) k_qr_f64(QrArgs a) {
  if (a.skip && *a.skip) return;
  __shared__ double sh[32];
  const Axis& fr = a.inT ? a.A.cols : a.A.rows;
  const Axis& fc = a.inT ? a.A.rows : a.A.cols;
  const int m = axis_len(fr), c = axis_len(fc);
  const int frl = dval(fr.lact), fcl = dval(fc.lact);
  const int arl = dval(a.A.rows.lact), acl = dval(a.A.cols.lact);
  const int r = min(m, c);
  {
    // shape guard: actual extents must fit the capacities of every view
    // and of the work buffer; otherwise flag and touch nothing
    const int fr_cap = fr.hcap * fr.lcap, fc_cap = fc.hcap * fc.lcap;
    const int qr_cap = a.qT ? a.Q.cols.hcap * a.Q.cols.lcap : a.Q.rows.hcap * a.Q.rows.lcap;
    const int qc_cap = a.qT ? a.Q.rows.hcap * a.Q.rows.lcap : a.Q.cols.hcap * a.Q.cols.lcap;
    const int rr_cap = a.rT ? a.R.cols.hcap * a.R.cols.lcap : a.R.rows.hcap * a.R.rows.lcap;
    const int rc_cap = a.rT ? a.R.rows.hcap * a.R.rows.lcap : a.R.cols.hcap * a.R.cols.lcap;
    const bool bad_shape = !view_ok(a.A) || !view_ok(a.Q) || !view_ok(a.R) ||
                           m < 1 || c < 1 || m > fr_cap || c > fc_cap || frl > fr.lcap ||
                           fcl > fc.lcap || m > qr_cap || r > qc_cap || r > rr_cap || c > rc_cap ||
                           (long long)m * c + (long long)m * r + 2LL * c > a.work_len;
    if (bad_shape) {
      if (threadIdx.x == 0 && a.err) atomicOr(a.err, QTT_DEVERR_SHAPE);
      return;
    }
  }
  double* W = a.work;                       // m x c
  double* Qw = W + (size_t)m * c;           // m x r
  double* tau = Qw + (size_t)m * r;         // c
  double* diag = tau + c;                   // c
  bool bad = false;
  for (long long e = threadIdx.x; e < (long long)m * c; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const long long off = a.inT ? view_off(a.A, j, i, arl, acl) : view_off(a.A, i, j, arl, acl);
    const double v = a.A.ptr[off];
    if (!isfinite(v)) bad = true;
    W[e] = v;
  }
  if (bad && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
  if (__syncthreads_or(bad)) {  // non-finite input: zero outputs, report, stop
    zero_view(a.Q);
    zero_view(a.R);
    if (threadIdx.x == 0 && a.r_out) *a.r_out = r;
    return;
  }
  householder(W, m, m, c, tau, diag, sh);
  for (long long e = threadIdx.x; e < (long long)m * r; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Qw[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  apply_reflectors(W, m, m, r, tau, Qw, m, r, true);
  zero_view(a.Q);
  zero_view(a.R);
  __syncthreads();
  const int qrl = dval(a.Q.rows.lact), qcl = dval(a.Q.cols.lact);
  for (long long e = threadIdx.x; e < (long long)m * r; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const long long off = a.qT ? view_off(a.Q, j, i, qrl, qcl) : view_off(a.Q, i, j, qrl, qcl);
    a.Q.ptr[off] = Qw[e];
  }
  const int rrl = dval(a.R.rows.lact), rcl = dval(a.R.cols.lact);
  for (long long e = threadIdx.x; e < (long long)r * c; e += blockDim.x) {
    const int i = (int)(e % r), j = (int)(e / r);
    double v = 0.0;
    if (j == i) v = diag[i];
    else if (j > i) v = W[(size_t)j * m + i];
    const long long off = a.rT ? view_off(a.R, j, i, rrl, rcl) : view_off(a.R, i, j, rrl, rcl);
    a.R.ptr[off] = v;
  }
  if (threadIdx.x == 0 && a.r_out) *a.r_out = r;
}

// Round-robin tournament: position k of round t holds column pos(k, t).
__device__ __forceinline__ int rr_pos(int k, int t, int cp) {
  return k == 0 ? 0 : 1 + (k - 1 + t) % (cp - 1);
}

__global__ void __launch_bounds__(512) k_svd_f64(SvdArgs a) {
  if (a.skip && *a.skip) return;
  __shared__ double sh[32];
  __shared__ int rotated;
  __shared__ int r_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int m = a.inT ? axis_len(a.M.cols) : axis_len(a.M.rows);
  const int N = a.inT ? axis_len(a.M.rows) : axis_len(a.M.cols);
  const int mrl = dval(a.M.rows.lact), mcl = dval(a.M.cols.lact);
  const bool wide = (m <= N);           // factor M^T when M is wide
  const int Rt = wide ? N : m;          // rows of the tall matrix
  const int c = wide ? m : N;           // its columns
  {
    const Axis& fr = a.inT ? a.M.cols : a.M.rows;
    const Axis& fc = a.inT ? a.M.rows : a.M.cols;
    const int us_r = a.usT ? a.US.cols.hcap * a.US.cols.lcap : a.US.rows.hcap * a.US.rows.lcap;
    const int us_c = a.usT ? a.US.rows.hcap * a.US.rows.lcap : a.US.cols.hcap * a.US.cols.lcap;
    const int vt_r = a.vtT ? a.VT.cols.hcap * a.VT.cols.lcap : a.VT.rows.hcap * a.VT.rows.lcap;
    const int vt_c = a.vtT ? a.VT.rows.hcap * a.VT.rows.lcap : a.VT.cols.hcap * a.VT.cols.lcap;
    const int rmax = min(c, min(a.chi, dval(a.rank_limit)));
    const long long need = (long long)Rt * c * 2 + (long long)c * c * 2 + 4LL * c + 2 + (c + 1) / 2;
    const bool bad_shape = !view_ok(a.M) || !view_ok(a.US) || !view_ok(a.VT) ||
                           m < 1 || N < 1 || m > fr.hcap * fr.lcap || N > fc.hcap * fc.lcap ||
                           dval(fr.lact) > fr.lcap || dval(fc.lact) > fc.lcap || m > us_r ||
                           max(rmax, 1) > us_c || max(rmax, 1) > vt_r || N > vt_c ||
                           need > a.work_len;
    if (bad_shape) {
      if (threadIdx.x == 0 && a.err) atomicOr(a.err, QTT_DEVERR_SHAPE);
      return;
    }
  }
  double* T = a.work;                          // Rt x c
  double* X = T + (size_t)Rt * c;              // c x c
  double* J = X + (size_t)c * c;               // c x c
  double* Bw = J + (size_t)c * c;              // Rt x c
  double* tau = Bw + (size_t)Rt * c;           // c
  double* diag = tau + c;                      // c
  double* sig = diag + c;                      // c
  double* tail = sig + c;                      // c + 1
  int* perm = (int*)(tail + c + 1);            // c
  bool bad = false;
  for (long long e = threadIdx.x; e < (long long)Rt * c; e += blockDim.x) {
    const int i = (int)(e % Rt), j = (int)(e / Rt);
    // T(i, j) = F(j, i) when wide, F(i, j) otherwise; F = M or M^T
    const int fi = wide ? j : i, fj = wide ? i : j;
    const long long off = a.inT ? view_off(a.M, fj, fi, mrl, mcl) : view_off(a.M, fi, fj, mrl, mcl);
    const double v = a.M.ptr[off];
    if (!isfinite(v)) bad = true;
    T[e] = v;
  }
  if (bad && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
  if (__syncthreads_or(bad)) {  // non-finite input: zero outputs, rank 1, stop
    zero_view(a.US);
    zero_view(a.VT);
    if (threadIdx.x == 0 && a.r_out) *a.r_out = 1;
    return;
  }
  householder(T, Rt, Rt, c, tau, diag, sh);
  // X = R^T (wide) or R (tall); J = I
  for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
    const int i = (int)(e % c), j = (int)(e / c);
    // R[p][q] = diag (p == q), T[q*Rt + p] (p < q), 0 (p > q)
    const int p = wide ? j : i, q = wide ? i : j;
    double rv = 0.0;
    if (p == q) rv = diag[p];
    else if (p < q) rv = T[(size_t)q * Rt + p];
    X[e] = rv;
    J[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // one-sided Jacobi on the columns of X
  const double tol = fmax(1e-15, 1e-16 * (double)c);
  const int cp = c + (c & 1);
  for (int sweep = 0; sweep < 80 && c > 1; sweep++) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int t = 0; t < cp - 1; t++) {
      for (int k = warp; k < cp / 2; k += nw) {
        int p = rr_pos(k, t, cp), q = rr_pos(cp - 1 - k, t, cp);
        if (p >= c || q >= c) continue;
        if (p > q) { int s_ = p; p = q; q = s_; }
        double* x = X + (size_t)p * c;
        double* y = X + (size_t)q * c;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < c; i += 32) {
          const double xi = x[i], yi = y[i];
          al += xi * xi;
          be += yi * yi;
          ga += xi * yi;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
          for (int i = lane; i < c; i += 32) {
            const double xi = x[i], yi = y[i];
            x[i] = cs * xi - sn * yi;
            y[i] = sn * xi + cs * yi;
          }
          double* jx = J + (size_t)p * c;
          double* jy = J + (size_t)q * c;
          for (int i = lane; i < c; i += 32) {
            const double xi = jx[i], yi = jy[i];
            jx[i] = cs * xi - sn * yi;
            jy[i] = sn * xi + cs * yi;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // singular values and descending order (ties by index)
  for (int k = warp; k < c; k += nw) {
    double s = 0.0;
    const double* x = X + (size_t)k * c;
    for (int i = lane; i < c; i += 32) s += x[i] * x[i];
    s = warp_sum(s);
    if (lane == 0) sig[k] = sqrt(s);
  }
  __syncthreads();
  // descending order under a strict total order (NaN ranks last, ties by
  // index), so perm is always a permutation of 0..c-1
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    int rank = 0;
    const double sk = isnan(sig[k]) ? -1.0 : sig[k];
    for (int j = 0; j < c; j++) {
      const double sj = isnan(sig[j]) ? -1.0 : sig[j];
      rank += (sj > sk) || (sj == sk && j < k);
    }
    perm[rank] = k;
  }
  {
    bool nan_seen = false;
    for (int k = threadIdx.x; k < c; k += blockDim.x) nan_seen |= !isfinite(sig[k]);
    if (nan_seen && a.err) atomicOr(a.err, QTT_DEVERR_NUMERIC);
  }
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
    r = min(r, a.chi);
    r = min(r, lim);
    r = max(r, 1);
    r = min(r, c);
    r_sh = r;
    if (a.r_out) *a.r_out = r;
  }
  __syncthreads();
  const int r = r_sh;
  if (a.sv_out)
    for (int k = threadIdx.x; k < c; k += blockDim.x) a.sv_out[k] = sig[perm[k]];
  // Bw = [J_perm ; 0] (wide: V = Q J) or [X_perm ; 0] (tall: U S = Q X)
  for (long long e = threadIdx.x; e < (long long)Rt * r; e += blockDim.x) {
    const int i = (int)(e % Rt), k = (int)(e / Rt);
    const double* src = wide ? J : X;
    Bw[e] = (i < c) ? src[(size_t)perm[k] * c + i] : 0.0;
  }
  __syncthreads();
  apply_reflectors(T, Rt, Rt, c, tau, Bw, Rt, r, false);
  if (!a.no_us) zero_view(a.US);
  zero_view(a.VT);
  __syncthreads();
  const int url = dval(a.US.rows.lact), ucl = dval(a.US.cols.lact);
  const int vrl = dval(a.VT.rows.lact), vcl = dval(a.VT.cols.lact);
  // U S (m x r)
  for (long long e = threadIdx.x; e < (long long)m * r && !a.no_us; e += blockDim.x) {
    const int i = (int)(e % m), k = (int)(e / m);
    const double v = wide ? X[(size_t)perm[k] * c + i] : Bw[(size_t)k * Rt + i];
    a.US.ptr[a.usT ? view_off(a.US, k, i, url, ucl) : view_off(a.US, i, k, url, ucl)] = v;
  }
  // V^T (r x N)
  for (long long e = threadIdx.x; e < (long long)N * r; e += blockDim.x) {
    const int j = (int)(e % N), k = (int)(e / N);
    const double v = wide ? Bw[(size_t)k * Rt + j] : J[(size_t)perm[k] * c + j];
    a.VT.ptr[a.vtT ? view_off(a.VT, j, k, vrl, vcl) : view_off(a.VT, k, j, vrl, vcl)] = v;
  }
}

}  // namespace

static long long view_extent(const MatView& v) {
  return (long long)(v.rows.hcap * v.rows.lcap - 1) * v.ld + v.cols.hcap * v.cols.lcap;
}

size_t qr_work_doubles(int mcap, int ccap) {
  const size_t r = (size_t)(mcap < ccap ? mcap : ccap);
  return (size_t)mcap * ccap + (size_t)mcap * r + 2 * (size_t)ccap + 8;
}

bool launch_qr_cluster(const QrArgs& a, int mcap, cudaStream_t s);
bool launch_svd_cluster(const SvdArgs& a, int mcap, int ncap, cudaStream_t s, bool fp32);

// Problems at least this large (capacity of the square factor) go to the
// cluster kernels; smaller ones stay on one CTA, where the cluster
// barriers would cost more than they save.
static int cluster_threshold() {
  static int t = [] {
    const char* e = getenv("QTT_CLUSTER_MIN");
    return e ? atoi(e) : 24;
  }();
  return t;
}

void launch_qr_f64(const QrArgs& a, int mcap, int ccap, cudaStream_t s) {
  check_range(a.A.ptr, view_extent(a.A), sizeof(double), "qr A");
  check_range(a.Q.ptr, view_extent(a.Q), sizeof(double), "qr Q");
  check_range(a.R.ptr, view_extent(a.R), sizeof(double), "qr R");
  check_range(a.work, (long long)qr_work_doubles(mcap, ccap), sizeof(double), "qr work");
  const double fm = mcap, fc = ccap < mcap ? ccap : mcap;
  const double flops = 4.0 * fm * fc * fc - 4.0 / 3.0 * fc * fc * fc;
  if ((ccap < mcap ? ccap : mcap) >= cluster_threshold() && launch_qr_cluster(a, mcap, s)) {
    const char* name = "k_qr_cluster";
    if (shape_profiling()) {
      char tag[48];
      snprintf(tag, sizeof tag, "%dx%d", mcap, ccap);
      name = shape_name(name, tag);
    }
    post_launch(name, s, flops);
    return;
  }
  pre_launch(s);
  k_qr_f64<<<1, 256, 0, s>>>(a);
  {
    // Householder factorisation plus explicit Q, at capacity shape
    const double m = mcap, c = ccap < mcap ? ccap : mcap;
    post_launch("k_qr_f64", s, 4.0 * m * c * c - 4.0 / 3.0 * c * c * c);
  }
}

double svd_flops(int mcap, int ncap);

// FP32 working precision for the subspace search of the mixed path; the
// caller refines the returned subspace in FP64 (one subspace iteration with
// a Householder QR).  Returns false when
// no cluster launch is possible or the problem is small (FP64 is used then).
bool launch_svd_subspace_f32(const SvdArgs& a, int mcap, int ncap, cudaStream_t s) {
  check_range(a.M.ptr, view_extent(a.M), sizeof(double), "svd M");
  check_range(a.US.ptr, view_extent(a.US), sizeof(double), "svd US");
  check_range(a.VT.ptr, view_extent(a.VT), sizeof(double), "svd VT");
  check_range(a.work, (long long)svd_work_doubles(mcap, ncap), sizeof(double), "svd work");
  if ((mcap < ncap ? mcap : ncap) < cluster_threshold()) return false;
  // the subspace search only ever wants V^T (both callers recompute the
  // other factor in FP64)
  SvdArgs b = a;
  b.no_us = 1;
  if (!launch_svd_cluster(b, mcap, ncap, s, true)) return false;
  const char* name = "k_svd_cluster_f32";
  if (shape_profiling()) {
    char tag[48];
    snprintf(tag, sizeof tag, "%dx%d", mcap, ncap);
    name = shape_name(name, tag);
  }
  post_launch(name, s, svd_flops(mcap, ncap));
  return true;
}

size_t svd_work_doubles(int mcap, int ncap) {
  const size_t Rt = (size_t)(mcap > ncap ? mcap : ncap);
  const size_t c = (size_t)(mcap < ncap ? mcap : ncap);
  return Rt * c * 2 + c * c * 2 + 4 * c + 8 + (c + 1) / 2 + 8;
}

// Algorithmic FLOPs of one SVD at capacity shape (m x N, c = min, Rt = max):
// Householder of the tall factor 2 Rt c^2 - 2/3 c^3, ten Jacobi sweeps of
// c (c - 1) / 2 pairs at 18 c FLOPs each (three dot products and the two
// column rotations of X and of J), and the back-transform 4 Rt c^2.
double svd_flops(int mcap, int ncap) {
  const double Rt = mcap > ncap ? mcap : ncap, c = mcap < ncap ? mcap : ncap;
  return 2.0 * Rt * c * c - 2.0 / 3.0 * c * c * c + 10.0 * c * (c - 1.0) / 2.0 * 18.0 * c +
         4.0 * Rt * c * c;
}

void launch_svd_f64(const SvdArgs& a, int mcap, int ncap, cudaStream_t s) {
  check_range(a.M.ptr, view_extent(a.M), sizeof(double), "svd M");
  check_range(a.US.ptr, view_extent(a.US), sizeof(double), "svd US");
  check_range(a.VT.ptr, view_extent(a.VT), sizeof(double), "svd VT");
  check_range(a.work, (long long)svd_work_doubles(mcap, ncap), sizeof(double), "svd work");
  if ((mcap < ncap ? mcap : ncap) >= cluster_threshold() && launch_svd_cluster(a, mcap, ncap, s, false)) {
    const char* name = "k_svd_cluster";
    if (shape_profiling()) {
      char tag[48];
      snprintf(tag, sizeof tag, "%dx%d", mcap, ncap);
      name = shape_name(name, tag);
    }
    post_launch(name, s, svd_flops(mcap, ncap));
    return;
  }
  pre_launch(s);
  k_svd_f64<<<1, 512, 0, s>>>(a);
  post_launch("k_svd_f64", s, svd_flops(mcap, ncap));
}
