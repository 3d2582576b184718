// Fourier-space work on dense velocity fields, on the device.
//
// Turbulent kinetic energy spectrum (the paper's TKE spectra, Sec. III.A):
// the dense fields of both components, their 2-D DFTs by radix-2 FFTs of
// the rows and then the columns (one CTA per line, the line in shared
// memory, decimation in time from a bit-reversed load), the power
// |u_hat|^2 + |v_hat|^2 per wavevector, and the sums over integer shells
// k = round(|m|), each shell summed by one CTA in a fixed order
// (bit-reproducible).
//
// Exact spectral projection (the alternative to the penalty that the
// paper's outlook, Sec. IV, points to for periodic boundaries): the same
// forward DFTs, the divergence removed per mode, v = w - sigma (sigma . w) /
// |sigma|^2 with sigma_j(m) = sum_k 2 c_k sin(2 pi k m_j / N) / dx the real
// symbol of the central difference D_j (D_j has symbol i sigma_j), modes
// with sigma = 0 kept, then inverse DFTs of the columns and the rows.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

__device__ __forceinline__ unsigned bitrev(unsigned i, int bits) {
  return __brev(i) >> (32 - bits);
}

// One line of N = 2^logn points per CTA: element e of line l is at
// l * lstride + e * estride of the input (real when re != null, else cin)
// and is written (complex) to the same place of `out`, or, when re_out is
// given, its real part times `scale` to that place of re_out.  inverse = 0:
// X_k = sum_j x_j exp(-2 pi i jk / N); inverse = 1: the same with
// exp(+2 pi i jk / N) (unnormalised).
__global__ void __launch_bounds__(512) k_fft_lines(const double* __restrict__ re,
                                                   const double2* cin, double2* out,
                                                   double* re_out, double scale, int logn,
                                                   long long lstride, long long estride,
                                                   int inverse) {
  extern __shared__ double2 sl[];
  const int N = 1 << logn;
  const long long base = (long long)blockIdx.x * lstride;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const long long at = base + (long long)i * estride;
    const double2 x = re ? make_double2(re[at], 0.0) : cin[at];
    sl[bitrev((unsigned)i, logn)] = x;
  }
  __syncthreads();
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
      const int pos = t % half;
      const int i0 = (t / half) * len + pos, i1 = i0 + half;
      double sn, cs;
      // exp(-+2 pi i pos / len)
      sincospi((inverse ? 2.0 : -2.0) * (double)pos / (double)len, &sn, &cs);
      const double2 a = sl[i0], b = sl[i1];
      const double2 bw = make_double2(b.x * cs - b.y * sn, b.x * sn + b.y * cs);
      sl[i0] = make_double2(a.x + bw.x, a.y + bw.y);
      sl[i1] = make_double2(a.x - bw.x, a.y - bw.y);
    }
    __syncthreads();
  }
  if (re_out) {
    for (int i = threadIdx.x; i < N; i += blockDim.x)
      re_out[base + (long long)i * estride] = sl[i].x * scale;
  } else {
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[base + (long long)i * estride] = sl[i];
  }
}

// sig[m] = sum_{k=1..nw} 2 c_k sin(2 pi k m' / N) / dx, m' = m - N [m >= N/2]:
// the real symbol of the central difference of weights c.  sinpi makes it
// exactly zero where 2 m' = 0 mod N (the mean and the Nyquist mode).
struct FdWeights {
  double c[4];
  int nw;
};

__global__ void k_fd_symbol(double* __restrict__ sig, int N, double dx, FdWeights w) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double mm = (double)(m < N / 2 ? m : m - N);
  double acc = 0.0;
  for (int k = 1; k <= w.nw; k++) acc += 2.0 * w.c[k - 1] * sinpi(2.0 * (double)k * mm / (double)N);
  sig[m] = acc / dx;
}

// Per wavevector (m1, m2) (row m1 along x1, column m2 along x2):
// t = (sigma_1 W_1 + sigma_2 W_2) / (sigma_1^2 + sigma_2^2), W_j -= sigma_j t;
// unchanged where both symbols vanish.
__global__ void k_spectral_project(double2* __restrict__ C1, double2* __restrict__ C2,
                                   const double* __restrict__ sig, int logn) {
  const long long NN = 1LL << (2 * logn);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NN) return;
  const double s1 = sig[e >> logn], s2 = sig[e & ((1LL << logn) - 1)];
  const double den = s1 * s1 + s2 * s2;
  if (!(den > 0.0)) return;
  const double2 a = C1[e], b = C2[e];
  const double tr = (s1 * a.x + s2 * b.x) / den, ti = (s1 * a.y + s2 * b.y) / den;
  C1[e] = make_double2(a.x - s1 * tr, a.y - s1 * ti);
  C2[e] = make_double2(b.x - s2 * tr, b.y - s2 * ti);
}

__global__ void k_power(const double2* __restrict__ A, const double2* __restrict__ B, long long n,
                        double* __restrict__ P) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double2 a = A[e], b = B[e];
  P[e] = a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
}

// floor(sqrt(x)) for 0 <= x < 2^52, exact
__device__ __forceinline__ long long isqrt_floor(long long x) {
  long long r = (long long)sqrt((double)x);
  while (r * r > x) r--;
  while ((r + 1) * (r + 1) <= x) r++;
  return r;
}

// E[k] = sum over wavevectors of shell k of P / (2 N^4): one CTA per shell;
// thread t sums the rows m1 = t, t + blockDim, ... in order, then a fixed
// tree over the threads.  Shell k holds q = m1^2 + m2^2 with
// k^2 - k + 1 <= q <= k^2 + k (q = 0 for k = 0); m = -N/2 .. N/2 - 1 with
// index m mod N.
__global__ void __launch_bounds__(256) k_shells(const double* __restrict__ P, int N,
                                                double* __restrict__ E) {
  __shared__ double red[256];
  const long long k = blockIdx.x;
  const long long qlo = k == 0 ? 0 : k * k - k + 1, qhi = k == 0 ? 0 : k * k + k;
  double acc = 0.0;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const long long m1 = r < N / 2 ? r : r - N;
    const long long hi = qhi - m1 * m1;
    if (hi < 0) continue;
    const long long lo = qlo - m1 * m1;
    const long long a = lo <= 0 ? 0 : isqrt_floor(lo - 1) + 1;  // smallest m2 >= 0, m2^2 >= lo
    const long long b = isqrt_floor(hi);                          // largest m2, m2^2 <= hi
    const double* row = P + (long long)r * N;
    for (long long m2 = a; m2 <= b && m2 <= N / 2; m2++) {
      if (m2 < N / 2) acc += row[m2];  // +m2
      if (m2 > 0) acc += row[N - m2];  // -m2 (includes -N/2)
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double n2 = (double)N * (double)N;
    E[k] = red[0] / (2.0 * n2 * n2);
  }
}

// up to 8192 points (128 KiB) per line in shared memory
constexpr int kFftMaxLog = 13;

bool fft_lines_smem_ready() {
  static const bool ok = cudaFuncSetAttribute(k_fft_lines,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (1 << kFftMaxLog) * (int)sizeof(double2)) ==
                         cudaSuccess;
  return ok;
}

int fft_threads(int N) { return N >= 1024 ? 512 : (N / 2 >= 32 ? N / 2 : 32); }

// C = DFT of the real N x N field u: rows (along x2), then columns (along x1)
void fft2_forward(const double* u, double2* C, int logn, cudaStream_t s) {
  const int N = 1 << logn;
  const size_t smem = (size_t)N * sizeof(double2);
  pre_launch(s);
  k_fft_lines<<<N, fft_threads(N), smem, s>>>(u, nullptr, C, nullptr, 1.0, logn, N, 1, 0);
  post_launch("k_fft_lines", s, 5.0 * N * N * logn);
  pre_launch(s);
  k_fft_lines<<<N, fft_threads(N), smem, s>>>(nullptr, C, C, nullptr, 1.0, logn, 1, N, 0);
  post_launch("k_fft_lines", s, 5.0 * N * N * logn);
}

// u = Re(inverse DFT of C) / N^2: columns, then rows (C is overwritten)
void fft2_inverse_real(double2* C, double* u, int logn, cudaStream_t s) {
  const int N = 1 << logn;
  const size_t smem = (size_t)N * sizeof(double2);
  const double scale = 1.0 / ((double)N * (double)N);
  pre_launch(s);
  k_fft_lines<<<N, fft_threads(N), smem, s>>>(nullptr, C, C, nullptr, 1.0, logn, 1, N, 1);
  post_launch("k_fft_lines", s, 5.0 * N * N * logn);
  pre_launch(s);
  k_fft_lines<<<N, fft_threads(N), smem, s>>>(nullptr, C, nullptr, u, scale, logn, N, 1, 1);
  post_launch("k_fft_lines", s, 5.0 * N * N * logn);
}

}  // namespace

// Spectrum of two dense components (device, N x N each, N = 2^logn <= 4096):
// C1, C2 receive the complex DFTs (N * N double2 each), P the power (N * N),
// E[0..kmax] the shell sums.
void launch_tke_spectrum(const double* u1, const double* u2, int logn, double2* C1, double2* C2,
                         double* P, double* E, int kmax, cudaStream_t s) {
  const int N = 1 << logn;
  const long long NN = (long long)N * N;
  check_range(u1, NN, sizeof(double), "spectrum u1");
  check_range(u2, NN, sizeof(double), "spectrum u2");
  check_range(C1, NN, sizeof(double2), "spectrum C1");
  check_range(C2, NN, sizeof(double2), "spectrum C2");
  check_range(P, NN, sizeof(double), "spectrum P");
  check_range(E, kmax + 1, sizeof(double), "spectrum E");
  const size_t smem = (size_t)N * sizeof(double2);
  if (!fft_lines_smem_ready() || smem > 64 * 1024)
    throw QttError(QTT_ERR_SHAPE, "spectrum: grid too large");
  for (int c = 0; c < 2; c++) fft2_forward(c ? u2 : u1, c ? C2 : C1, logn, s);
  pre_launch(s);
  k_power<<<ceil_div(NN, 256), 256, 0, s>>>(C1, C2, NN, P);
  post_launch("k_power", s);
  pre_launch(s);
  k_shells<<<kmax + 1, 256, 0, s>>>(P, N, E);
  post_launch("k_shells", s);
}

// Exact spectral projection of the dense pair (F1, F2) (device, N x N each,
// N = 2^logn <= 8192), in place; c[0..nw-1] the central-difference weights
// (nw <= 4), dx the grid spacing; C1, C2: N * N double2 scratch, sig: N.
void launch_spectral_project(double* F1, double* F2, int logn, const double* c, int nw, double dx,
                             double2* C1, double2* C2, double* sig, cudaStream_t s) {
  if (logn < 1 || logn > kFftMaxLog) throw QttError(QTT_ERR_SHAPE, "spectral projection: n > 13");
  if (nw < 1 || nw > 4) throw QttError(QTT_ERR_ARG, "spectral projection: stencil weights");
  const int N = 1 << logn;
  const long long NN = (long long)N * N;
  check_range(F1, NN, sizeof(double), "spectral projection F1");
  check_range(F2, NN, sizeof(double), "spectral projection F2");
  check_range(C1, NN, sizeof(double2), "spectral projection C1");
  check_range(C2, NN, sizeof(double2), "spectral projection C2");
  check_range(sig, N, sizeof(double), "spectral projection symbols");
  if (!fft_lines_smem_ready()) throw QttError(QTT_ERR_CUDA, "spectral projection: shared memory");
  FdWeights w{};
  for (int k = 0; k < nw; k++) w.c[k] = c[k];
  w.nw = nw;
  pre_launch(s);
  k_fd_symbol<<<ceil_div(N, 256), 256, 0, s>>>(sig, N, dx, w);
  post_launch("k_fd_symbol", s);
  fft2_forward(F1, C1, logn, s);
  fft2_forward(F2, C2, logn, s);
  pre_launch(s);
  k_spectral_project<<<ceil_div(NN, 256), 256, 0, s>>>(C1, C2, sig, logn);
  post_launch("k_spectral_project", s);
  fft2_inverse_real(C1, F1, logn, s);
  fft2_inverse_real(C2, F2, logn, s);
}
