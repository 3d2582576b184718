// Turbulent kinetic energy spectrum of a velocity field (the paper's TKE
// spectra, Sec. III.A) on the device: the dense fields of both components,
// their 2-D DFTs by radix-2 FFTs of the rows and then the columns (one CTA
// per line, the line in shared memory, decimation in time from a
// bit-reversed load), the power |u_hat|^2 + |v_hat|^2 per wavevector, and
// the sums over integer shells k = round(|m|), each shell summed by one CTA
// in a fixed order (bit-reproducible).
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace {

__device__ __forceinline__ unsigned bitrev(unsigned i, int bits) {
  return __brev(i) >> (32 - bits);
}

// One line of N = 2^logn points per CTA: element e of line l is at
// l * lstride + e * estride of the input (real when re != null, else cin)
// and is written (complex) to the same place of `out`.
__global__ void __launch_bounds__(512) k_fft_lines(const double* __restrict__ re,
                                                   const double2* cin, double2* out, int logn,
                                                   long long lstride, long long estride) {
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
      sincospi(-2.0 * (double)pos / (double)len, &sn, &cs);  // exp(-2 pi i pos / len)
      const double2 a = sl[i0], b = sl[i1];
      const double2 bw = make_double2(b.x * cs - b.y * sn, b.x * sn + b.y * cs);
      sl[i0] = make_double2(a.x + bw.x, a.y + bw.y);
      sl[i1] = make_double2(a.x - bw.x, a.y - bw.y);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) out[base + (long long)i * estride] = sl[i];
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
  static const bool attr = [] {
    return cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                64 * 1024) == cudaSuccess;
  }();
  if (!attr || smem > 64 * 1024) throw QttError(QTT_ERR_SHAPE, "spectrum: grid too large");
  const int th = N >= 1024 ? 512 : (N / 2 >= 32 ? N / 2 : 32);
  for (int c = 0; c < 2; c++) {
    const double* u = c ? u2 : u1;
    double2* C = c ? C2 : C1;
    pre_launch(s);
    k_fft_lines<<<N, th, smem, s>>>(u, nullptr, C, logn, N, 1);  // rows (along x2)
    post_launch("k_fft_lines", s, 5.0 * N * N * logn);
    pre_launch(s);
    k_fft_lines<<<N, th, smem, s>>>(nullptr, C, C, logn, 1, N);  // columns (along x1)
    post_launch("k_fft_lines", s, 5.0 * N * N * logn);
  }
  pre_launch(s);
  k_power<<<ceil_div(NN, 256), 256, 0, s>>>(C1, C2, NN, P);
  post_launch("k_power", s);
  pre_launch(s);
  k_shells<<<kmax + 1, 256, 0, s>>>(P, N, E);
  post_launch("k_shells", s);
}
