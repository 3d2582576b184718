// qtt_to_dense_noalloc: the dense readout of a QTT without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// field back: code that runs while a CUDA graph is being captured, a
// real-time loop that must never enter the allocator, or an application
// whose device memory belongs to another framework's pool.  They hand in
// the packed cores and the output buffer; the intermediate partial
// contractions live in a file-scope device array instead of memory the
// library would otherwise allocate per call.
//
// The array is QTT_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB), split into two
// halves of 2^18 doubles that hold the left partial contractions
// L_k (4^k x D_k).  Every GPU that loads the library keeps it until the
// process exits.  All calls share it and it keeps the last call's
// contents: nothing in it needs to start at zero (every entry is written
// before it is read), and two calls whose work overlaps on the GPU race on
// it, so callers must order them (one stream, or events).
#include <mutex>

#include "common.cuh"

#define QTT_NOALLOC_SCRATCH_DOUBLES (1 << 19)

static __device__ __align__(256) double g_noalloc_scratch[QTT_NOALLOC_SCRATCH_DOUBLES];

namespace {

struct NoallocArgs {
  const double* cores;
  int n;
  int bonds[QTT_MAX_N + 1];
  long long off[QTT_MAX_N + 1];
  double* scratch;
  double* F;
};

// L_{k+1}[(p, s)][j] = sum_a L_k[p][a] core_k[a][s][j]; the last step writes
// the field in grid order (omega index t -> (x1, x2)).
__global__ void __launch_bounds__(1024) k_to_dense_noalloc(NoallocArgs g) {
  const long long half = QTT_NOALLOC_SCRATCH_DOUBLES / 2;
  double* A = g.scratch;
  double* B = g.scratch + half;
  const int n = g.n;
  const long long N = 1LL << n;
  if (n == 1) {
    for (int t = threadIdx.x; t < 4; t += blockDim.x) g.F[(t >> 1) * N + (t & 1)] = g.cores[t];
    return;
  }
  const int D1 = g.bonds[1];
  for (long long e = threadIdx.x; e < 4LL * D1; e += blockDim.x) A[e] = g.cores[e];
  __syncthreads();
  long long rows = 4;  // 4^k
  for (int k = 1; k < n; k++) {
    const int Dk = g.bonds[k], Dk1 = g.bonds[k + 1];
    const double* core = g.cores + g.off[k];
    const bool last = (k == n - 1);
    const long long tot = rows * 4 * Dk1;
    for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
      const long long p = e / (4LL * Dk1);
      const int rem = (int)(e % (4LL * Dk1));
      const int s = rem / Dk1, j = rem % Dk1;
      double v = 0.0;
      for (int a = 0; a < Dk; a++) v = fma(A[p * Dk + a], core[((long long)a * 4 + s) * Dk1 + j], v);
      if (last) {
        const long long t = p * 4 + s;  // omega-ordered index of the grid point
        long long x1 = 0, x2 = 0;
        for (int q = 0; q < n; q++) {
          const int d = (int)((t >> (2 * (n - 1 - q))) & 3);
          x1 |= (long long)(d >> 1) << (n - 1 - q);
          x2 |= (long long)(d & 1) << (n - 1 - q);
        }
        g.F[x1 * N + x2] = v;
      } else {
        B[(p * 4 + s) * Dk1 + j] = v;
      }
    }
    __syncthreads();
    double* t = A;
    A = B;
    B = t;
    rows *= 4;
  }
}

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// The array's device address on device `dev` (which must be current),
// looked up once and cached; null if the lookup fails.
void* noalloc_address(int dev) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

// Called by qtt_create with its device current, so that a caller who made a
// context first never reaches the lookup inside a stream capture.
void noalloc_prepare_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) noalloc_address(dev);
}

extern "C" qtt_status qtt_to_dense_noalloc(const double* d_cores, const int* bonds, int n,
                                           double* d_field_out, void* cuda_stream) {
  if (!d_cores || !bonds || !d_field_out || n < 1 || n > 9) return QTT_ERR_ARG;
  if (bonds[0] != 1 || bonds[n] != 1) return QTT_ERR_SHAPE;
  NoallocArgs g{};
  g.cores = d_cores;
  g.n = n;
  g.F = d_field_out;
  long long o = 0, rows = 1;
  const long long half = QTT_NOALLOC_SCRATCH_DOUBLES / 2;
  for (int k = 0; k <= n; k++) {
    if (bonds[k] < 1) return QTT_ERR_SHAPE;
    g.bonds[k] = bonds[k];
  }
  for (int k = 0; k < n; k++) {
    g.off[k] = o;
    o += (long long)bonds[k] * 4 * bonds[k + 1];
    rows *= 4;
    // partial contraction L_{k+1} (4^{k+1} x D_{k+1}) must fit one half
    if (k + 1 < n && rows * bonds[k + 1] > half) return QTT_ERR_SHAPE;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QTT_ERR_CUDA;
  // the array's device address, looked up with this device current the
  // first time the device is seen (qtt_create does it for its device); the
  // cached address stays valid while the device's primary context lives,
  // i.e. until the process exits or resets the device
  void* scratch = noalloc_address(dev);
  if (!scratch) return QTT_ERR_CUDA;
  g.scratch = (double*)scratch;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_to_dense_noalloc<<<1, 1024, 0, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return QTT_ERR_CUDA;
  return QTT_OK;
}
