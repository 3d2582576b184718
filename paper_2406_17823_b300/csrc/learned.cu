// Learned truncation: the range-finder cut of one bond with a predicted
// rank, and the two-layer perceptron that predicts it.
//
// Range finder (Halko, Martinsson and Tropp, SIAM Review 53 (2011),
// Algorithm 4.1): Y = M Omega, Q = orth(Y), B = Q^T M, SVD of B.  The
// Gaussian test matrix comes from a counter-based generator so that every
// entry is produced independently: SplitMix64 (Steele, Lea and Flood,
// OOPSLA 2014) at state key + (i + 1) * 0x9E3779B97F4A7C15, the top 53 bits
// as a uniform in (0, 1), two uniforms per normal by the Box-Muller
// transform (Box and Muller 1958).  Entry (i, j) uses counters 2e, 2e + 1,
// e = i * 1024 + j, with i = s * D + b the row (s, b) of the unfolding at its
// ACTUAL width D.
//
// Perceptron: 33 inputs -> 64 ReLU units -> 1 output, FP32 parameters
// packed as W1 (64 x 33, row-major), b1 (64), W2 (64), b2.  Loss: mean
// squared error; optimiser: Adam (Kingma and Ba, ICLR 2015).  Gradients are
// reduced per parameter over the samples in sample order, so a training run
// is deterministic.
#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr int kFeat = QTT_MLP_FEATURES;
constexpr int kHid = QTT_MLP_HIDDEN;
constexpr int kParam = QTT_MLP_PARAMS;
constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long key, unsigned long long i) {
  return ((double)(splitmix64(key + (i + 1) * kGolden) >> 11) + 0.5) * 0x1.0p-53;
}

__device__ __forceinline__ double gaussian(unsigned long long key, unsigned long long e) {
  const double u1 = uniform01(key, 2 * e), u2 = uniform01(key, 2 * e + 1);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Omega (4 Dcap x wcap, row-major): capacity row s * Dcap + b holds logical
// row s * D + b (b < D); columns j < w; zero elsewhere.
__global__ void k_rf_omega(double* O, int Dcap, const int* Dact, int wcap, const int* wact,
                           unsigned long long key) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = 4LL * Dcap * wcap;
  if (e >= tot) return;
  const int row = (int)(e / wcap), j = (int)(e % wcap);
  const int s = row / Dcap, b = row % Dcap;
  const int D = Dact ? *Dact : Dcap;
  const int w = wact ? *wact : wcap;
  double v = 0.0;
  if (b < D && j < w && j < 1024) {
    const unsigned long long i = (unsigned long long)s * D + b;
    v = gaussian(key, i * 1024ull + (unsigned long long)j);
  }
  O[e] = v;
}

__device__ float mlp_eval(const float* P, const float* x) {
  const float* W1 = P;
  const float* b1 = P + kHid * kFeat;
  const float* W2 = b1 + kHid;
  const float b2 = W2[kHid];
  float out = b2;
  for (int h = 0; h < kHid; h++) {
    float z = b1[h];
    for (int f = 0; f < kFeat; f++) z = fmaf(W1[h * kFeat + f], x[f], z);
    out = fmaf(W2[h], fmaxf(z, 0.0f), out);
  }
  return out;
}

__global__ void k_mlp_forward(const float* P, const float* X, int N, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = mlp_eval(P, X + (long long)n * kFeat);
}

// per sample: pre-activations Z (N x 64) and dL/dout = 2 (out - y) / N
__global__ void k_mlp_fwd_store(const float* P, const float* X, const float* y, int N, float* Z,
                                float* dout) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float* x = X + (long long)n * kFeat;
  const float* W1 = P;
  const float* b1 = P + kHid * kFeat;
  const float* W2 = b1 + kHid;
  float out = W2[kHid];
  for (int h = 0; h < kHid; h++) {
    float z = b1[h];
    for (int f = 0; f < kFeat; f++) z = fmaf(W1[h * kFeat + f], x[f], z);
    Z[(long long)n * kHid + h] = z;
    out = fmaf(W2[h], fmaxf(z, 0.0f), out);
  }
  dout[n] = 2.0f * (out - y[n]) / (float)N;
}

// one thread per parameter (and one more for the loss), samples in order
__global__ void k_mlp_reduce(const float* P, const float* X, const float* y, int N,
                             const float* Z, const float* dout, float* G, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kParam) return;
  const float* W2 = P + kHid * kFeat + kHid;
  double acc = 0.0;
  if (p < kHid * kFeat) {  // W1[h][f]
    const int h = p / kFeat, f = p % kFeat;
    for (int n = 0; n < N; n++) {
      const float z = Z[(long long)n * kHid + h];
      if (z > 0.0f) acc += (double)dout[n] * W2[h] * X[(long long)n * kFeat + f];
    }
  } else if (p < kHid * kFeat + kHid) {  // b1[h]
    const int h = p - kHid * kFeat;
    for (int n = 0; n < N; n++)
      if (Z[(long long)n * kHid + h] > 0.0f) acc += (double)dout[n] * W2[h];
  } else if (p < kHid * kFeat + 2 * kHid) {  // W2[h]
    const int h = p - kHid * kFeat - kHid;
    for (int n = 0; n < N; n++) acc += (double)dout[n] * fmaxf(Z[(long long)n * kHid + h], 0.0f);
  } else if (p == kParam - 1) {  // b2
    for (int n = 0; n < N; n++) acc += (double)dout[n];
  } else {  // p == kParam: the loss, sum of r^2 / N with r = dout N / 2
    for (int n = 0; n < N; n++) {
      const double r = 0.5 * (double)dout[n] * N;
      acc += r * r;
    }
    *loss = (float)(acc / N);
    return;
  }
  G[p] = (float)acc;
}

__global__ void k_adam(float* P, const float* G, float* m, float* v, int t, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParam) return;
  const float b1 = 0.9f, b2 = 0.999f, e = 1e-8f;
  const float g = G[p];
  const float mm = b1 * m[p] + (1.0f - b1) * g;
  const float vv = b2 * v[p] + (1.0f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.0f - powf(b1, (float)t));
  const float vh = vv / (1.0f - powf(b2, (float)t));
  P[p] -= lr * mh / (sqrtf(vh) + e);
}

// Rank prediction for one bond: w = min(rank + p, wcap, D, N) from the
// previous step's features, or w = 1 and use_rf = 0 without them.
__global__ void k_rf_predict(const float* P, const float* feat, const int* valid, int chi,
                             int over, int wcap, const int* Dact, const int* Nact4, int* w_out,
                             int* use_rf) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int D = *Dact, N = 4 * *Nact4;
  int w = 1, use = 0;
  if (valid && *valid) {
    const float out = mlp_eval(P, feat);
    const float rf = rintf(out * (float)chi);
    int r = isfinite(rf) ? (int)fminf(fmaxf(rf, 1.0f), (float)chi) : chi;
    w = min(min(r + over, wcap), min(D, N));
    use = 1;
  }
  *w_out = max(w, 1);
  *use_rf = use;
}

// Accept the range finder when its outside weight |M|^2 - |B|^2 is at most
// 0.1 eps^2 |M|^2 (the sketch misses at most a tenth of the bond's
// truncation budget); skip_full = 1 then (the full SVD that follows is
// skipped).
__global__ void k_rf_decide(const double* nM, const double* nB, double eps, const int* use_rf,
                            int* skip_full, double* total, long long* counters) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double m = *nM, outside = fmax(m - *nB, 0.0);
  const int accept = (*use_rf) && !(outside > 0.1 * eps * eps * m);
  *skip_full = accept;
  *total = m;
  if (*use_rf) counters[accept ? 0 : 1] += 1;
}

// Features of the bond just cut (33 floats) and its rank, from the sorted
// singular values sv (c of them: w when the range finder was accepted,
// min(D, N) otherwise).
__global__ void k_rf_features(const double* sv, const int* skip_full, const int* w,
                              const int* Dact, const int* Nact4, const int* r, int bond, int n,
                              float* feat, int* rank, int* valid) {
  if (blockIdx.x != 0) return;
  const int c = (skip_full && *skip_full) ? *w : min(*Dact, 4 * *Nact4);
  const double s0 = c > 0 ? sv[0] : 0.0;
  for (int j = threadIdx.x; j < kFeat - 1; j += blockDim.x) {
    float f = -1.0f;
    if (s0 > 0.0 && j < c) {
      const double q = fmax(sv[j] / s0, 1e-300);
      f = (float)(fmax(log10(q), -16.0) / 16.0);
    }
    feat[j] = f;
  }
  if (threadIdx.x == 0) {
    feat[kFeat - 1] = (float)bond / (float)n;
    *rank = *r;
    *valid = 1;
  }
}

}  // namespace

void launch_rf_omega(double* O, int Dcap, const int* Dact, int wcap, const int* wact,
                     unsigned long long key, cudaStream_t s) {
  const long long tot = 4LL * Dcap * wcap;
  if (tot <= 0) return;
  check_range(O, tot, sizeof(double), "rf omega");
  pre_launch(s);
  k_rf_omega<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(O, Dcap, Dact, wcap, wact, key);
  post_launch("k_rf_omega", s);
}

void launch_mlp_forward(const float* P, const float* X, int N, float* out, cudaStream_t s) {
  if (N <= 0) return;
  check_range(P, kParam, sizeof(float), "ext mlp params");
  pre_launch(s);
  k_mlp_forward<<<(N + 127) / 128, 128, 0, s>>>(P, X, N, out);
  post_launch("k_mlp_forward", s);
}

void launch_mlp_grad(const float* P, const float* X, const float* y, int N, float* Z, float* dout,
                     float* G, float* loss, cudaStream_t s) {
  if (N <= 0) return;
  check_range(Z, (long long)N * kHid, sizeof(float), "mlp Z");
  check_range(dout, N, sizeof(float), "mlp dout");
  pre_launch(s);
  k_mlp_fwd_store<<<(N + 127) / 128, 128, 0, s>>>(P, X, y, N, Z, dout);
  post_launch("k_mlp_fwd_store", s);
  pre_launch(s);
  k_mlp_reduce<<<(kParam + 1 + 127) / 128, 128, 0, s>>>(P, X, y, N, Z, dout, G, loss);
  post_launch("k_mlp_reduce", s);
}

void launch_adam(float* P, const float* G, float* m, float* v, int t, float lr, cudaStream_t s) {
  check_range(m, kParam, sizeof(float), "adam m");
  check_range(v, kParam, sizeof(float), "adam v");
  pre_launch(s);
  k_adam<<<(kParam + 127) / 128, 128, 0, s>>>(P, G, m, v, t, lr);
  post_launch("k_adam", s);
}

void launch_rf_predict(const float* P, const float* feat, const int* valid, int chi, int over,
                       int wcap, const int* Dact, const int* Nact4, int* w_out, int* use_rf,
                       cudaStream_t s) {
  pre_launch(s);
  k_rf_predict<<<1, 32, 0, s>>>(P, feat, valid, chi, over, wcap, Dact, Nact4, w_out, use_rf);
  post_launch("k_rf_predict", s);
}

void launch_rf_decide(const double* nM, const double* nB, double eps, const int* use_rf,
                      int* skip_full, double* total, long long* counters, cudaStream_t s) {
  pre_launch(s);
  k_rf_decide<<<1, 32, 0, s>>>(nM, nB, eps, use_rf, skip_full, total, counters);
  post_launch("k_rf_decide", s);
}

void launch_rf_features(const double* sv, const int* skip_full, const int* w, const int* Dact,
                        const int* Nact4, const int* r, int bond, int n, float* feat, int* rank,
                        int* valid, cudaStream_t s) {
  pre_launch(s);
  k_rf_features<<<1, 32, 0, s>>>(sv, skip_full, w, Dact, Nact4, r, bond, n, feat, rank, valid);
  post_launch("k_rf_features", s);
}
