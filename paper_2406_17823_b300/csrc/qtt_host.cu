// Host orchestration of the QTT time step and the C ABI of include/qtt.h.
//
// Every operation is a fixed sequence of kernel launches on the context
// stream whose shapes are the host-known CAPACITIES; actual bond
// dimensions are decided and read on the device (see common.cuh), so
// nothing here waits for the GPU except the convergence tests of the
// projection (CG every few iterations, and once per sweep).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <map>
#include <memory>
#include <set>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

thread_local LaunchCounter* g_launch_counter = nullptr;

#include <iterator>
#include <map>
#include <mutex>
#include <thread>

namespace {
std::mutex g_reg_mu;
std::map<uintptr_t, size_t>& reg_map() {
  static std::map<uintptr_t, size_t> m;
  return m;
}
}  // namespace

// ---- launch profiler (events around every launch while a context profiles)
// noalloc.cu: resolve the allocation-free readout's static array on the
// current device (outside any stream capture)
void noalloc_prepare_current_device();

namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t e0, e1;
  double flops;
};
// Per-launch CUDA events of every context in the process (the recording is
// shared by host threads under a mutex; each thread keeps its own pending
// start event, so contexts stepped from different threads do not mix).
struct Profiler {
  bool on = false;
  std::mutex mu;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    std::lock_guard<std::mutex> g(mu);
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) throw QttError(QTT_ERR_CUDA, "cudaEventCreate failed");
    return e;
  }
};
Profiler g_prof;
thread_local cudaEvent_t t_pending = nullptr;
}  // namespace

void pre_launch(cudaStream_t s) {
  if (!g_prof.on) return;
  t_pending = g_prof.get();
  QTT_CUDA_CHECK(cudaEventRecord(t_pending, s));
}

bool shape_profiling() {
  static const bool on = getenv("QTT_PROFILE_SHAPES") != nullptr;
  return on;
}

const char* shape_name(const char* base, const char* tag) {
  if (!shape_profiling()) return base;
  static std::mutex mu;
  static std::set<std::string> names;
  std::lock_guard<std::mutex> lk(mu);
  return names.insert(std::string(base) + "[" + tag + "]").first->c_str();
}

void post_launch(const char* name, cudaStream_t s, double flops) {
  count_launch();
  if (g_prof.on && t_pending) {
    cudaEvent_t e1 = g_prof.get();
    QTT_CUDA_CHECK(cudaEventRecord(e1, s));
    {
      std::lock_guard<std::mutex> g(g_prof.mu);
      g_prof.recs.push_back(ProfRec{name, t_pending, e1, flops});
    }
    t_pending = nullptr;
  }
  static const bool dbg = getenv("QTT_DEBUG_SYNC") != nullptr;
  if (!dbg) return;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) throw CudaError(e, name, 0);
}

void reg_alloc(const void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_reg_mu);
  reg_map()[(uintptr_t)p] = bytes;
}
void reg_free(const void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_reg_mu);
  reg_map().erase((uintptr_t)p);
}
void check_range(const void* p, long long count, size_t eb, const char* what) {
  if (!p || count <= 0) return;
  std::lock_guard<std::mutex> g(g_reg_mu);
  auto& m = reg_map();
  const bool external = strncmp(what, "ext", 3) == 0;  // caller-owned buffer
  auto it = m.upper_bound((uintptr_t)p);
  const uintptr_t a = (uintptr_t)p;
  if (it == m.begin() || a >= std::prev(it)->first + std::prev(it)->second) {
    if (external) return;
    char buf[160];
    snprintf(buf, sizeof buf, "launch range check failed (%s): pointer outside every library "
             "allocation", what);
    throw QttError(QTT_ERR_SHAPE, buf);
  }
  --it;
  const uintptr_t base = it->first, end = base + it->second;
  if (a + (uintptr_t)count * eb > end) {
    char buf[200];
    snprintf(buf, sizeof buf, "launch range check failed (%s): %lld elements from offset %llu, "
             "allocation holds %llu bytes", what, count, (unsigned long long)(a - base),
             (unsigned long long)it->second);
    throw QttError(QTT_ERR_SHAPE, buf);
  }
}


// ------------------------------------------------------------------ objects
struct qtt_mps_s {
  qtt_ctx ctx = nullptr;
  int n = 0;
  std::vector<int> cap;     // n + 1
  std::vector<size_t> off;  // n + 1, off[n] = total doubles
  double* data = nullptr;   // device
  int* dims = nullptr;      // device, n + 1
  cudaStream_t stream = nullptr;
  double* core(int k) const { return data + off[k]; }
  size_t core_size(int k) const { return (size_t)cap[k] * 4 * cap[k + 1]; }
};

struct qtt_mpo_s {
  int n = 0;
  std::vector<int> w;                      // n + 1
  std::vector<std::vector<double>> h;      // W[p][so][si][q]
  double* dev = nullptr;                   // raw cores
  double* dev_k2 = nullptr;                // [(s q)][(p t)]
  double* dev_kr2 = nullptr;               // [(s p)][(q t)]
  std::vector<size_t> off;                 // per core offset (same for all three)
  int refs = 1;
  double* raw(int k) const { return dev + off[k]; }
  double* k2(int k) const { return dev_k2 + off[k]; }
  double* kr2(int k) const { return dev_kr2 + off[k]; }
  // the non-zeros of k2 / kr2 per core (host-built MPOs only)
  std::vector<SparseRows> sk2, skr2;
  const SparseRows* sp_k2(int k) const { return k < (int)sk2.size() ? &sk2[k] : nullptr; }
  const SparseRows* sp_kr2(int k) const { return k < (int)skr2.size() ? &skr2[k] : nullptr; }
};

// A stage's right-hand side captured as a CUDA graph: graph-owned input
// buffers (u_0, u_1, b_0, b_1; b unused when it aliases u) and outputs
// (w_0, w_1) with the capacities of the occurrence it was captured from.
struct StageGraph {
  cudaGraphExec_t exec = nullptr;
  qtt_mps in[4] = {nullptr, nullptr, nullptr, nullptr};
  qtt_mps out[2] = {nullptr, nullptr};
  long long launches = 0;  // kernels per replay
  int seen = 0;            // eager occurrences so far
  bool failed = false;     // not capturable: launched eagerly from then on
};

struct qtt_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  qtt_params p{};
  double dx = 0.0;
  std::string err;
  int* d_err = nullptr;
  qtt_mpo D[2] = {nullptr, nullptr};
  qtt_mpo lap = nullptr;
  qtt_mpo K[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  LaunchCounter launches;
  long long cg_iters = 0, sweeps = 0;
  int last_not_converged = 0;
  // worker streams for independent operations of a stage (non-blocking, so
  // the legacy default stream does not serialise them), joined by events
  static constexpr int kWorkers = 12;
  static constexpr int kStageWorkers = 10;  // the rest: the running sum of RK4 stages
  cudaStream_t workers[kWorkers] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t sum_ev = nullptr;  // hands a finished RK4 stage to the running sum
  cudaEvent_t join_ev[kWorkers] = {};
  static constexpr int kFlowEvents = 16;
  cudaEvent_t flow_ev[kFlowEvents] = {};  // cross-stream dependencies inside a stage
  cudaStream_t cur = nullptr;  // stream the current operation enqueues on
  // learned truncation: features / ranks / flags of every cut of the
  // previous (tab ^ 1) and the current (tab) step, [slot][bond][feature]
  static constexpr int kSlots = QTT_LEARNED_SLOTS;
  static constexpr int kBonds = 16;
  float* d_feat[2] = {nullptr, nullptr};
  int* d_rank[2] = {nullptr, nullptr};
  int* d_valid[2] = {nullptr, nullptr};
  int tab = 0;
  int slot = 0;
  float* d_mlp = nullptr;
  bool mlp_set = false;
  // [0] cuts served by the range finder, [1] its fallbacks; [2] tensor-core
  // subspace searches accepted, [3] searches that fell back to the FP32 SVD
  long long* d_rf_counts = nullptr;
  // stage graphs (params.graphs), keyed by input capacities, aliasing, h,
  // nu and a; captured on a private non-blocking stream
  cudaStream_t gstream = nullptr;
  std::map<std::string, std::unique_ptr<StageGraph>> graphs;
  static constexpr int kMaxGraphs = 16;  // captured graphs kept per context
  long long graphs_captured = 0, graph_replays = 0;
  // whole-step graphs (params.graphs = 2): the projection's CG and sweep
  // loops run as WHILE nodes, captured on the body streams; their counters
  // and the step statistics live on the device until the next sync
  std::map<std::string, std::unique_ptr<StageGraph>> step_graphs;
  cudaStream_t bstream[2] = {nullptr, nullptr};
  // the matvec chains inside loop body k run on bworkers[k][0..3] (a stream
  // joined to one capture cannot serve another)
  cudaStream_t bworkers[2][4] = {{nullptr, nullptr, nullptr, nullptr},
                                  {nullptr, nullptr, nullptr, nullptr}};
  bool dev_loops = false;      // set while a step is being captured
  long long* d_stats = nullptr;  // [0] CG iterations, [1] sweeps, [2] not converged,
                                 // [3] kernels run by loop bodies
  int* d_loop = nullptr;         // [0..1] loop counters, [2] sweep stop word
  bool stats_pending = false;
};

namespace {

// Set for the duration of a call on a mixed-precision context: the FP64
// products of eligible shapes run on the tensor cores (gemm_oz.cu) unless
// QTT_OZAKI=0.
thread_local bool t_gemm_emulate = false;

bool ozaki_allowed() {
  static const bool on = [] {
    const char* e = getenv("QTT_OZAKI");
    return !(e && e[0] == '0');
  }();
  return on;
}

struct CtxGuard {
  LaunchCounter* prev;
  bool prev_emulate;
  explicit CtxGuard(qtt_ctx c) : prev(g_launch_counter), prev_emulate(t_gemm_emulate) {
    g_launch_counter = &c->launches;
    g_dev_err = c->d_err;
    t_gemm_emulate = c->p.precision == QTT_PREC_MIXED && ozaki_allowed();
    cudaSetDevice(c->device);
  }
  ~CtxGuard() {
    g_launch_counter = prev;
    t_gemm_emulate = prev_emulate;
  }
};

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t n_, cudaStream_t s_) : n(n_), s(s_) {
    if (n) {
      cudaError_t e = cudaMallocAsync((void**)&p, n * sizeof(T), s);
      if (e != cudaSuccess) throw QttError(QTT_ERR_ALLOC, "cudaMallocAsync failed");
      reg_alloc(p, n * sizeof(T));
    }
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    release();
    p = o.p; n = o.n; s = o.s; o.p = nullptr;
    return *this;
  }
  void release() {
    if (p) {
      reg_free(p);
      cudaFreeAsync(p, s);
    }
    p = nullptr;
  }
  ~DBuf() { release(); }
};

// The stream operations enqueue on: a worker stream while a stage runs its
// independent operations concurrently, else the context stream.
cudaStream_t stream_of(qtt_ctx ctx) { return ctx->cur ? ctx->cur : ctx->stream; }

long long natural_cap(int n, int b) {
  long long a = 1, c = 1;
  for (int i = 0; i < b && a < (1LL << 40); i++) a *= 4;
  for (int i = 0; i < n - b && c < (1LL << 40); i++) c *= 4;
  return std::min(a, c);
}
int clampi(long long v) { return (int)std::min<long long>(v, 1 << 30); }

qtt_mps new_mps(qtt_ctx ctx, int n, const std::vector<int>& cap) {
  auto m = new qtt_mps_s;
  m->ctx = ctx;
  m->n = n;
  m->cap = cap;
  m->off.resize(n + 1);
  size_t o = 0;
  for (int k = 0; k < n; k++) {
    m->off[k] = o;
    o += (size_t)cap[k] * 4 * cap[k + 1];
  }
  m->off[n] = o;
  m->stream = stream_of(ctx);
  if (cudaMallocAsync((void**)&m->data, o * sizeof(double), m->stream) != cudaSuccess ||
      cudaMallocAsync((void**)&m->dims, (n + 1) * sizeof(int), m->stream) != cudaSuccess) {
    delete m;
    throw QttError(QTT_ERR_ALLOC, "MPS allocation failed");
  }
  reg_alloc(m->data, o * sizeof(double));
  reg_alloc(m->dims, (n + 1) * sizeof(int));
  QTT_CUDA_CHECK(cudaMemsetAsync(m->data, 0, o * sizeof(double), m->stream));
  return m;
}

void free_mps(qtt_mps m) {
  if (!m) return;
  reg_free(m->data);
  reg_free(m->dims);
  if (m->data) cudaFreeAsync(m->data, m->stream);
  if (m->dims) cudaFreeAsync(m->dims, m->stream);
  delete m;
}

struct MpsPtr {
  qtt_mps m = nullptr;
  MpsPtr() = default;
  explicit MpsPtr(qtt_mps x) : m(x) {}
  MpsPtr(const MpsPtr&) = delete;
  MpsPtr(MpsPtr&& o) noexcept : m(o.m) { o.m = nullptr; }
  MpsPtr& operator=(MpsPtr&& o) noexcept {
    if (m != o.m) free_mps(m);
    m = o.m;
    o.m = nullptr;
    return *this;
  }
  ~MpsPtr() { free_mps(m); }
  qtt_mps release() {
    qtt_mps t = m;
    m = nullptr;
    return t;
  }
  qtt_mps get() const { return m; }
  qtt_mps operator->() const { return m; }
};

// One product with a given tile (0: 64 x 64, 1: 32 x 32) and K cut into S
// slices (S > 1: single products only): the slices run as one batched
// launch into scratch, then C = alpha * (sum of the slices, in slice order:
// deterministic) + beta * C; a skip flag skips both launches.
// Split-K scratch supplied by the caller (a buffer made before a capture
// whose conditional bodies may not allocate); null: allocate per product.
thread_local double* t_gemm_scratch = nullptr;
thread_local size_t t_gemm_scratch_n = 0;
// set while a graph is being captured: products of a shape not met before
// take the fixed rule instead of being timed (timing waits for the device)
thread_local bool t_capturing = false;

void gemm_run(const GemmF64& g, int tile, int S, cudaStream_t s) {
  if (S <= 1 || g.nb1 * g.nb2 != 1 || g.K < 2) {
    launch_gemm_f64_tile(g, tile, s);
    return;
  }
  const int chunk = (g.K + S - 1) / S;
  const int full = g.K / chunk, rem = g.K - full * chunk;
  const int Sx = full + (rem > 0 ? 1 : 0);
  const size_t need = (size_t)Sx * g.M * g.N;
  DBuf<double> Pown;
  double* Pp = t_gemm_scratch;
  if (Pp) {
    if (need > t_gemm_scratch_n) throw QttError(QTT_ERR_SHAPE, "split-K scratch too small");
  } else {
    Pown = DBuf<double>(need, s);
    Pp = Pown.p;
  }
  GemmF64 b = g;
  b.C = Pp;
  b.ldc = g.N;
  b.alpha = 1.0;
  b.beta = 0.0;
  b.K = chunk;
  b.nb1 = full;
  b.nb2 = 1;
  b.sA1 = g.tA ? (long long)chunk * g.lda : chunk;  // A stored K x M (tA) or M x K
  b.sB1 = g.tB ? chunk : (long long)chunk * g.ldb;  // B stored N x K (tB) or K x N
  b.sC1 = (long long)g.M * g.N;
  launch_gemm_f64_tile(b, tile, s);
  if (rem > 0) {
    GemmF64 r = b;
    r.K = rem;
    r.nb1 = 1;
    r.A = g.A + full * b.sA1;
    r.B = g.B + full * b.sB1;
    r.C = Pp + full * b.sC1;
    launch_gemm_f64_tile(r, tile, s);
  }
  launch_sum_slices(Pp, Sx, g.M, g.N, g.C, g.ldc, g.alpha, g.beta, g.skip, s);
}

// The fixed rule: 64 x 64 tiles, K cut into slices of at least 32 while the
// output has too few tiles to occupy the GPU.
int split_rule(const GemmF64& g) {
  const int tiles = ((g.M + 63) / 64) * ((g.N + 63) / 64);
  int S = 1;
  while (g.nb1 * g.nb2 == 1 && tiles * S * 2 <= 2 * 148 && g.K / (S * 2) >= 32) S *= 2;
  return S;
}

// Autotuner: the first time a process meets a product shape (M, N, K,
// transposes, batch) it times every (tile, K split) candidate on the
// caller's stream, writing into scratch, and keeps the fastest for the rest
// of the process (so repeated runs use the same summation order).
// QTT_AUTOTUNE=0 keeps the fixed rule.
struct GemmKey {
  int M, N, K, tA, tB, nb;
  bool operator<(const GemmKey& o) const {
    return std::tie(M, N, K, tA, tB, nb) < std::tie(o.M, o.N, o.K, o.tA, o.tB, o.nb);
  }
};
struct GemmChoice {
  int tile, S;
};
std::mutex g_tune_mu;
std::map<GemmKey, GemmChoice>& tune_map() {
  static std::map<GemmKey, GemmChoice> m;
  return m;
}

// Optional persistence (QTT_TUNE_CACHE = a file path): the choices are read
// from that JSON file on first use and the file is rewritten whenever a new
// shape is tuned, so later processes reuse the same choices (and the same
// summation orders).  Format: {"version": 1, "entries": [[M, N, K, tA, tB,
// batch, tile, split], ...]}.  Callers hold g_tune_mu.
const char* tune_cache_path() {
  static const char* p = getenv("QTT_TUNE_CACHE");
  return (p && p[0]) ? p : nullptr;
}
void tune_cache_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, got);
  fclose(f);
  const size_t at = txt.find("\"entries\"");
  if (at == std::string::npos) return;
  std::vector<long long> v;
  const char* c = txt.c_str() + at;
  while (*c) {
    if ((*c >= '0' && *c <= '9') || *c == '-') {
      char* end = nullptr;
      v.push_back(strtoll(c, &end, 10));
      c = end;
    } else {
      c++;
    }
  }
  for (size_t i = 0; i + 8 <= v.size(); i += 8) {
    const GemmKey k{(int)v[i], (int)v[i + 1], (int)v[i + 2], (int)v[i + 3], (int)v[i + 4],
                    (int)v[i + 5]};
    const int tile = (int)v[i + 6], S = (int)v[i + 7];
    if (tile < 0 || tile > 3 || S < 1 || S > 16 || (S & (S - 1))) continue;  // not ours
    tune_map().emplace(k, GemmChoice{tile, S});
  }
}
void tune_cache_save() {
  const char* path = tune_cache_path();
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\"version\": 1, \"entries\": [");
  bool first = true;
  for (const auto& kv : tune_map()) {
    const GemmKey& k = kv.first;
    fprintf(f, "%s\n  [%d, %d, %d, %d, %d, %d, %d, %d]", first ? "" : ",", k.M, k.N, k.K, k.tA,
            k.tB, k.nb, kv.second.tile, kv.second.S);
    first = false;
  }
  fprintf(f, "\n]}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

GemmChoice gemm_tune(const GemmF64& g, cudaStream_t s) {
  const int nb = g.nb1 * g.nb2;
  // scratch output, compact layout (the candidates' results are discarded)
  DBuf<double> Cs((size_t)g.M * g.N * nb, s);
  GemmF64 t = g;
  t.C = Cs.p;
  t.ldc = g.N;
  t.sC2 = (long long)g.M * g.N;
  t.sC1 = t.sC2 * g.nb2;
  t.alpha = 1.0;
  t.beta = 0.0;
  t.skip = nullptr;
  cudaEvent_t e0, e1;
  QTT_CUDA_CHECK(cudaEventCreate(&e0));
  QTT_CUDA_CHECK(cudaEventCreate(&e1));
  GemmChoice best{0, split_rule(g)};
  float tbest = 1e30f;
  for (int tile = 0; tile < 4; tile++)
    for (int S = 1; S <= 16; S *= 2) {
      if (tile == 2 && g.M > 32) break;  // the skinny tile only for outputs of a few rows
      if (tile == 3 && !gemm_small_eligible(g)) break;
      if (S > 1 && (nb != 1 || g.K / S < 32)) break;
      gemm_run(t, tile, S, s);  // warm
      QTT_CUDA_CHECK(cudaEventRecord(e0, s));
      gemm_run(t, tile, S, s);
      QTT_CUDA_CHECK(cudaEventRecord(e1, s));
      QTT_CUDA_CHECK(cudaEventSynchronize(e1));
      float ms = 0.f;
      QTT_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < tbest) {
        tbest = ms;
        best = GemmChoice{tile, S};
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void gemm(const GemmF64& g, cudaStream_t s) {
  static const bool tune = [] {
    const char* e = getenv("QTT_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.nb1 * g.nb2 <= 0) {
    launch_gemm_f64(g, s);  // empty product or C = beta C
    return;
  }
  // A single product whose K exceeds what one emulated launch takes (16384:
  // the environment contractions at chi >= 128, K = 3 chi^2) runs as K
  // pieces on the tensor cores, accumulated in order into C (beta of the
  // first piece, 1 after); QTT_OZ_SPLIT_K=0 leaves it to the FP64 GEMM.
  static const bool split_long_k = [] {
    const char* e = getenv("QTT_OZ_SPLIT_K");
    return !(e && e[0] == '0');
  }();
  constexpr int kOzMaxK1 = 16384;
  if (t_gemm_emulate && split_long_k && g.nb1 * g.nb2 == 1 && g.K > kOzMaxK1) {
    GemmF64 h = g;
    h.K = kOzMaxK1;
    if (gemm_oz_dispatch(h)) {
      for (int k0 = 0; k0 < g.K; k0 += kOzMaxK1) {
        h.K = std::min(kOzMaxK1, g.K - k0);
        h.A = g.A + (g.tA ? (long long)k0 * g.lda : k0);  // A stored K x M (tA) or M x K
        h.B = g.B + (g.tB ? k0 : (long long)k0 * g.ldb);  // B stored N x K (tB) or K x N
        h.beta = k0 == 0 ? g.beta : 1.0;
        gemm(h, s);
      }
      return;
    }
  }
  if (t_gemm_emulate && gemm_oz_dispatch(g)) {
    // an unbatched product with a small output (M N <= kOzWideSplitMN) and
    // few output tiles may deal its K chunks over up to 64 slices (the
    // public entry point's plan stops at 16): a rule of the shape alone, so
    // eager and captured runs take the same plan, and the projection's
    // captured scratch is sized for it; QTT_OZ_MAX_SPLITS=16 keeps 16
    static const int env_max = [] {
      const char* e = getenv("QTT_OZ_MAX_SPLITS");
      const int v = e ? atoi(e) : 64;
      return v < 16 ? 16 : (v > 64 ? 64 : v);
    }();
    const int max_s = (long long)g.M * g.N <= kOzWideSplitMN ? env_max : 16;
    const int S = gemm_oz_splits(g, max_s);
    if (S <= 1) {
      launch_gemm_oz(g, g_dev_err, s, false, nullptr, 0, max_s);
      return;
    }
    // K slices: partial products in the caller's split-K scratch (inside
    // captured loop bodies) or a stream-ordered buffer
    const size_t need = (size_t)S * g.M * g.N;
    DBuf<double> own;
    double* P = t_gemm_scratch;
    size_t cap = t_gemm_scratch_n;
    if (P) {
      if (need > cap) throw QttError(QTT_ERR_SHAPE, "split-K scratch too small");
    } else {
      own = DBuf<double>(need, s);
      P = own.p;
      cap = need;
    }
    launch_gemm_oz(g, g_dev_err, s, false, P, cap, max_s);
    return;
  }
  // QTT_GEMM_TILE=t: every product on tile t with the fixed K split (a
  // check that the tiles give the same bits, and a way to time one tile)
  static const int forced = [] {
    const char* e = getenv("QTT_GEMM_TILE");
    return e && e[0] >= '0' && e[0] <= '3' && e[1] == 0 ? e[0] - '0' : -1;
  }();
  if (forced >= 0) {
    gemm_run(g, forced, split_rule(g), s);
    return;
  }
  if (!tune) {
    gemm_run(g, 0, split_rule(g), s);
    return;
  }
  const GemmKey key{g.M, g.N, g.K, g.tA, g.tB, g.nb1 * g.nb2};
  GemmChoice ch;
  bool found = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = tune_map().find(key);
    if (it != tune_map().end()) {
      ch = it->second;
      found = true;
    }
  }
  if (!found && t_capturing) {
    gemm_run(g, 0, split_rule(g), s);
    return;
  }
  if (!found) {
    ch = gemm_tune(g, s);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto ins = tune_map().emplace(key, ch);  // another thread may have tuned it first
    ch = ins.first->second;
    if (ins.second) tune_cache_save();
  }
  gemm_run(g, ch.tile, ch.S, s);
}

// C_z = A B_z with A one MPO core reshaped as k2 or kr2 and shared by the
// batch: the sparse-row kernel over the core's non-zeros when they were
// stored (the dense product's FMA chain without its zero terms: the same
// values); QTT_MPO_SPARSE=0 keeps every such product on the GEMM.
void mpo_gemm(const GemmF64& g, const SparseRows* sp, cudaStream_t s) {
  static const bool on = [] {
    const char* e = getenv("QTT_MPO_SPARSE");
    return !(e && e[0] == '0');
  }();
  if (on && sp && sp->nnz >= 0 && sp->rows == g.M && sp->cols == g.K && g.tA == 0 &&
      g.tB == 0 && g.nb2 == 1 && g.sA1 == 0 && g.alpha == 1.0 && g.beta == 0.0 && !g.skip &&
      g.M > 0 && g.N > 0 && g.nb1 > 0) {
    launch_sparse_rows(*sp, g.B, g.ldb, g.sB1, g.C, g.ldc, g.sC1, g.N, g.nb1, s);
    return;
  }
  gemm(g, s);
}

// Split-K product with the fixed rule (Gram matrices of long factors).
void gemm_splitk(const GemmF64& g, cudaStream_t s) { gemm(g, s); }

// --------------------------------------------------------------- MPO build
// Carry tensor of App. A, Table "diff_mpo": C[p][so][si][q], p = alpha_m
// (carry to the more significant site), q = alpha_{m+1} (request from the
// less significant site: 0 keep, 1 add one, 2 subtract one), acting on the
// x1 bit (axis 1) or the x2 bit (axis 2) of omega; so is the output index
// and si the input index, so that the operator maps U to U(x +- 1).
void carry_tensor(int axis, double C[3][4][4][3]) {
  memset(C, 0, sizeof(double) * 3 * 4 * 4 * 3);
  for (int q = 0; q < 3; q++)
    for (int so = 0; so < 4; so++) {
      const int x = so >> 1, y = so & 1;
      const int bit = axis == 1 ? x : y;
      int nb = bit, p = 0;
      if (q == 1) { nb = bit + 1; if (nb == 2) { nb = 0; p = 1; } }
      if (q == 2) { nb = bit - 1; if (nb == -1) { nb = 1; p = 2; } }
      const int si = axis == 1 ? (nb << 1 | y) : (x << 1 | nb);
      C[p][so][si][q] = 1.0;
    }
}

// Generic host MPO: cores as flat vectors with bonds w.
struct HostMpo {
  int n;
  std::vector<int> w;
  std::vector<std::vector<double>> c;  // [p][so][si][q]
};

// A finite-state carry MPO for coef0 * I + sum_t coef_t * S_{axis_t}^{shift_t}
// with shift_t in {-2, -1, +1, +2} and (S U)(x) = U(x + shift) along the
// axis.  Bond states: 0 = idle, plus one state per (axis, sign) meaning
// "add sign to this axis bit" requested by the less significant side; a
// bit overflow passes the same state on as a carry (App. A, Table
// "diff_mpo", generalised).  A shift by 2 leaves the least significant bit
// unchanged and starts its request one site up.  The final carry out of
// the most significant site is dropped (periodic grid).
HostMpo shift_sum_mpo(int n, double coef0, const std::vector<int>& axes,
                      const std::vector<int>& shifts, const std::vector<double>& coefs) {
  std::vector<std::pair<int, int>> st{{0, 0}};
  auto sid = [&](int axis, int sign) {
    for (size_t i = 1; i < st.size(); i++)
      if (st[i].first == axis && st[i].second == sign) return (int)i;
    st.push_back({axis, sign});
    return (int)st.size() - 1;
  };
  for (size_t t = 0; t < axes.size(); t++) sid(axes[t], shifts[t] > 0 ? 1 : -1);
  const int S = (int)st.size();
  // C[p][so][si][q]: request q applied to omega (so = output, si = input)
  std::vector<double> C((size_t)S * 16 * S, 0.0);
  for (int q = 0; q < S; q++)
    for (int so = 0; so < 4; so++) {
      const int x = so >> 1, y = so & 1;
      int p = 0, si = so;
      if (q != 0) {
        const int axis = st[q].first, sign = st[q].second;
        int nb = (axis == 1 ? x : y) + sign;
        bool carry = false;
        if (nb == 2) { nb = 0; carry = true; }
        if (nb == -1) { nb = 1; carry = true; }
        si = axis == 1 ? (nb << 1 | y) : (x << 1 | nb);
        p = carry ? q : 0;
      }
      C[((size_t)(p * 4 + so) * 4 + si) * S + q] = 1.0;
    }
  std::vector<double> Rn(S, 0.0), Rn1(S, 0.0);  // requests entering site n / site n-1
  Rn[0] = coef0;
  for (size_t t = 0; t < axes.size(); t++) {
    const int id = sid(axes[t], shifts[t] > 0 ? 1 : -1);
    if (std::abs(shifts[t]) == 1) Rn[id] += coefs[t];
    else Rn1[id] += coefs[t];
  }
  HostMpo m;
  m.n = n;
  m.w.assign(n + 1, S);
  m.w[0] = 1;
  m.w[n] = 1;
  m.c.resize(n);
  for (int k = 0; k < n; k++) {
    const int wr = m.w[k + 1];
    m.c[k].assign((size_t)m.w[k] * 16 * wr, 0.0);
    for (int p = 0; p < S; p++)
      for (int so = 0; so < 4; so++)
        for (int si = 0; si < 4; si++) {
          const int pi = (k == 0) ? 0 : p;  // L = all ones
          if (k == n - 1) {
            double v = 0.0;
            for (int q = 0; q < S; q++) v += C[((size_t)(p * 4 + so) * 4 + si) * S + q] * Rn[q];
            if (so == si && p > 0) v += Rn1[p];  // shift by 2: pass through, request upward
            if (v != 0.0) m.c[k][((size_t)(pi * 4 + so) * 4 + si) * wr] += v;
          } else {
            for (int q = 0; q < S; q++) {
              const double v = C[((size_t)(p * 4 + so) * 4 + si) * S + q];
              if (v != 0.0) m.c[k][((size_t)(pi * 4 + so) * 4 + si) * wr + q] += v;
            }
          }
        }
  }
  return m;
}

qtt_mpo upload_mpo(qtt_ctx ctx, const HostMpo& hm) {
  auto m = new qtt_mpo_s;
  m->n = hm.n;
  m->w = hm.w;
  m->h = hm.c;
  m->off.resize(hm.n + 1);
  size_t o = 0;
  for (int k = 0; k < hm.n; k++) {
    m->off[k] = o;
    o += hm.c[k].size();
  }
  m->off[hm.n] = o;
  std::vector<double> raw(o), k2(o), kr2(o);
  for (int k = 0; k < hm.n; k++) {
    const int wl = hm.w[k], wr = hm.w[k + 1];
    for (int p = 0; p < wl; p++)
      for (int s = 0; s < 4; s++)
        for (int t = 0; t < 4; t++)
          for (int q = 0; q < wr; q++) {
            const double v = hm.c[k][((p * 4 + s) * 4 + t) * wr + q];
            raw[m->off[k] + ((p * 4 + s) * 4 + t) * wr + q] = v;
            // k2[(s q)][(p t)]
            k2[m->off[k] + (size_t)(s * wr + q) * (wl * 4) + (p * 4 + t)] = v;
            // kr2[(s p)][(q t)]
            kr2[m->off[k] + (size_t)(s * wl + p) * (wr * 4) + (q * 4 + t)] = v;
          }
  }
  // compressed rows of k2 ((s q) x (p t)) and kr2 ((s p) x (q t)) for the
  // sparse-row product; a core with too many non-zeros keeps nnz = -1
  auto compress_rows = [](const double* M, int rows, int cols) {
    SparseRows sp;
    sp.rows = rows;
    sp.cols = cols;
    if (rows > kSparseMaxRows) return sp;
    int nnz = 0;
    sp.ptr[0] = 0;
    for (int r = 0; r < rows; r++) {
      for (int c = 0; c < cols; c++) {
        const double v = M[(size_t)r * cols + c];
        if (v == 0.0) continue;
        if (nnz == kSparseMaxNnz) return sp;
        sp.col[nnz] = c;
        sp.val[nnz++] = v;
      }
      sp.ptr[r + 1] = nnz;
    }
    sp.nnz = nnz;
    return sp;
  };
  m->sk2.resize(hm.n);
  m->skr2.resize(hm.n);
  for (int k = 0; k < hm.n; k++) {
    const int wl = hm.w[k], wr = hm.w[k + 1];
    m->sk2[k] = compress_rows(k2.data() + m->off[k], 4 * wr, 4 * wl);
    m->skr2[k] = compress_rows(kr2.data() + m->off[k], 4 * wl, 4 * wr);
  }
  cudaSetDevice(ctx->device);
  if (cudaMalloc((void**)&m->dev, 3 * o * sizeof(double)) != cudaSuccess) {
    delete m;
    throw QttError(QTT_ERR_ALLOC, "MPO allocation failed");
  }
  reg_alloc(m->dev, 3 * o * sizeof(double));
  m->dev_k2 = m->dev + o;
  m->dev_kr2 = m->dev + 2 * o;
  QTT_CUDA_CHECK(cudaMemcpy(m->dev, raw.data(), o * sizeof(double), cudaMemcpyHostToDevice));
  QTT_CUDA_CHECK(cudaMemcpy(m->dev_k2, k2.data(), o * sizeof(double), cudaMemcpyHostToDevice));
  QTT_CUDA_CHECK(cudaMemcpy(m->dev_kr2, kr2.data(), o * sizeof(double), cudaMemcpyHostToDevice));
  return m;
}

void mpo_release(qtt_mpo m) {
  if (!m) return;
  if (--m->refs > 0) return;
  reg_free(m->dev);
  if (m->dev) cudaFree(m->dev);
  delete m;
}

// D_axis (App. A): L = (1,1,1), R = (0, 1, -1) / (2 dx), carry table.
HostMpo diff_mpo(int n, int axis, double dx) {
  double C[3][4][4][3];
  carry_tensor(axis, C);
  HostMpo m;
  m.n = n;
  m.w.assign(n + 1, 3);
  m.w[0] = m.w[n] = 1;
  m.c.resize(n);
  const double R[3] = {0.0, 1.0 / (2.0 * dx), -1.0 / (2.0 * dx)};
  for (int k = 0; k < n; k++) {
    const int wl = m.w[k], wr = m.w[k + 1];
    m.c[k].assign((size_t)wl * 16 * wr, 0.0);
    for (int p = 0; p < 3; p++)
      for (int so = 0; so < 4; so++)
        for (int si = 0; si < 4; si++)
          for (int q = 0; q < 3; q++) {
            double v = C[p][so][si][q];
            if (v == 0.0) continue;
            if (k == n - 1) v *= R[q];
            const int pi = (k == 0) ? 0 : p, qi = (k == n - 1) ? 0 : q;
            m.c[k][((pi * 4 + so) * 4 + si) * wr + qi] += v;  // L = (1,1,1) sums p at k = 0
          }
  }
  return m;
}

// Product of two host MPOs A.B (B acts first), bonds multiply.
HostMpo mpo_mul(const HostMpo& A, const HostMpo& B) {
  HostMpo m;
  m.n = A.n;
  m.w.resize(A.n + 1);
  for (int b = 0; b <= A.n; b++) m.w[b] = A.w[b] * B.w[b];
  m.c.resize(A.n);
  for (int k = 0; k < A.n; k++) {
    const int al = A.w[k], ar = A.w[k + 1], bl = B.w[k], br = B.w[k + 1];
    const int wr = ar * br;
    m.c[k].assign((size_t)al * bl * 16 * wr, 0.0);
    for (int pa = 0; pa < al; pa++)
      for (int pb = 0; pb < bl; pb++)
        for (int so = 0; so < 4; so++)
          for (int si = 0; si < 4; si++)
            for (int qa = 0; qa < ar; qa++)
              for (int qb = 0; qb < br; qb++) {
                double v = 0.0;
                for (int t = 0; t < 4; t++)
                  v += A.c[k][((pa * 4 + so) * 4 + t) * ar + qa] *
                       B.c[k][((pb * 4 + t) * 4 + si) * br + qb];
                if (v == 0.0) continue;
                m.c[k][(((pa * bl + pb) * 4 + so) * 4 + si) * wr + (qa * br + qb)] = v;
              }
  }
  return m;
}

HostMpo mpo_scaled(HostMpo m, double s) {
  for (double& v : m.c[0]) v *= s;
  return m;
}

// Weights c_1..c_m of the central difference of even order 2m,
// D U(x) = sum_k c_k (U(x + k dx) - U(x - k dx)) / dx (Sec. II.B, any order;
// App. D, 8th order): by Taylor expansion the difference holds only odd
// derivatives, so D U = U' + O(dx^2m) needs sum_k c_k k = 1/2 and
// sum_k c_k k^j = 0 for odd j = 3..2m-1.  Gaussian elimination with partial
// pivoting on that m x m system.
std::vector<double> central_weights(int order) {
  const int m = order / 2;
  std::vector<std::vector<double>> A(m, std::vector<double>(m + 1, 0.0));
  for (int i = 0; i < m; i++) {
    for (int k = 1; k <= m; k++) A[i][k - 1] = std::pow((double)k, 2 * i + 1);
    A[i][m] = i == 0 ? 0.5 : 0.0;
  }
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    std::swap(A[c], A[piv]);
    for (int r = c + 1; r < m; r++) {
      const double f = A[r][c] / A[c][c];
      for (int q = c; q <= m; q++) A[r][q] -= f * A[c][q];
    }
  }
  std::vector<double> x(m);
  for (int r = m - 1; r >= 0; r--) {
    double v = A[r][m];
    for (int q = r + 1; q < m; q++) v -= A[r][q] * x[q];
    x[r] = v / A[r][r];
  }
  return x;
}

// MPO of coef0 I + sum_t coef_t S_{axis_t}^{a_t} for any integer shifts,
// (S^a U)(x) = U(x + a e_axis) on the periodic grid.  A finite-state
// machine over the bits read from the least significant site up: the bond
// carries (axis, p), the integer p still to be added to that axis' more
// significant part (p = 0 is one idle state shared by both axes).  At a site
// with output bit b the input bit is (b + p) mod 2 and the state becomes
// (axis, floor((b + p) / 2)) -- App. A's carry table, generalised from +-1
// to any constant.  The value left over at the most significant site is a
// multiple of N and is dropped (periodic wrap: L sums every state).  Bond
// states are the values reachable from the requested shifts at each bond.
HostMpo translation_mpo(int n, double coef0, const std::vector<int>& axes,
                        const std::vector<int>& shifts, const std::vector<double>& coefs) {
  using St = std::pair<int, long long>;  // (axis, p); (0, 0) idle
  auto fdiv2 = [](long long x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); };
  auto next = [&](const St& q, int b) -> St {
    if (q.first == 0) return St{0, 0};
    const long long p = fdiv2(b + q.second);
    return p == 0 ? St{0, 0} : St{q.first, p};
  };
  std::map<St, double> start;
  start[St{0, 0}] += coef0;
  for (size_t t = 0; t < axes.size(); t++) {
    const St q = shifts[t] == 0 ? St{0, 0} : St{axes[t], (long long)shifts[t]};
    start[q] += coefs[t];
  }
  std::vector<std::vector<St>> st(n + 1);
  for (auto& kv : start) st[n].push_back(kv.first);
  for (int k = n - 1; k >= 0; k--) {
    std::set<St> nx;
    for (const St& q : st[k + 1])
      for (int b = 0; b < 2; b++) nx.insert(next(q, b));
    st[k].assign(nx.begin(), nx.end());
  }
  auto index = [](const std::vector<St>& v, const St& q) {
    return (int)(std::lower_bound(v.begin(), v.end(), q) - v.begin());
  };
  HostMpo m;
  m.n = n;
  m.w.resize(n + 1);
  for (int b = 0; b <= n; b++) m.w[b] = (int)st[b].size();
  m.w[0] = 1;
  m.w[n] = 1;
  m.c.resize(n);
  for (int k = 0; k < n; k++) {
    const int wl = m.w[k], wr = m.w[k + 1];
    m.c[k].assign((size_t)wl * 16 * wr, 0.0);
    for (size_t qi = 0; qi < st[k + 1].size(); qi++) {
      const St q = st[k + 1][qi];
      const double wq = (k == n - 1) ? start[q] : 1.0;  // R: the requested shifts
      const int qo = (k == n - 1) ? 0 : (int)qi;
      for (int so = 0; so < 4; so++) {
        const int x = so >> 1, y = so & 1;
        int si = so;
        if (q.first != 0) {
          const int b = q.first == 1 ? x : y;
          const int nb = (int)(((b + q.second) % 2 + 2) % 2);
          si = q.first == 1 ? (nb << 1 | y) : (x << 1 | nb);
        }
        const int pl = (k == 0) ? 0 : index(st[k], next(q, q.first == 1 ? x : y));
        m.c[k][((size_t)(pl * 4 + so) * 4 + si) * wr + qo] += wq;  // L sums at k = 0
      }
    }
  }
  return m;
}

// Central difference of order `order` along `axis` raised to `power` (1: D,
// 2: D D, the literal square of App. B) with spacing dx, as translations.
HostMpo fd_mpo(int n, int axis, int power, int order, double dx) {
  const std::vector<double> c = central_weights(order);
  const int m = (int)c.size();
  std::map<int, double> d;  // shift -> coefficient of D
  for (int k = 1; k <= m; k++) {
    d[k] += c[k - 1] / dx;
    d[-k] -= c[k - 1] / dx;
  }
  std::map<int, double> e = d;
  if (power == 2) {
    e.clear();
    for (auto& a : d)
      for (auto& b : d) e[a.first + b.first] += a.second * b.second;
  }
  double coef0 = 0.0;
  std::vector<int> axes, shifts;
  std::vector<double> coefs;
  for (auto& kv : e) {
    if (kv.first == 0) {
      coef0 += kv.second;
      continue;
    }
    axes.push_back(axis);
    shifts.push_back(kv.first);
    coefs.push_back(kv.second);
  }
  return translation_mpo(n, coef0, axes, shifts, coefs);
}

// The Laplacian D_1 D_1 + D_2 D_2 of order `order` (the literal squares of
// App. B) as one translation machine over both axes.
HostMpo fd_laplacian(int n, int order, double dx) {
  const std::vector<double> c = central_weights(order);
  const int m = (int)c.size();
  std::map<int, double> d, e;
  for (int k = 1; k <= m; k++) {
    d[k] += c[k - 1] / dx;
    d[-k] -= c[k - 1] / dx;
  }
  for (auto& x : d)
    for (auto& y : d) e[x.first + y.first] += x.second * y.second;
  double coef0 = 0.0;
  std::vector<int> axes, shifts;
  std::vector<double> coefs;
  for (int ax = 1; ax <= 2; ax++)
    for (auto& kv : e) {
      if (kv.first == 0) {
        coef0 += kv.second;
        continue;
      }
      axes.push_back(ax);
      shifts.push_back(kv.first);
      coefs.push_back(kv.second);
    }
  return translation_mpo(n, coef0, axes, shifts, coefs);
}

// ------------------------------------------------------------ compression
// The mixed form's subspace search on the tensor cores (QTT_TC_SEARCH=0
// selects the FP32 cluster Jacobi search instead) and its power iterations
// after the sketch (QTT_TC_ITERS, default 6).
// QTT_TC_SEARCH: 0 off, z zip-up cuts only (default), c compression cuts
// only, a all.
int tc_search_mode() {
  static const int m = [] {
    const char* e = getenv("QTT_TC_SEARCH");
    if (!e) return 1;
    return e[0] == '0' ? 0 : e[0] == 'z' ? 1 : e[0] == 'c' ? 2 : 3;
  }();
  return m;
}
bool tc_search_zipup() { return tc_search_mode() & 1; }
bool tc_search_compress() { return tc_search_mode() & 2; }
// Largest accepted contraction rho = (sigma_p / sigma_keep)^2 of a
// tensor-core search (QTT_TC_RHO, default 1e-1): after the FP64 subspace
// iteration the kept directions' error is about the search's FP32-level floor
// times rho (about 1e-8 of the factor's norm at 1e-1).
double tc_rho_max() {
  static const double r = [] {
    const char* e = getenv("QTT_TC_RHO");
    return e ? atof(e) : 1e-1;
  }();
  return r;
}
// FP64 subspace iterations after the search (QTT_FP64_ITERS, default 1)
int mixed_fp64_iters() {
  static const int it = [] {
    const char* e = getenv("QTT_FP64_ITERS");
    const int v = e ? atoi(e) : 1;
    return v < 1 ? 1 : v > 4 ? 4 : v;
  }();
  return it;
}
int tc_search_iters() {
  static const int it = [] {
    const char* e = getenv("QTT_TC_ITERS");
    const int v = e ? atoi(e) : 6;
    return v < 0 ? 0 : v > 16 ? 16 : v;
  }();
  return it;
}

// compress X -> new MPS with caps ocap; X unchanged.
qtt_mps compress_impl(qtt_ctx ctx, qtt_mps X, double eps, int chi, bool left_canonical = false) {
  const int n = X->n;
  cudaStream_t s = stream_of(ctx);
  const auto& cin = X->cap;
  std::vector<int> qcap(n + 1, 1), ocap(n + 1, 1);
  for (int b = 1; b < n; b++) qcap[b] = std::min(4 * qcap[b - 1], cin[b]);
  for (int b = n - 1; b >= 1; b--)
    ocap[b] = std::min({qcap[b], 4 * ocap[b + 1], chi, clampi(natural_cap(n, b))});
  // A left-canonical input (cores 1..n-1 with orthonormal columns, stored at
  // the capacities the sweep would give them) is its own left-to-right QR
  // sweep: Q_k = X_k and R = I.  The sweep is skipped.
  bool lc = left_canonical;
  for (int b = 0; b <= n && lc; b++) lc = qcap[b] == cin[b];
  MpsPtr Y(new_mps(ctx, n, ocap));
  launch_fill_int(Y->dims, n + 1, 1, s);  // interior bonds are written by the SVDs
  if (n == 1) {
    launch_copy(Y->core(0), X->core(0), 4, s);
    return Y.release();
  }
  // workspace
  size_t qcore_tot = 0;
  std::vector<size_t> qoff(n);
  for (int k = 0; k < n - 1; k++) {
    qoff[k] = qcore_tot;
    qcore_tot += (size_t)qcap[k] * 4 * qcap[k + 1];
  }
  size_t rmax = 1, tmax = 1, usmax = 1, mmax = 1, qrw = 1, svw = 1;
  for (int b = 1; b < n; b++) rmax = std::max(rmax, (size_t)qcap[b] * cin[b]);
  for (int k = 0; k < n; k++) tmax = std::max(tmax, (size_t)qcap[k] * 4 * cin[k + 1]);
  for (int b = 1; b < n; b++) usmax = std::max(usmax, (size_t)qcap[b] * ocap[b]);
  for (int k = 0; k < n; k++) mmax = std::max(mmax, (size_t)qcap[k] * 4 * ocap[k + 1]);
  for (int k = 0; k < n - 1; k++) qrw = std::max(qrw, qr_work_doubles(4 * qcap[k], cin[k + 1]));
  for (int k = 1; k < n; k++) svw = std::max(svw, svd_work_doubles(qcap[k], 4 * ocap[k + 1]));
  DBuf<double> Qc(lc ? 0 : qcore_tot, s), Rb(lc ? 0 : rmax, s), Tb(lc ? 0 : tmax, s),
      USb(usmax, s), Mb(mmax, s), W(std::max(qrw, svw), s);
  DBuf<int> qD(lc ? 0 : n + 1, s);
  if (!lc) launch_fill_int(qD.p, n + 1, 1, s);
  // Q cores of the left-to-right sweep, their actual right dims, and the last core R X_{n-1}
  auto qcore = [&](int k) -> const double* { return lc ? X->core(k) : Qc.p + qoff[k]; };
  int* const qdims = lc ? X->dims : qD.p;
  const bool mixed = ctx->p.precision == QTT_PREC_MIXED;
  constexpr int kOver = 16;
  size_t vtm = 1, bmm = 1, vbm = 1, rsm = 1;
  if (mixed)
    for (int k = 1; k < n; k++) {
      const size_t rpo = std::min({qcap[k], 4 * ocap[k + 1], chi + kOver});
      vtm = std::max(vtm, rpo * 4 * ocap[k + 1]);
      bmm = std::max(bmm, (size_t)qcap[k] * rpo);
      vbm = std::max(vbm, (size_t)ocap[k] * rpo);
      rsm = std::max(rsm, rpo * rpo);
    }
  // tensor-core subspace search of the mixed form: scratch for the widest cut
  size_t tcm = 0;
  if (mixed && tc_search_compress())
    for (int k = 1; k < n; k++) {
      const int rpo = std::min({qcap[k], 4 * ocap[k + 1], chi + kOver});
      if (tc_search_supported(4 * ocap[k + 1], qcap[k], rpo))
        tcm = std::max(tcm, tc_search_scratch_floats(4 * ocap[k + 1], qcap[k], rpo));
    }
  DBuf<float> TCs(tcm, s);
  DBuf<int> tca(tcm ? 2 : 0, s);  // accept flag, stop word
  DBuf<double> Rs(mixed ? rsm : 0, s), Vt(mixed ? vtm : 0, s), Bm(mixed ? bmm : 0, s),
      Vb(mixed ? vbm : 0, s), wM(1, s);
  DBuf<int> rp(1, s);
  // learned truncation: this call's slot, and the range finder's buffers
  const int lmode = ctx->p.learned_trunc;
  const int slot = lmode != QTT_LEARNED_OFF ? ctx->slot++ : -1;
  const bool logged = slot >= 0 && slot < qtt_ctx_s::kSlots && n < qtt_ctx_s::kBonds;
  const bool learn = logged && lmode == QTT_LEARNED_ON && ctx->mlp_set && eps > 0.0;
  const int over = ctx->p.rf_oversample;
  std::vector<int> wcap(n + 1, 1);
  size_t om = 1, ym = 1, bbm = 1, ubm = 1, rrm = 1, svm = 1;
  for (int k = 1; k < n; k++) {
    wcap[k] = std::max(1, std::min({qcap[k], 4 * ocap[k + 1], chi + over}));
    om = std::max(om, (size_t)4 * ocap[k + 1] * wcap[k]);
    ym = std::max(ym, (size_t)qcap[k] * wcap[k]);
    bbm = std::max(bbm, (size_t)wcap[k] * 4 * ocap[k + 1]);
    ubm = std::max(ubm, (size_t)wcap[k] * ocap[k]);
    rrm = std::max(rrm, (size_t)wcap[k] * wcap[k]);
    svm = std::max(svm, (size_t)std::min(qcap[k], 4 * ocap[k + 1]));
  }
  DBuf<double> Om(learn ? om : 0, s), Yr(learn ? ym : 0, s), Qy(learn ? ym : 0, s),
      Bb(learn ? bbm : 0, s), Ubr(learn ? ubm : 0, s), Rr(learn ? rrm : 0, s),
      sv(logged ? svm : 0, s), rfd(learn ? 3 : 0, s);
  DBuf<int> rfi(learn ? 3 : 0, s);  // width, use_rf, skip_full
  // left-to-right QR
  for (int k = 0; k < n - 1 && !lc; k++) {
    const double* Tp;
    if (k == 0) {
      Tp = X->core(0);
    } else {
      GemmF64 g = gemm_plain(Rb.p, X->core(k), Tb.p, qcap[k], 4 * cin[k + 1], cin[k], cin[k],
                             4 * cin[k + 1], 4 * cin[k + 1]);
      gemm(g, s);
      Tp = Tb.p;
    }
    QrArgs a{};
    a.A = MatView{const_cast<double*>(Tp), cin[k + 1], axis_pair(qcap[k], dref(qD.p + k), 4, dconst(4)),
                  axis_prefix(cin[k + 1], dref(X->dims + k + 1))};
    a.Q = MatView{Qc.p + qoff[k], qcap[k + 1], axis_pair(qcap[k], dref(qD.p + k), 4, dconst(4)),
                  axis_prefix(qcap[k + 1], dconst(1))};
    a.R = MatView{Rb.p, cin[k + 1], axis_prefix(qcap[k + 1], dconst(1)),
                  axis_prefix(cin[k + 1], dref(X->dims + k + 1))};
    a.r_out = qD.p + k + 1;
    a.work = W.p;
    a.work_len = (long long)W.n;
    a.err = ctx->d_err;
    launch_qr_f64(a, 4 * qcap[k], cin[k + 1], s);
  }
  // last core after the sweep: T = R * X_{n-1}  (qcap[n-1] x 4)
  if (!lc) {
    GemmF64 g = gemm_plain(Rb.p, X->core(n - 1), Tb.p, qcap[n - 1], 4, cin[n - 1], cin[n - 1], 4, 4);
    gemm(g, s);
  }
  // right-to-left truncated SVD
  for (int k = n - 1; k >= 1; k--) {
    const double* Mp;
    if (k == n - 1) {
      Mp = lc ? X->core(n - 1) : Tb.p;
    } else {
      // M = Qcore_k (4 qcap[k] x qcap[k+1]) * US (qcap[k+1] x ocap[k+1])
      GemmF64 g = gemm_plain(qcore(k), USb.p, Mb.p, 4 * qcap[k], ocap[k + 1], qcap[k + 1],
                             qcap[k + 1], ocap[k + 1], ocap[k + 1]);
      gemm(g, s);
      Mp = Mb.p;
    }
    SvdArgs a{};
    a.M = MatView{const_cast<double*>(Mp), 4 * ocap[k + 1], axis_prefix(qcap[k], dref(qdims + k)),
                  axis_pair(4, dconst(4), ocap[k + 1], dref(Y->dims + k + 1))};
    a.US = MatView{USb.p, ocap[k], axis_prefix(qcap[k], dref(qdims + k)),
                   axis_prefix(ocap[k], dconst(1))};
    a.VT = MatView{Y->core(k), 4 * ocap[k + 1], axis_prefix(ocap[k], dconst(1)),
                   axis_pair(4, dconst(4), ocap[k + 1], dref(Y->dims + k + 1))};
    a.eps = eps;
    a.chi = chi;
    a.rank_limit = dconst(1 << 30);
    a.r_out = Y->dims + k;
    a.work = W.p;
    a.work_len = (long long)W.n;
    a.err = ctx->d_err;
    if (logged) a.sv_out = sv.p;
    bool done = false;
    // the range finder pays only where the full factor is wide: narrower
    // cuts keep the plain SVD (and are still logged)
    if (learn && std::min(qcap[k], 4 * ocap[k + 1]) >= ctx->p.rf_min_width) {
      // range finder of predicted width (Halko et al. 2011, Alg. 4.1), then
      // the plain SVD unless the sketch holds all but eps^2 of the weight
      const int Wc = wcap[k];
      const int N4 = 4 * ocap[k + 1];
      const size_t cell = (size_t)slot * qtt_ctx_s::kBonds + k;
      const int prev = ctx->tab ^ 1;
      int* wdev = rfi.p;
      int* use_rf = rfi.p + 1;
      int* skip_full = rfi.p + 2;
      launch_rf_predict(ctx->d_mlp, ctx->d_feat[prev] + cell * QTT_MLP_FEATURES,
                        ctx->d_valid[prev] + cell, chi, over, Wc, qdims + k, Y->dims + k + 1, wdev,
                        use_rf, s);
      const unsigned long long key = ((unsigned long long)slot << 8) ^ (unsigned long long)k;
      launch_rf_omega(Om.p, ocap[k + 1], Y->dims + k + 1, Wc, wdev, key, s);
      gemm(gemm_plain(Mp, Om.p, Yr.p, qcap[k], Wc, N4, N4, Wc, Wc), s);  // Y = M Omega
      QrArgs q{};
      q.A = MatView{Yr.p, Wc, axis_prefix(qcap[k], dref(qdims + k)), axis_prefix(Wc, dref(wdev))};
      q.Q = MatView{Qy.p, Wc, axis_prefix(qcap[k], dref(qdims + k)), axis_prefix(Wc, dconst(1))};
      q.R = MatView{Rr.p, Wc, axis_prefix(Wc, dconst(1)), axis_prefix(Wc, dconst(1))};
      q.work = W.p;
      q.work_len = (long long)W.n;
      q.err = ctx->d_err;
      launch_qr_f64(q, qcap[k], Wc, s);
      {
        GemmF64 g = gemm_plain(Qy.p, Mp, Bb.p, Wc, N4, qcap[k], Wc, N4, N4);  // B = Q^T M
        g.tA = 1;
        gemm(g, s);
      }
      launch_sumsq2(Mp, (long long)qcap[k] * N4, Mp, 0, rfd.p, s);
      launch_sumsq2(Bb.p, (long long)Wc * N4, Bb.p, 0, rfd.p + 1, s);
      launch_rf_decide(rfd.p, rfd.p + 1, eps, use_rf, skip_full, rfd.p + 2, ctx->d_rf_counts, s);
      SvdArgs b = a;
      b.M = MatView{Bb.p, N4, axis_prefix(Wc, dref(wdev)), a.M.cols};
      b.US = MatView{Ubr.p, ocap[k], axis_prefix(Wc, dconst(1)), axis_prefix(ocap[k], dconst(1))};
      b.total_weight = rfd.p + 2;
      launch_svd_f64(b, Wc, N4, s);
      gemm(gemm_plain(Qy.p, Ubr.p, USb.p, qcap[k], ocap[k], Wc, Wc, ocap[k], ocap[k]), s);
      SvdArgs f = a;
      f.skip = skip_full;
      launch_svd_f64(f, qcap[k], N4, s);
      if (logged) {
        const int t = ctx->tab;
        launch_rf_features(sv.p, skip_full, wdev, qdims + k, Y->dims + k + 1, Y->dims + k, k, n,
                           ctx->d_feat[t] + cell * QTT_MLP_FEATURES, ctx->d_rank[t] + cell,
                           ctx->d_valid[t] + cell, s);
      }
      done = true;
    }
    if (!done && mixed) {
      // Rayleigh-Ritz: FP32 finds an oversampled subspace of right vectors,
      // one FP64 subspace iteration refines it and orthonormalises it, B =
      // M V is projected exactly and the (eps, chi) cut is made by an FP64
      // SVD of B, counting the weight of M outside the subspace
      // (|M|^2 - |B|^2, FP64) as discarded.
      const int rpo = std::min({qcap[k], 4 * ocap[k + 1], chi + kOver});
      SvdArgs a32 = a;
      a32.eps = -1.0;
      a32.chi = chi + kOver;
      a32.US = MatView{Bm.p, rpo, a.US.rows, axis_prefix(rpo, dconst(1))};
      a32.VT = MatView{Vt.p, 4 * ocap[k + 1], axis_prefix(rpo, dconst(1)), a.VT.cols};
      a32.r_out = rp.p;
      bool found = false;
      if (TCs.p && tc_search_supported(4 * ocap[k + 1], qcap[k], rpo)) {
        // right vectors of M: the subspace is on the column side (4 D_{k+1})
        TcSearch t{};
        t.X = Mp;
        t.ld = 4 * ocap[k + 1];
        t.rows = qcap[k];
        t.cols = 4 * ocap[k + 1];
        t.small_is_rows = 0;
        t.sact = DimRef{Y->dims + k + 1, 4};
        t.lact = dref(qdims + k);
        t.lact2 = dconst(1);
        t.lact2.p = nullptr;
        t.p = rpo;
        t.iters = tc_search_iters();
        t.key = 0x51ED0000ull + (unsigned long long)k;
        t.out = Vt.p;
        t.ldo = 4 * ocap[k + 1];
        t.outT = 1;
        t.r_out = rp.p;
        t.keep = std::min(chi, rpo);
        t.rho_max = tc_rho_max();
        t.accept = tca.p;
        t.stop = tca.p + 1;
        t.counts = ctx->d_rf_counts + 2;
        tc_search(t, TCs.p, TCs.n, ctx->d_err, s);
        // the FP32 cluster SVD overwrites the result unless it was accepted
        SvdArgs f32 = a32;
        f32.skip = tca.p;
        launch_svd_subspace_f32(f32, qcap[k], 4 * ocap[k + 1], s);
        found = true;
      }
      if (!found) found = launch_svd_subspace_f32(a32, qcap[k], 4 * ocap[k + 1], s);
      if (found) {
        QrArgs q{};
        q.A = MatView{Vt.p, 4 * ocap[k + 1], axis_prefix(rpo, dref(rp.p)), a.VT.cols};
        q.inT = 1;
        q.Q = MatView{Vt.p, 4 * ocap[k + 1], axis_prefix(rpo, dconst(1)), a.VT.cols};
        q.qT = 1;
        q.R = MatView{Rs.p, rpo, axis_prefix(rpo, dconst(1)), axis_prefix(rpo, dconst(1))};
        q.work = W.p;
        q.work_len = (long long)W.n;
        q.err = ctx->d_err;
        // one FP64 subspace iteration from the FP32 vectors V_32:
        // V = orth(M^T M V_32) = orth((B_0^T M)^T) with B_0 = M V_32.  The
        // FP32 search leaves every kept direction off by about the FP32
        // rounding of M (relative to |M|); the iteration shrinks that by
        // (sigma_{p+1} / sigma_i)^2, p = rpo, and its Householder QR makes V
        // orthonormal in FP64.  Then B = M V (qcap x rpo), and |M|_F^2.
        GemmF64 g = gemm_plain(Mp, Vt.p, Bm.p, qcap[k], rpo, 4 * ocap[k + 1], 4 * ocap[k + 1],
                               4 * ocap[k + 1], rpo);
        g.tB = 1;
        gemm(g, s);
        for (int it = 0; it < mixed_fp64_iters(); it++) {
          GemmF64 gz = gemm_plain(Bm.p, Mp, Vt.p, rpo, 4 * ocap[k + 1], qcap[k], rpo,
                                  4 * ocap[k + 1], 4 * ocap[k + 1]);
          gz.tA = 1;
          gemm(gz, s);
          launch_qr_f64(q, 4 * ocap[k + 1], rpo, s);
          gemm(g, s);
        }
        launch_sumsq2(Mp, (long long)qcap[k] * 4 * ocap[k + 1], Mp, 0, wM.p, s);
        // G = B^T B (rpo x rpo, into Rs, free after the subspace QR): its SVD
        // gives V_B and the weights sigma_B^2 without factoring B itself
        {
          GemmF64 gg = gemm_plain(Bm.p, Bm.p, Rs.p, rpo, rpo, qcap[k], rpo, rpo, rpo);
          gg.tA = 1;
          gemm_splitk(gg, s);
        }
        SvdArgs b64 = a;
        b64.M = MatView{Rs.p, rpo, axis_prefix(rpo, dref(rp.p)), axis_prefix(rpo, dref(rp.p))};
        b64.gram = 1;
        b64.no_us = 1;
        b64.VT = MatView{Vb.p, rpo, axis_prefix(ocap[k], dconst(1)), axis_prefix(rpo, dconst(1))};
        b64.total_weight = wM.p;
        launch_svd_f64(b64, rpo, rpo, s);
        // carry U_B S_B = B V_B  (qcap x ocap[k])
        {
          GemmF64 gc = gemm_plain(Bm.p, Vb.p, USb.p, qcap[k], ocap[k], rpo, rpo, rpo, ocap[k]);
          gc.tB = 1;
          gemm(gc, s);
        }
        // core = V_B^T V^T  (r x N)
        gemm(gemm_plain(Vb.p, Vt.p, Y->core(k), ocap[k], 4 * ocap[k + 1], rpo, rpo,
                        4 * ocap[k + 1], 4 * ocap[k + 1]), s);
        done = true;
      }
    }
    if (!done) {
      // only V^T from the factorisation (for a tall unfolding it needs
      // neither the rotation accumulator nor Q); the carry U S = M V is an
      // FP64 product
      a.no_us = 1;
      launch_svd_f64(a, qcap[k], 4 * ocap[k + 1], s);
      {
        GemmF64 gc = gemm_plain(Mp, Y->core(k), USb.p, qcap[k], ocap[k], 4 * ocap[k + 1],
                                4 * ocap[k + 1], 4 * ocap[k + 1], ocap[k]);
        gc.tB = 1;
        gemm(gc, s);
      }
      if (logged) {
        const size_t cell = (size_t)slot * qtt_ctx_s::kBonds + k;
        const int t = ctx->tab;
        launch_rf_features(sv.p, nullptr, nullptr, qdims + k, Y->dims + k + 1, Y->dims + k, k, n,
                           ctx->d_feat[t] + cell * QTT_MLP_FEATURES, ctx->d_rank[t] + cell,
                           ctx->d_valid[t] + cell, s);
      }
    }
  }
  // first core: Y_0 = Qcore_0 (4 x qcap[1]) * US (qcap[1] x ocap[1])
  {
    GemmF64 g = gemm_plain(qcore(0), USb.p, Y->core(0), 4, ocap[1], qcap[1], qcap[1],
                           ocap[1], ocap[1]);
    gemm(g, s);
  }
  return Y.release();
}

// ------------------------------------------------------------ apply / add
qtt_mps expand_mpo(qtt_ctx ctx, qtt_mpo W, qtt_mps A) {
  const int n = A->n;
  cudaStream_t s = stream_of(ctx);
  std::vector<int> cap(n + 1);
  for (int b = 0; b <= n; b++) cap[b] = A->cap[b] * W->w[b];
  MpsPtr X(new_mps(ctx, n, cap));
  for (int k = 0; k < n; k++)
    launch_mpo_expand(W->raw(k), W->w[k], W->w[k + 1], A->core(k), A->cap[k], A->cap[k + 1],
                      X->core(k), s);
  const int* src[1] = {A->dims};
  int mul[1][QTT_MAX_N + 1];
  for (int b = 0; b <= n; b++) mul[0][b] = W->w[b];
  launch_dims(src, mul, 1, n + 1, X->dims, s);
  return X.release();
}

qtt_mps add_exact(qtt_ctx ctx, int K, const double* coef, const qtt_mps* terms) {
  const int n = terms[0]->n;
  cudaStream_t s = stream_of(ctx);
  std::vector<int> cap(n + 1, 0);
  for (int b = 0; b <= n; b++)
    for (int t = 0; t < K; t++) cap[b] += terms[t]->cap[b];
  cap[0] = cap[n] = 1;
  MpsPtr X(new_mps(ctx, n, cap));
  for (int k = 0; k < n; k++) {
    AddTerm tt[8];
    for (int t = 0; t < K; t++)
      tt[t] = AddTerm{terms[t]->core(k), terms[t]->cap[k], terms[t]->cap[k + 1],
                      terms[t]->dims + k, terms[t]->dims + k + 1, coef[t]};
    launch_add_assemble(tt, K, k == 0, k == n - 1, X->core(k), cap[k], cap[k + 1], s);
  }
  const int* src[8];
  int mul[8][QTT_MAX_N + 1];
  for (int t = 0; t < K; t++) {
    src[t] = terms[t]->dims;
    for (int b = 0; b <= n; b++) mul[t][b] = 1;
  }
  launch_dims(src, mul, K, n + 1, X->dims, s);
  return X.release();
}

qtt_mps apply_impl(qtt_ctx ctx, qtt_mpo W, qtt_mps A, double eps, int chi) {
  MpsPtr X(expand_mpo(ctx, W, A));
  return compress_impl(ctx, X.get(), eps, chi);
}

qtt_mps add_impl(qtt_ctx ctx, int K, const double* coef, const qtt_mps* terms, double eps,
                 int chi) {
  if (K > 8) throw QttError(QTT_ERR_ARG, "qtt_add supports at most 8 terms");
  MpsPtr X(add_exact(ctx, K, coef, terms));
  return compress_impl(ctx, X.get(), eps, chi);
}

qtt_mps add2(qtt_ctx ctx, double c1, qtt_mps a, double c2, qtt_mps b) {
  const double cf[2] = {c1, c2};
  const qtt_mps t[2] = {a, b};
  return add_impl(ctx, 2, cf, t, ctx->p.eps, ctx->p.chi_max);
}

// ------------------------------------------------------------ Hadamard
qtt_mps hadamard_impl(qtt_ctx ctx, qtt_mps A, qtt_mps B, double eps, int chi) {
  const int n = A->n;
  cudaStream_t s = stream_of(ctx);
  const auto& ca = A->cap;
  const auto& cb = B->cap;
  std::vector<int> rcap(n + 1, 1);
  // the zip-up keeps min(4 r, Da Db, chi) directions; this may exceed the
  // natural bound 4^(n-b) (extra directions carry zero weight) and is
  // reduced by the compression that follows
  for (int b = 1; b < n; b++)
    rcap[b] = std::min({4 * rcap[b - 1], clampi((long long)ca[b] * cb[b]), chi});
  MpsPtr C(new_mps(ctx, n, rcap));
  launch_fill_int(C->dims, n + 1, 1, s);
  size_t xmax = 1, tmax = 1, rmax = 1, svw = 1;
  for (int k = 0; k < n; k++) {
    xmax = std::max(xmax, (size_t)rcap[k] * cb[k] * 4 * ca[k + 1]);
    tmax = std::max(tmax, (size_t)rcap[k] * 4 * ca[k + 1] * cb[k + 1]);
    rmax = std::max(rmax, (size_t)rcap[k] * ca[k] * cb[k]);
    if (k < n - 1)
      svw = std::max(svw, svd_work_doubles(4 * rcap[k], ca[k + 1] * cb[k + 1]));
  }
  const bool mixed = ctx->p.precision == QTT_PREC_MIXED;
  int rcmax = 1;
  for (int b = 0; b <= n; b++) rcmax = std::max(rcmax, rcap[b]);
  size_t qrw = 1;
  for (int k = 0; k < n - 1; k++) qrw = std::max(qrw, qr_work_doubles(4 * rcap[k], rcap[k + 1]));
  // mixed path buffers: oversampled factor, projected matrix, small factor
  constexpr int kOver = 16;
  size_t utm = 1, btm = 1, ubm = 1, rsm = 1;
  if (mixed) {
    for (int k = 0; k < n - 1; k++) {
      const size_t rpo = std::min({4 * rcap[k], ca[k + 1] * cb[k + 1], chi + kOver});
      utm = std::max(utm, (size_t)4 * rcap[k] * rpo);
      btm = std::max(btm, rpo * ca[k + 1] * cb[k + 1]);
      ubm = std::max(ubm, rpo * rcap[k + 1]);
      rsm = std::max(rsm, rpo * rpo);
      qrw = std::max(qrw, qr_work_doubles(4 * rcap[k], (int)rpo));
    }
  }
  DBuf<double> R0(rmax, s), R1(rmax, s), Xb(xmax, s), Tb(tmax, s), W(std::max(svw, qrw), s);
  size_t tcm = 0;
  if (mixed && tc_search_zipup())
    for (int k = 0; k < n - 1; k++) {
      const int rpo = std::min({4 * rcap[k], ca[k + 1] * cb[k + 1], chi + kOver});
      if (tc_search_supported(4 * rcap[k], ca[k + 1] * cb[k + 1], rpo))
        tcm = std::max(tcm, tc_search_scratch_floats(4 * rcap[k], ca[k + 1] * cb[k + 1], rpo));
    }
  DBuf<float> TCs(tcm, s);
  DBuf<int> tca(tcm ? 2 : 0, s);  // accept flag, stop word
  DBuf<double> Rs(mixed ? rsm : 0, s), Ut(mixed ? utm : 0, s), Bt(mixed ? btm : 0, s),
      Ub(mixed ? ubm : 0, s);
  DBuf<int> rp(1, s);
  (void)rcmax;
  launch_fill(R0.p, 1, 1.0, s);
  double* Rc = R0.p;
  double* Rn = R1.p;
  for (int k = 0; k < n; k++) {
    // X[r][b][s][a'] = sum_a R[r][a][b] A[a][s][a']
    GemmF64 g1{};
    g1.A = Rc; g1.B = A->core(k); g1.C = Xb.p;
    g1.M = cb[k]; g1.N = 4 * ca[k + 1]; g1.K = ca[k];
    g1.lda = cb[k]; g1.ldb = 4 * ca[k + 1]; g1.ldc = 4 * ca[k + 1];
    g1.tA = 1;
    g1.nb1 = rcap[k]; g1.nb2 = 1;
    g1.sA1 = (long long)ca[k] * cb[k]; g1.sB1 = 0; g1.sC1 = (long long)cb[k] * 4 * ca[k + 1];
    g1.alpha = 1.0; g1.beta = 0.0;
    gemm(g1, s);
    // T[r][s][a'][b'] = sum_b X[r][b][s][a'] B[b][s][b']
    double* Tout = (k == n - 1) ? C->core(n - 1) : Tb.p;
    GemmF64 g2{};
    g2.A = Xb.p; g2.B = B->core(k); g2.C = Tout;
    g2.M = ca[k + 1]; g2.N = cb[k + 1]; g2.K = cb[k];
    g2.lda = 4 * ca[k + 1]; g2.ldb = 4 * cb[k + 1]; g2.ldc = cb[k + 1];
    g2.tA = 1;
    g2.nb1 = rcap[k]; g2.nb2 = 4;
    g2.sA1 = (long long)cb[k] * 4 * ca[k + 1]; g2.sA2 = ca[k + 1];
    g2.sB1 = 0; g2.sB2 = cb[k + 1];
    g2.sC1 = (long long)4 * ca[k + 1] * cb[k + 1]; g2.sC2 = (long long)ca[k + 1] * cb[k + 1];
    g2.alpha = 1.0; g2.beta = 0.0;
    gemm(g2, s);
    if (k == n - 1) break;
    // zip-up split of T ((r,s) x (a',b')): core U, carry S V^T, cap only.
    // Factor T^T so that U comes out of the orthonormal V^T side.
    SvdArgs a{};
    a.M = MatView{Tb.p, ca[k + 1] * cb[k + 1], axis_pair(rcap[k], dref(C->dims + k), 4, dconst(4)),
                  axis_pair(ca[k + 1], dref(A->dims + k + 1), cb[k + 1], dref(B->dims + k + 1))};
    a.inT = 1;
    // US of T^T = V S  -> written transposed: carry (r' x (a',b'))
    a.US = MatView{Rn, ca[k + 1] * cb[k + 1], axis_prefix(rcap[k + 1], dconst(1)),
                   axis_pair(ca[k + 1], dref(A->dims + k + 1), cb[k + 1], dref(B->dims + k + 1))};
    a.usT = 1;
    // V^T of T^T = U^T -> written transposed: core ((r,s) x r')
    a.VT = MatView{C->core(k), rcap[k + 1], axis_pair(rcap[k], dref(C->dims + k), 4, dconst(4)),
                   axis_prefix(rcap[k + 1], dconst(1))};
    a.vtT = 1;
    a.eps = -1.0;
    a.chi = chi;
    a.rank_limit = dconst(1 << 30);
    a.r_out = C->dims + k + 1;
    a.work = W.p;
    a.work_len = (long long)W.n;
    a.err = ctx->d_err;
    bool done = false;
    if (mixed) {
      // Rayleigh-Ritz: FP32 finds an oversampled subspace (chi + kOver
      // directions), one FP64 subspace iteration refines it and
      // orthonormalises it (Householder), B = Q^T T is projected exactly
      // and the cap-chi cut is made by an FP64 SVD of B.
      const int rpo = std::min({4 * rcap[k], ca[k + 1] * cb[k + 1], chi + kOver});
      SvdArgs a32 = a;
      a32.chi = chi + kOver;
      a32.US = MatView{Bt.p, ca[k + 1] * cb[k + 1], axis_prefix(rpo, dconst(1)), a.US.cols};
      a32.VT = MatView{Ut.p, rpo, a.VT.rows, axis_prefix(rpo, dconst(1))};
      a32.r_out = rp.p;
      bool found = false;
      if (TCs.p && tc_search_supported(4 * rcap[k], ca[k + 1] * cb[k + 1], rpo)) {
        // left vectors of T ((r, s) x (a', b')): the subspace is on the row side
        TcSearch t{};
        t.X = Tb.p;
        t.ld = ca[k + 1] * cb[k + 1];
        t.rows = 4 * rcap[k];
        t.cols = ca[k + 1] * cb[k + 1];
        t.small_is_rows = 1;
        t.sact = DimRef{C->dims + k, 4};
        t.lact = dref(A->dims + k + 1);
        t.lact2 = dref(B->dims + k + 1);
        t.p = rpo;
        t.iters = tc_search_iters();
        t.key = 0x2A9000ull + (unsigned long long)k;
        t.out = Ut.p;
        t.ldo = rpo;
        t.outT = 0;
        t.r_out = rp.p;
        t.keep = std::min(chi, rpo);
        t.rho_max = tc_rho_max();
        t.accept = tca.p;
        t.stop = tca.p + 1;
        t.counts = ctx->d_rf_counts + 2;
        tc_search(t, TCs.p, TCs.n, ctx->d_err, s);
        // the FP32 cluster SVD overwrites the result unless it was accepted
        SvdArgs f32 = a32;
        f32.skip = tca.p;
        launch_svd_subspace_f32(f32, ca[k + 1] * cb[k + 1], 4 * rcap[k], s);
        found = true;
      }
      if (!found) found = launch_svd_subspace_f32(a32, ca[k + 1] * cb[k + 1], 4 * rcap[k], s);
      if (found) {
        QrArgs q{};
        q.A = MatView{Ut.p, rpo, a.VT.rows, axis_prefix(rpo, dref(rp.p))};
        q.Q = MatView{Ut.p, rpo, a.VT.rows, axis_prefix(rpo, dconst(1))};
        q.R = MatView{Rs.p, rpo, axis_prefix(rpo, dconst(1)), axis_prefix(rpo, dconst(1))};
        q.work = W.p;
        q.work_len = (long long)W.n;
        q.err = ctx->d_err;
        // one FP64 subspace iteration from the FP32 vectors U_32:
        // Q = orth(T T^T U_32) = orth(T B_0^T) with B_0 = U_32^T T (the FP32
        // search's error shrinks by (sigma_{p+1} / sigma_i)^2; the
        // Householder QR makes Q orthonormal in FP64); then B = Q^T T
        // (rpo x (a', b'))
        GemmF64 g = gemm_plain(Ut.p, Tb.p, Bt.p, rpo, ca[k + 1] * cb[k + 1], 4 * rcap[k], rpo,
                               ca[k + 1] * cb[k + 1], ca[k + 1] * cb[k + 1]);
        g.tA = 1;
        gemm(g, s);
        for (int it = 0; it < mixed_fp64_iters(); it++) {
          GemmF64 gy = gemm_plain(Tb.p, Bt.p, Ut.p, 4 * rcap[k], rpo, ca[k + 1] * cb[k + 1],
                                  ca[k + 1] * cb[k + 1], ca[k + 1] * cb[k + 1], rpo);
          gy.tB = 1;
          gemm(gy, s);
          launch_qr_f64(q, 4 * rcap[k], rpo, s);
          gemm(g, s);
        }
        // G = B B^T (rpo x rpo, into Rs): its SVD gives U_B (into Ub) for
        // the cap-chi cut without factoring the long B
        {
          GemmF64 gg = gemm_plain(Bt.p, Bt.p, Rs.p, rpo, rpo, ca[k + 1] * cb[k + 1],
                                  ca[k + 1] * cb[k + 1], ca[k + 1] * cb[k + 1], rpo);
          gg.tB = 1;
          gemm_splitk(gg, s);
        }
        SvdArgs b64 = a;
        b64.M = MatView{Rs.p, rpo, axis_prefix(rpo, dref(rp.p)), axis_prefix(rpo, dref(rp.p))};
        b64.inT = 0;
        b64.gram = 1;
        b64.no_us = 1;
        b64.VT = MatView{Ub.p, rcap[k + 1], axis_prefix(rpo, dconst(1)),
                         axis_prefix(rcap[k + 1], dconst(1))};
        b64.vtT = 1;
        launch_svd_f64(b64, rpo, rpo, s);
        // carry S_B V_B^T = U_B^T B  (r' x (a', b'))
        {
          GemmF64 gc = gemm_plain(Ub.p, Bt.p, Rn, rcap[k + 1], ca[k + 1] * cb[k + 1], rpo,
                                  rcap[k + 1], ca[k + 1] * cb[k + 1], ca[k + 1] * cb[k + 1]);
          gc.tA = 1;
          gemm(gc, s);
        }
        // core = Q U_B  ((r, s) x r')
        gemm(gemm_plain(Ut.p, Ub.p, C->core(k), 4 * rcap[k], rcap[k + 1], rpo, rpo, rcap[k + 1],
                        rcap[k + 1]), s);
        done = true;
      }
    }
    if (!done) {
      // only the core from the factorisation; the carry S V_T^T = U^T T is
      // an FP64 product ((r' x (r, s)) x ((r, s) x (a', b')))
      a.no_us = 1;
      launch_svd_f64(a, ca[k + 1] * cb[k + 1], 4 * rcap[k], s);
      GemmF64 gc = gemm_plain(C->core(k), Tb.p, Rn, rcap[k + 1], ca[k + 1] * cb[k + 1], 4 * rcap[k],
                              rcap[k + 1], ca[k + 1] * cb[k + 1], ca[k + 1] * cb[k + 1]);
      gc.tA = 1;
      gemm(gc, s);
    }
    std::swap(Rc, Rn);
  }
  // the zip-up leaves C left-canonical (orthonormal cores, centre at site n)
  return compress_impl(ctx, C.get(), eps, chi, true);
}

}  // namespace

// ===================================================================== projection
namespace {

struct Env {
  std::vector<DBuf<double>> b;  // per bond
};

// Launches captured inside WHILE bodies (nested ones included) since the
// enclosing capture began: they run once per pass, counted on the device.
thread_local long long t_body_launches = 0;
long long launches_now() { return g_launch_counter ? g_launch_counter->n : 0; }

// Appends to the graph that stream s is capturing a WHILE node whose body
// is captured from body(bs) on stream bs, followed by the loop condition:
// iteration i (0 on entry) runs while i < cap and *stop == 0, so the loop
// ends after at most cap iterations whatever the stop word does.  Each pass
// adds the kernels of this body (not of nested bodies, which count their
// own passes) to *launched.
template <typename F>
void capture_while(cudaStream_t s, cudaStream_t bs, int* counter, const int* stop, int cap,
                   long long* launched, F&& body) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  QTT_CUDA_CHECK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) throw QttError(QTT_ERR_CUDA, "device loop outside a capture");
  cudaGraphConditionalHandle h;
  QTT_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  launch_loop_cond(h, counter, stop, cap, 1, s);
  QTT_CUDA_CHECK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  QTT_CUDA_CHECK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  cudaGraph_t body_graph = cp.conditional.phGraph_out[0];
  QTT_CUDA_CHECK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies));
  QTT_CUDA_CHECK(cudaStreamBeginCaptureToGraph(bs, body_graph, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
  const long long before = launches_now(), nested0 = t_body_launches;
  t_body_launches = 0;
  try {
    body(bs);
    const long long own = launches_now() - before - t_body_launches + 1;  // + the condition
    launch_loop_cond(h, counter, stop, cap, 0, bs, own, launched);
  } catch (...) {
    t_body_launches = nested0;
    cudaGraph_t x = nullptr;
    cudaStreamEndCapture(bs, &x);
    throw;
  }
  t_body_launches = nested0 + (launches_now() - before);
  cudaGraph_t done = nullptr;
  QTT_CUDA_CHECK(cudaStreamEndCapture(bs, &done));
}

struct Projector {
  qtt_ctx ctx;
  cudaStream_t s;
  int n;
  double c;  // mu h^2
  qtt_mps V[2];
  qtt_mps W[2];
  qtt_mpo K[2][2];
  // environments per block, per bond
  std::vector<DBuf<double>> LE[2][2], RE[2][2], LW[2], RW[2];
  DBuf<double> t1, t2, rb, tmp, work, vt_i, vt_j, wt;
  DBuf<double> t1b, t2b;  // scratch of component 1's matvec row (runs beside row 0)
  DBuf<double> rb2, tmp2, work2, wt2;  // component 1's copies of rb, tmp, work, wt
  DBuf<double> t1c, t2c, t1d, t2d;     // scratch of the matvec's (i, j = 1) chains
  DBuf<double> zb[2];                   // row i's j = 1 block, added to Y_i at the end
  DBuf<double> cg_r[2], cg_p[2], cg_ap[2], rhs[2];
  DBuf<double> scal;
  DBuf<int> ist;
  size_t maxcore = 0;
  size_t maxout = 1;  // largest product output of the projection (split-K scratch sizing)
  // Extra right-hand-side terms (the paper's implicit form, App. B): the
  // right-hand side of component i is wcoef <basis|W_i> + sum over its terms
  // of coef <basis| P X>, P an MPO applied to the MPS X, each term with its
  // own environments of V_i against (P, X).
  //
  // kind 0: P a general MPO.  The two nonlinear kinds keep the Hadamard's
  // delta instead of forming the product MPO (P = H_B D or D H_B, bond
  // cap_B w): kind 1 is B (.) (D X), environments [a][c][p][e]; kind 2 is
  // D (B (.) X), environments [a][p][c][e] (a: V_i, c: B, p: D, e: X), each
  // site update four GEMMs (about a quarter of the product MPO's work).
  struct XTerm {
    double coef;
    qtt_mpo P;
    qtt_mps X;
    std::vector<DBuf<double>> L, R;
    int kind = 0;
    qtt_mps B = nullptr;
    qtt_mpo Dm = nullptr;
    int wbond(int k) const { return kind ? B->cap[k] * Dm->w[k] : P->w[k]; }
  };
  std::vector<XTerm> xt[2];
  double wcoef = 1.0;
  DBuf<double> xtT[2];  // transposed core of a term's X (right environments)
  DBuf<double> t3, t3b;  // third scratch of the nonlinear kinds (per component)

  const std::vector<int>& cap(int i) const { return V[i]->cap; }

  void alloc() {
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        LE[i][j].resize(n + 1);
        RE[i][j].resize(n + 1);
        for (int b = 0; b <= n; b++) {
          const size_t sz = (size_t)cap(i)[b] * K[i][j]->w[b] * cap(j)[b];
          LE[i][j][b] = DBuf<double>(sz, s);
          RE[i][j][b] = DBuf<double>(sz, s);
        }
      }
    for (int i = 0; i < 2; i++) {
      LW[i].resize(n + 1);
      RW[i].resize(n + 1);
      for (int b = 0; b <= n; b++) {
        LW[i][b] = DBuf<double>((size_t)cap(i)[b] * W[i]->cap[b], s);
        RW[i][b] = DBuf<double>((size_t)cap(i)[b] * W[i]->cap[b], s);
      }
    }
    size_t t1m = 1, t2m = 1, t3m = 1, cm = 1, qrw = 1;
    int wmax = 1;
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++)
        for (int b = 0; b <= n; b++) wmax = std::max(wmax, K[i][j]->w[b]);
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++)
        for (int k = 0; k < n; k++) {
          const size_t ci = cap(i)[k], cj = cap(j)[k], ci1 = cap(i)[k + 1], cj1 = cap(j)[k + 1];
          t1m = std::max(t1m, ci * wmax * 4 * cj1);          // left: a p t z
          t1m = std::max(t1m, ci1 * wmax * 4 * cj);          // right: b q t x
          t2m = std::max(t2m, ci * 4 * wmax * cj1);          // a s q z
          t2m = std::max(t2m, ci1 * 4 * wmax * cj);          // b s p x
          t1m = std::max(t1m, ci1 * 4 * (size_t)W[i]->cap[k]);
          t1m = std::max(t1m, ci * 4 * (size_t)W[i]->cap[k + 1]);
        }
    for (int i = 0; i < 2; i++)
      for (int k = 0; k < n; k++) {
        cm = std::max(cm, V[i]->core_size(k));
        cm = std::max(cm, W[i]->core_size(k));
        qrw = std::max(qrw, qr_work_doubles(4 * cap(i)[k], cap(i)[k + 1]));
        qrw = std::max(qrw, qr_work_doubles(4 * cap(i)[k + 1], cap(i)[k]));
      }
    for (int i = 0; i < 2; i++)
      for (XTerm& T : xt[i]) {
        T.L.resize(n + 1);
        T.R.resize(n + 1);
        for (int b = 0; b <= n; b++) {
          const size_t sz = (size_t)cap(i)[b] * T.wbond(b) * T.X->cap[b];
          T.L[b] = DBuf<double>(sz, s);
          T.R[b] = DBuf<double>(sz, s);
        }
        for (int k = 0; k < n; k++) {
          const size_t ci = cap(i)[k], ci1 = cap(i)[k + 1], cx = T.X->cap[k], cx1 = T.X->cap[k + 1];
          const size_t wl = T.wbond(k), wr = T.wbond(k + 1);
          // (wl, wr here count the product bond cap_B w; the nonlinear kinds'
          // three intermediates have the same sizes as the product MPO's two,
          // the third one's size taken into t3m)
          t1m = std::max({t1m, ci * wl * 4 * cx1, ci1 * wr * 4 * cx});
          t2m = std::max({t2m, ci * 4 * wr * cx1, ci1 * 4 * wl * cx});
          if (T.kind) {
            t3m = std::max({t3m, ci * 4 * wr * cx1, ci1 * 4 * wl * cx});
            // the middle intermediates take B's and D's bonds separately
            const size_t cb = T.B->cap[k], cb1 = T.B->cap[k + 1];
            const size_t dl = T.Dm->w[k], dr = T.Dm->w[k + 1];
            t2m = std::max({t2m, ci * cb * 4 * dr * cx1, ci * dl * 4 * cb1 * cx1,
                            ci1 * cb1 * 4 * dl * cx, ci1 * dr * 4 * cb * cx});
          }
          cm = std::max(cm, T.X->core_size(k));
        }
      }
    maxcore = cm;
    maxout = std::max({t1m, t2m, cm});
    for (int i = 0; i < 2; i++)
      for (XTerm& T : xt[i])
        for (int b = 0; b <= n; b++) maxout = std::max(maxout, T.L[b].n);
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++)
        for (int b = 0; b <= n; b++) maxout = std::max(maxout, LE[i][j][b].n);
    for (int i = 0; i < 2; i++)
      for (int b = 0; b <= n; b++) maxout = std::max(maxout, LW[i][b].n);
    t1 = DBuf<double>(t1m, s);
    t2 = DBuf<double>(t2m, s);
    t1b = DBuf<double>(t1m, s);
    t2b = DBuf<double>(t2m, s);
    int cmax = 1;
    for (int i = 0; i < 2; i++)
      for (int b = 0; b <= n; b++) cmax = std::max(cmax, cap(i)[b]);
    rb = DBuf<double>((size_t)cmax * cmax, s);
    maxout = std::max(maxout, (size_t)cmax * cmax);
    tmp = DBuf<double>(cm, s);
    work = DBuf<double>(qrw, s);
    t1c = DBuf<double>(t1m, s);
    t2c = DBuf<double>(t2m, s);
    t1d = DBuf<double>(t1m, s);
    t2d = DBuf<double>(t2m, s);
    for (int i = 0; i < 2; i++) zb[i] = DBuf<double>(cm, s);
    rb2 = DBuf<double>((size_t)cmax * cmax, s);
    tmp2 = DBuf<double>(cm, s);
    work2 = DBuf<double>(qrw, s);
    wt2 = DBuf<double>(cm, s);
    vt_i = DBuf<double>(cm, s);
    vt_j = DBuf<double>(cm, s);
    wt = DBuf<double>(cm, s);
    for (int i = 0; i < 2; i++) {
      cg_r[i] = DBuf<double>(cm, s);
      cg_p[i] = DBuf<double>(cm, s);
      cg_ap[i] = DBuf<double>(cm, s);
      rhs[i] = DBuf<double>(cm, s);
    }
    scal = DBuf<double>(8, s);
    ist = DBuf<int>(4, s);
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        launch_fill(LE[i][j][0].p, 1, 1.0, s);
        launch_fill(RE[i][j][n].p, 1, 1.0, s);
      }
    for (int i = 0; i < 2; i++) {
      launch_fill(LW[i][0].p, 1, 1.0, s);
      launch_fill(RW[i][n].p, 1, 1.0, s);
      for (XTerm& T : xt[i]) {
        launch_fill(T.L[0].p, 1, 1.0, s);
        launch_fill(T.R[n].p, 1, 1.0, s);
      }
      if (!xt[i].empty()) xtT[i] = DBuf<double>(cm, s);
    }
    bool nl = false;
    for (int i = 0; i < 2; i++)
      for (XTerm& T : xt[i]) nl = nl || T.kind != 0;
    if (nl) {
      t3 = DBuf<double>(t3m, s);
      t3b = DBuf<double>(t3m, s);
      maxout = std::max(maxout, t3m);
    }
  }

  // Steps 1-3 of a nonlinear term at site k from its left environment L:
  //   kind 1 (B (.) (D X)): T3[(a so)][(c' p' e')]
  //   kind 2 (D (B (.) X)): T3[(a so)][(p' c' e')]
  // (the left environment of bond k + 1 is V^T T3; the local right-hand side
  // is T3 R^T).
  void nl_left3(int i, XTerm& T, int k, const double* L, double* t1p, double* t2p, double* t3p) {
    const int ci = cap(i)[k];
    const int cb = T.B->cap[k], cb1 = T.B->cap[k + 1], wl = T.Dm->w[k], wr = T.Dm->w[k + 1];
    const int ce = T.X->cap[k], ce1 = T.X->cap[k + 1];
    const double* Bc = T.B->core(k);
    // T1[(a [c p | p c])][(t e')] = L[..][e] X[e][(t e')]
    gemm(gemm_plain(L, T.X->core(k), t1p, ci * cb * wl, 4 * ce1, ce, ce, 4 * ce1, 4 * ce1), s);
    if (T.kind == 1) {
      // T2[(a c)][(so p')][e'] = D2[(so p')][(p t)] T1[(a c)][(p t)][e']
      GemmF64 g{};
      g.A = T.Dm->k2(k); g.B = t1p; g.C = t2p;
      g.M = 4 * wr; g.N = ce1; g.K = 4 * wl;
      g.lda = 4 * wl; g.ldb = ce1; g.ldc = ce1;
      g.nb1 = ci * cb; g.nb2 = 1;
      g.sB1 = (long long)wl * 4 * ce1; g.sC1 = (long long)4 * wr * ce1;
      g.alpha = 1.0;
      mpo_gemm(g, T.Dm->sp_k2(k), s);
      // T3[(a so)][c'][(p' e')] = B_so[c][c']^T T2[(a c)][so][(p' e')], batch (a, so)
      GemmF64 h{};
      h.A = Bc; h.B = t2p; h.C = t3p;
      h.M = cb1; h.N = wr * ce1; h.K = cb;
      h.tA = 1; h.lda = 4 * cb1; h.ldb = 4 * wr * ce1; h.ldc = wr * ce1;
      h.nb1 = ci; h.nb2 = 4;
      h.sA1 = 0; h.sA2 = cb1;
      h.sB1 = (long long)cb * 4 * wr * ce1; h.sB2 = (long long)wr * ce1;
      h.sC1 = (long long)4 * cb1 * wr * ce1; h.sC2 = (long long)cb1 * wr * ce1;
      h.alpha = 1.0;
      gemm(h, s);
    } else {
      // T2[(a p)][t][c'][e'] = B_t[c][c']^T T1[(a p)][c][t][e'], batch (a p) for each t
      for (int t = 0; t < 4; t++) {
        GemmF64 h{};
        h.A = Bc + t * cb1; h.B = t1p + (long long)t * ce1; h.C = t2p + (long long)t * cb1 * ce1;
        h.M = cb1; h.N = ce1; h.K = cb;
        h.tA = 1; h.lda = 4 * cb1; h.ldb = 4 * ce1; h.ldc = ce1;
        h.nb1 = ci * wl; h.nb2 = 1;
        h.sA1 = 0; h.sB1 = (long long)cb * 4 * ce1; h.sC1 = (long long)4 * cb1 * ce1;
        h.alpha = 1.0;
        gemm(h, s);
      }
      // T3[a][(so p')][(c' e')] = D2[(so p')][(p t)] T2[a][(p t)][(c' e')], batch a
      GemmF64 g{};
      g.A = T.Dm->k2(k); g.B = t2p; g.C = t3p;
      g.M = 4 * wr; g.N = cb1 * ce1; g.K = 4 * wl;
      g.lda = 4 * wl; g.ldb = cb1 * ce1; g.ldc = cb1 * ce1;
      g.nb1 = ci; g.nb2 = 1;
      g.sB1 = (long long)wl * 4 * cb1 * ce1; g.sC1 = (long long)4 * wr * cb1 * ce1;
      g.alpha = 1.0;
      mpo_gemm(g, T.Dm->sp_k2(k), s);
    }
  }

  // Left environment of bond k + 1 of a nonlinear term.
  void nl_left(int i, XTerm& T, int k, double* t1p, double* t2p, double* t3p) {
    nl_left3(i, T, k, T.L[k].p, t1p, t2p, t3p);
    const int ci = cap(i)[k], ci1 = cap(i)[k + 1];
    const int n1 = T.B->cap[k + 1] * T.Dm->w[k + 1] * T.X->cap[k + 1];
    GemmF64 g = gemm_plain(V[i]->core(k), t3p, T.L[k + 1].p, ci1, n1, 4 * ci, ci1, n1, n1);
    g.tA = 1;
    gemm(g, s);
  }

  // Right environment of bond k of a nonlinear term from bond k + 1; ViT the
  // transposed V_i core [a'][so][a].
  void nl_right(int i, XTerm& T, int k, const double* ViT, double* t1p, double* t2p,
                double* t3p) {
    const int ci = cap(i)[k], ci1 = cap(i)[k + 1];
    const int cb = T.B->cap[k], cb1 = T.B->cap[k + 1], wl = T.Dm->w[k], wr = T.Dm->w[k + 1];
    const int ce = T.X->cap[k], ce1 = T.X->cap[k + 1];
    const double* Bc = T.B->core(k);
    launch_core_transpose(T.X->core(k), ce, ce1, xtT[i].p, s);
    // T1[(a' [c' p' | p' c'])][(t e)] = R[..][e'] XT[e'][(t e)]
    gemm(gemm_plain(T.R[k + 1].p, xtT[i].p, t1p, ci1 * cb1 * wr, 4 * ce, ce1, ce1, 4 * ce,
                    4 * ce), s);
    if (T.kind == 1) {
      // T2[(a' c')][(so p)][e] = DR2[(so p)][(p' t)] T1[(a' c')][(p' t)][e]
      GemmF64 g{};
      g.A = T.Dm->kr2(k); g.B = t1p; g.C = t2p;
      g.M = 4 * wl; g.N = ce; g.K = 4 * wr;
      g.lda = 4 * wr; g.ldb = ce; g.ldc = ce;
      g.nb1 = ci1 * cb1; g.nb2 = 1;
      g.sB1 = (long long)wr * 4 * ce; g.sC1 = (long long)4 * wl * ce;
      g.alpha = 1.0;
      mpo_gemm(g, T.Dm->sp_kr2(k), s);
      // T3[(a' so)][c][(p e)] = B_so[c][c'] T2[(a' c')][so][(p e)], batch (a', so)
      GemmF64 h{};
      h.A = Bc; h.B = t2p; h.C = t3p;
      h.M = cb; h.N = wl * ce; h.K = cb1;
      h.lda = 4 * cb1; h.ldb = 4 * wl * ce; h.ldc = wl * ce;
      h.nb1 = ci1; h.nb2 = 4;
      h.sA1 = 0; h.sA2 = cb1;
      h.sB1 = (long long)cb1 * 4 * wl * ce; h.sB2 = (long long)wl * ce;
      h.sC1 = (long long)4 * cb * wl * ce; h.sC2 = (long long)cb * wl * ce;
      h.alpha = 1.0;
      gemm(h, s);
    } else {
      // T2[(a' p')][t][c][e] = B_t[c][c'] T1[(a' p')][c'][t][e], batch (a' p') for each t
      for (int t = 0; t < 4; t++) {
        GemmF64 h{};
        h.A = Bc + t * cb1; h.B = t1p + (long long)t * ce; h.C = t2p + (long long)t * cb * ce;
        h.M = cb; h.N = ce; h.K = cb1;
        h.lda = 4 * cb1; h.ldb = 4 * ce; h.ldc = ce;
        h.nb1 = ci1 * wr; h.nb2 = 1;
        h.sA1 = 0; h.sB1 = (long long)cb1 * 4 * ce; h.sC1 = (long long)4 * cb * ce;
        h.alpha = 1.0;
        gemm(h, s);
      }
      // T3[a'][(so p)][(c e)] = DR2[(so p)][(p' t)] T2[a'][(p' t)][(c e)], batch a'
      GemmF64 g{};
      g.A = T.Dm->kr2(k); g.B = t2p; g.C = t3p;
      g.M = 4 * wl; g.N = cb * ce; g.K = 4 * wr;
      g.lda = 4 * wr; g.ldb = cb * ce; g.ldc = cb * ce;
      g.nb1 = ci1; g.nb2 = 1;
      g.sB1 = (long long)wr * 4 * cb * ce; g.sC1 = (long long)4 * wl * cb * ce;
      g.alpha = 1.0;
      mpo_gemm(g, T.Dm->sp_kr2(k), s);
    }
    // R[k][a][...] = ViT[(a' so)][a]^T T3[(a' so)][...]
    const int n0 = cb * wl * ce;
    GemmF64 g3 = gemm_plain(ViT, t3p, T.R[k].p, ci, n0, ci1 * 4, ci, n0, n0);
    g3.tA = 1;
    gemm(g3, s);
  }

  // A term's right environment at bond k from bond k + 1 (MPO sandwich, as
  // the coupling blocks with V_j replaced by X); ViT the transposed V_i core.
  void xterm_right(int i, XTerm& T, int k, const double* ViT, double* t1p, double* t2p) {
    const int wl = T.P->w[k], wr = T.P->w[k + 1];
    const int ci = cap(i)[k], ci1 = cap(i)[k + 1], cx = T.X->cap[k], cx1 = T.X->cap[k + 1];
    launch_core_transpose(T.X->core(k), cx, cx1, xtT[i].p, s);
    gemm(gemm_plain(T.R[k + 1].p, xtT[i].p, t1p, ci1 * wr, 4 * cx, cx1, cx1, 4 * cx, 4 * cx), s);
    GemmF64 g{};
    g.A = T.P->kr2(k); g.B = t1p; g.C = t2p;
    g.M = 4 * wl; g.N = cx; g.K = wr * 4;
    g.lda = wr * 4; g.ldb = cx; g.ldc = cx;
    g.nb1 = ci1; g.nb2 = 1;
    g.sA1 = 0; g.sB1 = (long long)wr * 4 * cx; g.sC1 = (long long)4 * wl * cx;
    g.alpha = 1.0;
    mpo_gemm(g, T.P->sp_kr2(k), s);
    GemmF64 g3 = gemm_plain(ViT, t2p, T.R[k].p, ci, wl * cx, ci1 * 4, ci, wl * cx, wl * cx);
    g3.tA = 1;
    gemm(g3, s);
  }

  // A term's left environment at bond k + 1 from bond k.
  void xterm_left(int i, XTerm& T, int k, double* t1p, double* t2p) {
    const int wl = T.P->w[k], wr = T.P->w[k + 1];
    const int ci = cap(i)[k], ci1 = cap(i)[k + 1], cx = T.X->cap[k], cx1 = T.X->cap[k + 1];
    gemm(gemm_plain(T.L[k].p, T.X->core(k), t1p, ci * wl, 4 * cx1, cx, cx, 4 * cx1, 4 * cx1), s);
    GemmF64 g{};
    g.A = T.P->k2(k); g.B = t1p; g.C = t2p;
    g.M = 4 * wr; g.N = cx1; g.K = 4 * wl;
    g.lda = 4 * wl; g.ldb = cx1; g.ldc = cx1;
    g.nb1 = ci; g.nb2 = 1;
    g.sA1 = 0; g.sB1 = (long long)wl * 4 * cx1; g.sC1 = (long long)4 * wr * cx1;
    g.alpha = 1.0;
    mpo_gemm(g, T.P->sp_k2(k), s);
    GemmF64 g3 = gemm_plain(V[i]->core(k), t2p, T.L[k + 1].p, ci1, wr * cx1, 4 * ci, ci1,
                            wr * cx1, wr * cx1);
    g3.tA = 1;
    gemm(g3, s);
  }

  // RE[b] from RE[b+1] and site b (sites b..n-1), all blocks + overlaps.
  void build_right(int k) {
    for (int j = 0; j < 2; j++) {
      // transposed copy of V_j[k] ([b][s][a]) into vt_j; reused for every i
      launch_core_transpose(V[j]->core(k), cap(j)[k], cap(j)[k + 1], j == 0 ? vt_i.p : vt_j.p, s);
    }
    by_component([&](int i) {
      double* const t1p = i == 0 ? t1.p : t1b.p;
      double* const t2p = i == 0 ? t2.p : t2b.p;
      const double* ViT = (i == 0) ? vt_i.p : vt_j.p;
      for (int j = 0; j < 2; j++) {
        const double* VjT = (j == 0) ? vt_i.p : vt_j.p;
        qtt_mpo Kij = K[i][j];
        const int wl = Kij->w[k], wr = Kij->w[k + 1];
        const int ci = cap(i)[k], cj = cap(j)[k], ci1 = cap(i)[k + 1], cj1 = cap(j)[k + 1];
        // T1[(b q)][(t x)] = RE[k+1][(b q)][z] * VjT[z][(t x)]
        gemm(gemm_plain(RE[i][j][k + 1].p, VjT, t1p, ci1 * wr, 4 * cj, cj1, cj1, 4 * cj, 4 * cj), s);
        // T2[b][(s p)][x] = KR2[(s p)][(q t)] * T1[b][(q t)][x]
        GemmF64 g{};
        g.A = Kij->kr2(k); g.B = t1p; g.C = t2p;
        g.M = 4 * wl; g.N = cj; g.K = wr * 4;
        g.lda = wr * 4; g.ldb = cj; g.ldc = cj;
        g.nb1 = ci1; g.nb2 = 1;
        g.sA1 = 0; g.sB1 = (long long)wr * 4 * cj; g.sC1 = (long long)4 * wl * cj;
        g.alpha = 1.0;
        mpo_gemm(g, Kij->sp_kr2(k), s);
        // RE[k][a][(p x)] = ViT[(b s)][a]^T * T2[(b s)][(p x)]
        GemmF64 g3 = gemm_plain(ViT, t2p, RE[i][j][k].p, ci, wl * cj, ci1 * 4, ci, wl * cj, wl * cj);
        g3.tA = 1;
        gemm(g3, s);
      }
      double* const wtp = i == 0 ? wt.p : wt2.p;
      const int ci = cap(i)[k], ci1 = cap(i)[k + 1];
      const int cw = W[i]->cap[k], cw1 = W[i]->cap[k + 1];
      launch_core_transpose(W[i]->core(k), cw, cw1, wtp, s);
      // T1[b][(s c)] = RW[k+1][b][d] * WiT[d][(s c)]
      gemm(gemm_plain(RW[i][k + 1].p, wtp, t1p, ci1, 4 * cw, cw1, cw1, 4 * cw, 4 * cw), s);
      // RW[k][a][c] = ViT[(b s)][a]^T * T1[(b s)][c]
      GemmF64 g = gemm_plain(ViT, t1p, RW[i][k].p, ci, cw, ci1 * 4, ci, cw, cw);
      g.tA = 1;
      gemm(g, s);
      double* const t3p = i == 0 ? t3.p : t3b.p;
      for (XTerm& T : xt[i]) {
        if (T.kind) nl_right(i, T, k, ViT, t1p, t2p, t3p);
        else xterm_right(i, T, k, ViT, t1p, t2p);
      }
    });
  }

  // LE[k+1] from LE[k] and site k.
  void build_left(int k) {
    by_component([&](int i) {
      double* const t1p = i == 0 ? t1.p : t1b.p;
      double* const t2p = i == 0 ? t2.p : t2b.p;
      for (int j = 0; j < 2; j++) {
        qtt_mpo Kij = K[i][j];
        const int wl = Kij->w[k], wr = Kij->w[k + 1];
        const int ci = cap(i)[k], cj = cap(j)[k], ci1 = cap(i)[k + 1], cj1 = cap(j)[k + 1];
        // T1[(a p)][(t z)] = LE[k][(a p)][x] * Vj[k][x][(t z)]
        gemm(gemm_plain(LE[i][j][k].p, V[j]->core(k), t1p, ci * wl, 4 * cj1, cj, cj, 4 * cj1, 4 * cj1), s);
        // T2[a][(s q)][z] = K2[(s q)][(p t)] * T1[a][(p t)][z]
        GemmF64 g{};
        g.A = Kij->k2(k); g.B = t1p; g.C = t2p;
        g.M = 4 * wr; g.N = cj1; g.K = 4 * wl;
        g.lda = 4 * wl; g.ldb = cj1; g.ldc = cj1;
        g.nb1 = ci; g.nb2 = 1;
        g.sA1 = 0; g.sB1 = (long long)wl * 4 * cj1; g.sC1 = (long long)4 * wr * cj1;
        g.alpha = 1.0;
        mpo_gemm(g, Kij->sp_k2(k), s);
        // LE[k+1][b][(q z)] = Vi[(a s)][b]^T * T2[(a s)][(q z)]
        GemmF64 g3 = gemm_plain(V[i]->core(k), t2p, LE[i][j][k + 1].p, ci1, wr * cj1, 4 * ci, ci1,
                                wr * cj1, wr * cj1);
        g3.tA = 1;
        gemm(g3, s);
      }
      const int ci = cap(i)[k], ci1 = cap(i)[k + 1];
      const int cw = W[i]->cap[k], cw1 = W[i]->cap[k + 1];
      // T1[a][(s d)] = LW[k][a][c] * Wi[c][(s d)]
      gemm(gemm_plain(LW[i][k].p, W[i]->core(k), t1p, ci, 4 * cw1, cw, cw, 4 * cw1, 4 * cw1), s);
      // LW[k+1][b][d] = Vi[(a s)][b]^T * T1[(a s)][d]
      GemmF64 g = gemm_plain(V[i]->core(k), t1p, LW[i][k + 1].p, ci1, cw1, 4 * ci, ci1, cw1, cw1);
      g.tA = 1;
      gemm(g, s);
      double* const t3p = i == 0 ? t3.p : t3b.p;
      for (XTerm& T : xt[i]) {
        if (T.kind) nl_left(i, T, k, t1p, t2p, t3p);
        else xterm_left(i, T, k, t1p, t2p);
      }
    });
  }

  // Y = (1 + c sum_j K_ij) X at site d; X, Y two-component local tensors.
  // Y_i = X_i + c sum_j (D_i^T D_j block applied to X_j); the two rows i run
  // on two worker streams (own scratch), joined back into the projection
  // stream.
  void matvec(int d, double* const X[2], double* const Y[2], const int* skip) {
    // four chains, one per block (i, j): Y_i = X_i + c K_i0-block(X_0) on
    // chain (i, 0), Z_i = c K_i1-block(X_1) on chain (i, 1), then Y_i += Z_i;
    // eagerly on the context's workers 0..3, inside a captured loop body on
    // that body's four streams (the workers belong to the enclosing capture)
    const cudaStream_t ps = s;
    cudaStream_t ch[4] = {ctx->workers[0], ctx->workers[1], ctx->workers[2], ctx->workers[3]};
    if (ctx->dev_loops) {
      const int lvl = ps == ctx->bstream[1] ? 1 : ps == ctx->bstream[0] ? 0 : -1;
      for (int q = 0; q < 4; q++) ch[q] = lvl >= 0 ? ctx->bworkers[lvl][q] : nullptr;
    }
    const bool par = ch[0] && ch[1] && ch[2] && ch[3];
    // events: fork, block (i, 1) done (i = 0, 1), rows joined (i = 0, 1)
    cudaEvent_t ev[5];
    for (int q = 0; q < 5; q++)
      ev[q] = ctx->dev_loops ? ctx->flow_ev[11 + q] : (q == 0 ? ctx->fork_ev : ctx->join_ev[q - 1]);
    if (par) {
      QTT_CUDA_CHECK(cudaEventRecord(ev[0], ps));
      for (int q = 0; q < 4; q++) QTT_CUDA_CHECK(cudaStreamWaitEvent(ch[q], ev[0], 0));
    }
    // each chain takes a quarter of the split-K scratch
    double* const scr = t_gemm_scratch;
    const size_t scr_n = t_gemm_scratch_n;
    double* const t1s[4] = {t1.p, t1b.p, t1c.p, t1d.p};
    double* const t2s[4] = {t2.p, t2b.p, t2c.p, t2d.p};
    auto block = [&](int i, int j, double* out, double beta, cudaStream_t cs) {
      const int q = 2 * j + i;  // chain index
      if (scr && par) {
        t_gemm_scratch = scr + q * (scr_n / 4);
        t_gemm_scratch_n = scr_n / 4;
      }
      double* const t1p = t1s[q];
      double* const t2p = t2s[q];
      qtt_mpo Kij = K[i][j];
      const int wl = Kij->w[d], wr = Kij->w[d + 1];
      const int ci = cap(i)[d], cj = cap(j)[d], ci1 = cap(i)[d + 1], cj1 = cap(j)[d + 1];
      GemmF64 g1 = gemm_plain(LE[i][j][d].p, X[j], t1p, ci * wl, 4 * cj1, cj, cj, 4 * cj1, 4 * cj1);
      g1.skip = skip;
      gemm(g1, cs);
      GemmF64 g{};
      g.A = Kij->k2(d); g.B = t1p; g.C = t2p;
      g.M = 4 * wr; g.N = cj1; g.K = 4 * wl;
      g.lda = 4 * wl; g.ldb = cj1; g.ldc = cj1;
      g.nb1 = ci; g.nb2 = 1;
      g.sA1 = 0; g.sB1 = (long long)wl * 4 * cj1; g.sC1 = (long long)4 * wr * cj1;
      g.alpha = 1.0;
      g.skip = skip;
      gemm(g, cs);
      // out[(a s)][b] (+)= c * T2[(a s)][(q z)] * RE[d+1][b][(q z)]^T
      GemmF64 g3 = gemm_plain(t2p, RE[i][j][d + 1].p, out, 4 * ci, ci1, wr * cj1, wr * cj1,
                              wr * cj1, ci1);
      g3.tB = 1;
      g3.alpha = c;
      g3.beta = beta;
      g3.skip = skip;
      gemm(g3, cs);
    };
    try {
      for (int i = 0; i < 2; i++) {
        const cudaStream_t c0 = par ? ch[i] : ps, c1 = par ? ch[2 + i] : ps;
        block(i, 1, zb[i].p, 0.0, c1);
        launch_copy(Y[i], X[i], V[i]->core_size(d), c0);
        block(i, 0, Y[i], 1.0, c0);
        if (par) {
          QTT_CUDA_CHECK(cudaEventRecord(ev[1 + i], c1));
          QTT_CUDA_CHECK(cudaStreamWaitEvent(c0, ev[1 + i], 0));
        }
        const int ci = cap(i)[d], ci1 = cap(i)[d + 1];
        launch_sum_slices(zb[i].p, 1, 4 * ci, ci1, Y[i], ci1, 1.0, 1.0, skip, c0);
      }
    } catch (...) {
      t_gemm_scratch = scr;
      t_gemm_scratch_n = scr_n;
      throw;
    }
    t_gemm_scratch = scr;
    t_gemm_scratch_n = scr_n;
    if (par) {
      for (int i = 0; i < 2; i++) {
        QTT_CUDA_CHECK(cudaEventRecord(ev[3 + i], ch[i]));
        QTT_CUDA_CHECK(cudaStreamWaitEvent(ps, ev[3 + i], 0));
      }
    }
  }

  void local_rhs(int d) {
    by_component([&](int i) {
      double* const t1p = i == 0 ? t1.p : t1b.p;
      double* const t2p = i == 0 ? t2.p : t2b.p;
      const int ci = cap(i)[d], ci1 = cap(i)[d + 1];
      const int cw = W[i]->cap[d], cw1 = W[i]->cap[d + 1];
      gemm(gemm_plain(LW[i][d].p, W[i]->core(d), t1p, ci, 4 * cw1, cw, cw, 4 * cw1, 4 * cw1), s);
      GemmF64 g = gemm_plain(t1p, RW[i][d + 1].p, rhs[i].p, 4 * ci, ci1, cw1, cw1, cw1, ci1);
      g.tB = 1;
      g.alpha = wcoef;
      gemm(g, s);
      // the implicit terms: rhs += coef L P X R (the coupling blocks' pattern)
      double* const t3p = i == 0 ? t3.p : t3b.p;
      for (XTerm& T : xt[i]) {
        if (T.kind) {
          nl_left3(i, T, d, T.L[d].p, t1p, t2p, t3p);
          const int n1 = T.B->cap[d + 1] * T.Dm->w[d + 1] * T.X->cap[d + 1];
          GemmF64 g3 = gemm_plain(t3p, T.R[d + 1].p, rhs[i].p, 4 * ci, ci1, n1, n1, n1, ci1);
          g3.tB = 1;
          g3.alpha = T.coef;
          g3.beta = 1.0;
          gemm(g3, s);
          continue;
        }
        const int wl = T.P->w[d], wr = T.P->w[d + 1];
        const int cx = T.X->cap[d], cx1 = T.X->cap[d + 1];
        gemm(gemm_plain(T.L[d].p, T.X->core(d), t1p, ci * wl, 4 * cx1, cx, cx, 4 * cx1, 4 * cx1), s);
        GemmF64 g2{};
        g2.A = T.P->k2(d); g2.B = t1p; g2.C = t2p;
        g2.M = 4 * wr; g2.N = cx1; g2.K = 4 * wl;
        g2.lda = 4 * wl; g2.ldb = cx1; g2.ldc = cx1;
        g2.nb1 = ci; g2.nb2 = 1;
        g2.sA1 = 0; g2.sB1 = (long long)wl * 4 * cx1; g2.sC1 = (long long)4 * wr * cx1;
        g2.alpha = 1.0;
        gemm(g2, s);
        GemmF64 g3 = gemm_plain(t2p, T.R[d + 1].p, rhs[i].p, 4 * ci, ci1, wr * cx1, wr * cx1,
                                wr * cx1, ci1);
        g3.tB = 1;
        g3.alpha = T.coef;
        g3.beta = 1.0;
        gemm(g3, s);
      }
    });
  }

  int solve(int d) {
    local_rhs(d);
    CgVec v{};
    double* X[2] = {V[0]->core(d), V[1]->core(d)};
    double* AP[2] = {cg_ap[0].p, cg_ap[1].p};
    double* P[2] = {cg_p[0].p, cg_p[1].p};
    for (int i = 0; i < 2; i++) {
      v.x[i] = X[i];
      v.r[i] = cg_r[i].p;
      v.p[i] = cg_p[i].p;
      v.ap[i] = cg_ap[i].p;
      v.len[i] = (long long)V[i]->core_size(d);
    }
    matvec(d, X, AP, nullptr);
    launch_cg_start(v, rhs[0].p, rhs[1].p, scal.p, ist.p, ctx->p.cg_tol, ctx->d_err, s);
    const int maxit = ctx->p.cg_maxit;
    if (ctx->dev_loops) {
      // a WHILE node of at most maxit iterations, ended by the CG's own stop
      // word (converged, iteration cap, breakdown): the host loop below
      // without its reads, iterations counted on the device
      const cudaStream_t outer = s;
      capture_while(outer, ctx->bstream[1], ctx->d_loop + 1, ist.p, maxit, ctx->d_stats + 3,
                    [&](cudaStream_t bs) {
        s = bs;
        matvec(d, P, AP, ist.p);
        launch_cg_step(v, scal.p, ist.p, maxit, ctx->d_err, s);
        s = outer;
      });
      launch_cg_account(ist.p, ctx->d_stats, maxit, s);
      return 0;
    }
    int done_iters = 0;
    const int chunk = 8;
    for (int it = 0; it < maxit; it += chunk) {
      const int m = std::min(chunk, maxit - it);
      for (int q = 0; q < m; q++) {
        matvec(d, P, AP, ist.p);
        launch_cg_step(v, scal.p, ist.p, maxit, ctx->d_err, s);
      }
      int h[2];
      QTT_CUDA_CHECK(cudaMemcpyAsync(h, ist.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      QTT_CUDA_CHECK(cudaStreamSynchronize(s));
      done_iters = h[1];
      if (h[0]) break;
    }
    if (done_iters >= maxit) ctx->last_not_converged = 1;
    return done_iters;
  }

  // centre moves right: V_i[d] = Q, V_i[d+1] = R V_i[d+1]
  // The two components' streams for work that splits by component: the
  // context's workers (eagerly, or in the enclosing capture of a step), or
  // the stream pair of the loop body being captured (a stream joined to one
  // capture cannot serve another).  Null: run on s.
  void row_streams(cudaStream_t out[2]) const {
    out[0] = ctx->workers[0];
    out[1] = ctx->workers[1];
    if (ctx->dev_loops) {
      const int lvl = s == ctx->bstream[1] ? 1 : s == ctx->bstream[0] ? 0 : -1;
      if (lvl >= 0) {
        out[0] = ctx->bworkers[lvl][0];
        out[1] = ctx->bworkers[lvl][1];
      }
    }
  }
  // f(i) for the two components, concurrently on the row streams (s is the
  // component's stream while f runs; each takes its own half of a split-K
  // scratch), joined back into s
  template <typename F>
  void by_component(F&& f) {
    const cudaStream_t ps = s;
    cudaStream_t rs[2];
    row_streams(rs);
    const bool par = rs[0] != nullptr && rs[1] != nullptr;
    cudaEvent_t fe = ctx->dev_loops ? ctx->flow_ev[12] : ctx->fork_ev;
    if (par) {
      QTT_CUDA_CHECK(cudaEventRecord(fe, ps));
      for (int i = 0; i < 2; i++) QTT_CUDA_CHECK(cudaStreamWaitEvent(rs[i], fe, 0));
    }
    double* const scr = t_gemm_scratch;
    const size_t scr_n = t_gemm_scratch_n;
    try {
      for (int i = 0; i < 2; i++) {
        s = par ? rs[i] : ps;
        if (scr && par) {
          t_gemm_scratch = scr + i * (scr_n / 2);
          t_gemm_scratch_n = scr_n / 2;
        }
        f(i);
      }
    } catch (...) {
      s = ps;
      t_gemm_scratch = scr;
      t_gemm_scratch_n = scr_n;
      throw;
    }
    s = ps;
    t_gemm_scratch = scr;
    t_gemm_scratch_n = scr_n;
    if (par) {
      for (int i = 0; i < 2; i++) {
        cudaEvent_t je = ctx->dev_loops ? ctx->flow_ev[13 + i] : ctx->join_ev[i];
        QTT_CUDA_CHECK(cudaEventRecord(je, rs[i]));
        QTT_CUDA_CHECK(cudaStreamWaitEvent(ps, je, 0));
      }
    }
  }

  void shift_right(int d) {
    by_component([&](int i) {
      double* const rbp = i == 0 ? rb.p : rb2.p;
      double* const tmpp = i == 0 ? tmp.p : tmp2.p;
      DBuf<double>& wk = i == 0 ? work : work2;
      const int cl = cap(i)[d], cr = cap(i)[d + 1], cr2 = cap(i)[d + 2];
      QrArgs a{};
      a.A = MatView{V[i]->core(d), cr, axis_pair(cl, dref(V[i]->dims + d), 4, dconst(4)),
                    axis_prefix(cr, dref(V[i]->dims + d + 1))};
      a.Q = MatView{V[i]->core(d), cr, axis_pair(cl, dref(V[i]->dims + d), 4, dconst(4)),
                    axis_prefix(cr, dconst(1))};
      a.R = MatView{rbp, cr, axis_prefix(cr, dconst(1)), axis_prefix(cr, dref(V[i]->dims + d + 1))};
      a.r_out = V[i]->dims + d + 1;
      a.work = wk.p;
      a.work_len = (long long)wk.n;
      a.err = ctx->d_err;
      launch_qr_f64(a, 4 * cl, cr, s);
      gemm(gemm_plain(rbp, V[i]->core(d + 1), tmpp, cr, 4 * cr2, cr, cr, 4 * cr2, 4 * cr2), s);
      launch_copy(V[i]->core(d + 1), tmpp, V[i]->core_size(d + 1), s);
    });
  }

  // centre moves left: V_i[d] = Q^T (right isometry), V_i[d-1] = V_i[d-1] R^T
  void shift_left(int d) {
    by_component([&](int i) {
      double* const rbp = i == 0 ? rb.p : rb2.p;
      double* const tmpp = i == 0 ? tmp.p : tmp2.p;
      DBuf<double>& wk = i == 0 ? work : work2;
      const int cl = cap(i)[d], cr = cap(i)[d + 1], cl0 = cap(i)[d - 1];
      QrArgs a{};
      a.A = MatView{V[i]->core(d), 4 * cr, axis_prefix(cl, dref(V[i]->dims + d)),
                    axis_pair(4, dconst(4), cr, dref(V[i]->dims + d + 1))};
      a.inT = 1;
      a.Q = MatView{V[i]->core(d), 4 * cr, axis_prefix(cl, dconst(1)),
                    axis_pair(4, dconst(4), cr, dref(V[i]->dims + d + 1))};
      a.qT = 1;
      a.R = MatView{rbp, cl, axis_prefix(cl, dref(V[i]->dims + d)), axis_prefix(cl, dconst(1))};
      a.rT = 1;
      a.r_out = V[i]->dims + d;
      a.work = wk.p;
      a.work_len = (long long)wk.n;
      a.err = ctx->d_err;
      launch_qr_f64(a, 4 * cr, cl, s);
      gemm(gemm_plain(V[i]->core(d - 1), rbp, tmpp, 4 * cl0, cl, cl, cl, cl, cl), s);
      launch_copy(V[i]->core(d - 1), tmpp, V[i]->core_size(d - 1), s);
    });
  }

  double norm_total() {
    launch_sumsq2(V[0]->core(0), (long long)V[0]->core_size(0), V[1]->core(0),
                  (long long)V[1]->core_size(0), scal.p + 6, s);
    double h;
    QTT_CUDA_CHECK(cudaMemcpyAsync(&h, scal.p + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA_CHECK(cudaStreamSynchronize(s));
    return h;
  }
};

qtt_mps copy_mps(qtt_ctx ctx, qtt_mps A) {
  MpsPtr X(new_mps(ctx, A->n, A->cap));
  launch_copy(X->data, A->data, A->off[A->n], stream_of(ctx));
  QTT_CUDA_CHECK(cudaMemcpyAsync(X->dims, A->dims, (A->n + 1) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, stream_of(ctx)));
  return X.release();
}

// The sweeps of a projector whose V, W, K and terms are set (Sec. II.C,
// App. B): environments allocated here, centre brought to site 1, then
// single-site sweeps until the norm test or the cap; the results are V0, V1.
void run_projection(qtt_ctx ctx, Projector& P, MpsPtr& V0, MpsPtr& V1, qtt_mps* v1,
                    qtt_mps* v2, int* cg_out, int* sw_out) {
  const int n = P.n;
  P.alloc();
  // a quarter per matvec chain; a quarter holds 16 split-K slices of the
  // largest output, or 64 of an output up to kOzWideSplitMN (the emulated
  // GEMM's wide split)
  const size_t quarter = std::max<size_t>(16 * P.maxout,
                                          64 * std::min<size_t>(P.maxout, kOzWideSplitMN));
  DBuf<double> arena(ctx->dev_loops ? 4 * quarter : 0, P.s);
  struct ScratchScope {  // split-K scratch of a captured step's loop bodies
    explicit ScratchScope(DBuf<double>& a) {
      t_gemm_scratch = a.p;
      t_gemm_scratch_n = a.n;
    }
    ~ScratchScope() {
      t_gemm_scratch = nullptr;
      t_gemm_scratch_n = 0;
    }
  };
  std::unique_ptr<ScratchScope> scope(ctx->dev_loops ? new ScratchScope(arena) : nullptr);
  // right-canonical initial guess (centre at site 1)
  for (int d = n - 1; d >= 1; d--) P.shift_left(d);
  for (int k = n - 1; k >= 1; k--) P.build_right(k);
  if (ctx->dev_loops) {
    // the sweep loop as a WHILE node (each solve a nested one): the host
    // loop below with its convergence test on the device
    launch_sumsq2(P.V[0]->core(0), (long long)P.V[0]->core_size(0), P.V[1]->core(0),
                  (long long)P.V[1]->core_size(0), P.scal.p + 6, P.s);
    launch_sweep_check(P.scal.p, ctx->d_loop + 2, ctx->d_stats, ctx->p.sweep_tol, 1, P.s);
    if (n > 1) {
      const cudaStream_t outer = P.s;
      capture_while(outer, ctx->bstream[0], ctx->d_loop + 0, ctx->d_loop + 2, ctx->p.max_sweeps,
                    ctx->d_stats + 3, [&](cudaStream_t bs) {
                      P.s = bs;
                      for (int d = 0; d < n - 1; d++) {
                        P.solve(d);
                        P.shift_right(d);
                        P.build_left(d);
                      }
                      for (int d = n - 1; d >= 1; d--) {
                        P.solve(d);
                        P.shift_left(d);
                        P.build_right(d);
                      }
                      launch_sumsq2(P.V[0]->core(0), (long long)P.V[0]->core_size(0),
                                    P.V[1]->core(0), (long long)P.V[1]->core_size(0),
                                    P.scal.p + 6, P.s);
                      launch_sweep_check(P.scal.p, ctx->d_loop + 2, ctx->d_stats,
                                         ctx->p.sweep_tol, 0, P.s);
                      P.s = outer;
                    });
      launch_sweep_final(ctx->d_loop + 2, ctx->d_stats, P.s);
    }
    if (cg_out) *cg_out = 0;
    if (sw_out) *sw_out = 0;
    *v1 = V0.release();
    *v2 = V1.release();
    return;
  }
  long long cg = 0;
  int sweeps = 0;
  ctx->last_not_converged = 0;
  double nprev = P.norm_total();
  bool conv = false;
  for (int sw = 0; sw < ctx->p.max_sweeps; sw++) {
    for (int d = 0; d < n - 1; d++) {
      cg += P.solve(d);
      P.shift_right(d);
      P.build_left(d);
    }
    for (int d = n - 1; d >= 1; d--) {
      cg += P.solve(d);
      P.shift_left(d);
      P.build_right(d);
    }
    sweeps = sw + 1;
    const double nn = P.norm_total();
    if (nn == 0.0 || fabs(nn - nprev) <= ctx->p.sweep_tol * nn) {
      conv = true;
      break;
    }
    nprev = nn;
  }
  if (n == 1) conv = true;
  if (!conv) ctx->last_not_converged = 1;
  ctx->cg_iters += cg;
  ctx->sweeps += sweeps;
  if (cg_out) *cg_out = (int)cg;
  if (sw_out) *sw_out = sweeps;
  *v1 = V0.release();
  *v2 = V1.release();
}

void project_impl(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, double h, double mu, qtt_mps* v1,
                  qtt_mps* v2, int* cg_out, int* sw_out) {
  Projector P;
  P.ctx = ctx;
  P.s = ctx->stream;
  P.n = w1->n;
  P.c = mu * h * h;
  MpsPtr V0(copy_mps(ctx, w1)), V1(copy_mps(ctx, w2));
  P.V[0] = V0.get();
  P.V[1] = V1.get();
  P.W[0] = w1;
  P.W[1] = w2;
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) P.K[i][j] = ctx->K[i][j];
  run_projection(ctx, P, V0, V1, v1, v2, cg_out, sw_out);
}

// The product MPO of the Hadamard MPO of b with W (order 0: H_b W, so that
// P X = b (.) (W X); order 1: W H_b, P X = W (b (.) X)), built on the device
// at the capacities of b and W (bond cap_b w); the memory is `buf`.
std::unique_ptr<qtt_mpo_s> hadamard_mpo_device(qtt_ctx ctx, qtt_mps b, qtt_mpo W, int order,
                                               DBuf<double>& buf) {
  const int n = b->n;
  cudaStream_t s = stream_of(ctx);
  std::unique_ptr<qtt_mpo_s> m(new qtt_mpo_s);
  m->n = n;
  m->w.resize(n + 1);
  for (int k = 0; k <= n; k++) m->w[k] = b->cap[k] * W->w[k];
  m->off.resize(n + 1);
  size_t o = 0;
  for (int k = 0; k < n; k++) {
    m->off[k] = o;
    o += (size_t)m->w[k] * 16 * m->w[k + 1];
  }
  m->off[n] = o;
  buf = DBuf<double>(3 * o, s);
  m->dev = buf.p;
  m->dev_k2 = buf.p + o;
  m->dev_kr2 = buf.p + 2 * o;
  for (int k = 0; k < n; k++)
    launch_hadamard_mpo(b->core(k), b->cap[k], b->cap[k + 1], W->raw(k), W->w[k], W->w[k + 1],
                        order, m->raw(k), m->k2(k), m->kr2(k), s);
  return m;
}

// The projection with the paper's implicit right-hand side (Sec. II.C,
// App. B, Eq. for B_i inside the cost Theta): a u_i - h B_i(b) is never
// formed; component i's local right-hand side sums a <u_i>, -h/2 <(H_{b_j}
// D_j) b_i>, -h/2 <(D_j H_{b_j}) b_i> (j = 1, 2) and h nu <Lap b_i>, each
// through its own environments.  Initial guess a u (the paper: the previous
// time step), so the result keeps the bonds of u.
void project_implicit_impl(qtt_ctx ctx, qtt_mps u[2], qtt_mps b[2], double h, double nu,
                           double a_scale, qtt_mps* v1, qtt_mps* v2, int* cg_out, int* sw_out) {
  // QTT_IMPLICIT_PRODUCT: contract the product MPOs H_b D_j, D_j H_b (built
  // on the device) instead of the structured nonlinear terms (same sums)
  static const bool product = getenv("QTT_IMPLICIT_PRODUCT") != nullptr;
  DBuf<double> mbuf[4];
  std::unique_ptr<qtt_mpo_s> HD[2], DH[2];
  for (int j = 0; j < 2 && product; j++) {
    HD[j] = hadamard_mpo_device(ctx, b[j], ctx->D[j], 0, mbuf[2 * j]);
    DH[j] = hadamard_mpo_device(ctx, b[j], ctx->D[j], 1, mbuf[2 * j + 1]);
  }
  Projector P;
  P.ctx = ctx;
  P.s = ctx->stream;
  P.n = u[0]->n;
  P.c = ctx->p.mu * h * h;
  MpsPtr V0(add_exact(ctx, 1, &a_scale, &u[0])), V1(add_exact(ctx, 1, &a_scale, &u[1]));
  P.V[0] = V0.get();
  P.V[1] = V1.get();
  P.W[0] = u[0];
  P.W[1] = u[1];
  P.wcoef = a_scale;
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) P.K[i][j] = ctx->K[i][j];
  for (int i = 0; i < 2; i++) {
    for (int j = 0; j < 2; j++) {
      if (product) {
        P.xt[i].push_back(Projector::XTerm{-0.5 * h, HD[j].get(), b[i], {}, {}});
        P.xt[i].push_back(Projector::XTerm{-0.5 * h, DH[j].get(), b[i], {}, {}});
      } else {
        P.xt[i].push_back(Projector::XTerm{-0.5 * h, nullptr, b[i], {}, {}, 1, b[j], ctx->D[j]});
        P.xt[i].push_back(Projector::XTerm{-0.5 * h, nullptr, b[i], {}, {}, 2, b[j], ctx->D[j]});
      }
    }
    P.xt[i].push_back(Projector::XTerm{h * nu, ctx->lap, b[i], {}, {}});
  }
  run_projection(ctx, P, V0, V1, v1, v2, cg_out, sw_out);
}

// ===================================================================== RK4
// Concurrency of independent operations: fork() makes every worker stream
// wait for the context stream, run(k, f) enqueues operation f on worker k,
// join() makes the context stream wait for every worker and hands the
// outputs (allocated on workers) to the context stream for release.  These
// are the first kStageWorkers streams; the last two carry the running sum
// of the RK4 stages (rk4_core) and are forked and joined there.
struct Workers {
  qtt_ctx ctx;
  bool serial;
  explicit Workers(qtt_ctx c) : ctx(c) {
    static const bool ser = getenv("QTT_SERIAL") != nullptr;
    serial = ser || !c->workers[0];
  }
  void fork() {
    if (serial) return;
    QTT_CUDA_CHECK(cudaEventRecord(ctx->fork_ev, ctx->stream));
    for (int k = 0; k < qtt_ctx_s::kStageWorkers; k++)
      QTT_CUDA_CHECK(cudaStreamWaitEvent(ctx->workers[k], ctx->fork_ev, 0));
  }
  template <typename F>
  qtt_mps run(int k, F&& f) {
    if (serial) return f();
    if (k < 0 || k >= qtt_ctx_s::kStageWorkers) throw QttError(QTT_ERR_ARG, "worker index");
    ctx->cur = ctx->workers[k];
    qtt_mps out = nullptr;
    try {
      out = f();
    } catch (...) {
      ctx->cur = nullptr;
      throw;
    }
    ctx->cur = nullptr;
    return out;
  }
  // cross-stream dependency: worker `to` waits for everything enqueued so far
  // on worker `from` (an event of the context's pool, reused stage by stage)
  int nflow = 0;
  void after(int to, int from) {
    if (serial || to == from) return;
    if (nflow >= qtt_ctx_s::kFlowEvents) throw QttError(QTT_ERR_ARG, "flow event pool exhausted");
    if (to < 0 || from < 0 || to >= qtt_ctx_s::kStageWorkers || from >= qtt_ctx_s::kStageWorkers)
      throw QttError(QTT_ERR_ARG, "worker index");
    cudaEvent_t e = ctx->flow_ev[nflow++];
    QTT_CUDA_CHECK(cudaEventRecord(e, ctx->workers[from]));
    QTT_CUDA_CHECK(cudaStreamWaitEvent(ctx->workers[to], e, 0));
  }
  void join(std::initializer_list<qtt_mps> outs) {
    if (serial) return;
    for (int k = 0; k < qtt_ctx_s::kStageWorkers; k++) {
      QTT_CUDA_CHECK(cudaEventRecord(ctx->join_ev[k], ctx->workers[k]));
      QTT_CUDA_CHECK(cudaStreamWaitEvent(ctx->stream, ctx->join_ev[k], 0));
    }
    for (qtt_mps m : outs)
      if (m) m->stream = ctx->stream;
  }
};

// The exact spectral projection (the alternative to the penalty that the
// paper's outlook, Sec. IV, points to for periodic boundaries): both
// components read out densely, the divergence removed per Fourier mode on
// the device (launch_spectral_project: the orthogonal projection onto the
// kernel of [D_1 D_2], the penalty's mu -> infinity limit), then each
// component encoded again by TT-SVD to the context's (eps, chi_max), the two
// encodings on two worker streams.
qtt_mps from_dense_impl(qtt_ctx ctx, const double* F, double eps, int chi);
void to_dense_impl(qtt_ctx ctx, qtt_mps A, double* F);

void project_spectral_impl(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, qtt_mps* v1, qtt_mps* v2) {
  const int n = w1->n;
  if (w2->n != n) throw QttError(QTT_ERR_SHAPE, "components on different grids");
  if (n > 13) throw QttError(QTT_ERR_SHAPE, "spectral projection: n > 13");
  cudaStream_t s = stream_of(ctx);
  const size_t N = (size_t)1 << n, NN = N * N;
  DBuf<double> F1(NN, s), F2(NN, s), sig(N, s);
  {
    DBuf<double2> C1(NN, s), C2(NN, s);
    to_dense_impl(ctx, w1, F1.p);
    to_dense_impl(ctx, w2, F2.p);
    const std::vector<double> c = central_weights(ctx->p.fd_order == 0 ? 2 : ctx->p.fd_order);
    launch_spectral_project(F1.p, F2.p, n, c.data(), (int)c.size(), ctx->p.L / (double)N, C1.p,
                            C2.p, sig.p, s);
  }
  Workers wk(ctx);
  wk.fork();
  MpsPtr o[2];
  for (int i = 0; i < 2; i++)
    o[i] = MpsPtr(wk.run(i, [&] { return from_dense_impl(ctx, i ? F2.p : F1.p, ctx->p.eps,
                                                          ctx->p.chi_max); }));
  wk.join({o[0].get(), o[1].get()});
  *v1 = o[0].release();
  *v2 = o[1].release();
}

// The projection of one Euler minimisation with an explicit right-hand side
// w: the paper's penalty solve or, with QTT_PROJ_SPECTRAL, the exact one.
void project_stage(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, double h, qtt_mps* v1, qtt_mps* v2,
                   int* cg_out, int* sw_out) {
  if (ctx->p.projection == QTT_PROJ_SPECTRAL) {
    project_spectral_impl(ctx, w1, w2, v1, v2);
    ctx->last_not_converged = 0;
    if (cg_out) *cg_out = 0;
    if (sw_out) *sw_out = 0;
    return;
  }
  project_impl(ctx, w1, w2, h, ctx->p.mu, v1, v2, cg_out, sw_out);
}

void stage_w(qtt_ctx ctx, qtt_mps u[2], qtt_mps b[2], double h, double nu, MpsPtr w[2],
             double a_scale = 0.25) {
  const double eps = ctx->p.eps;
  const int chi = ctx->p.chi_max;
  Workers wk(ctx);
  MpsPtr Db[2][2], P[2][2], Q[2][2], DQ[2][2], Lb[2];
  MpsPtr ca[2], cb[2], conv[2], e[2];
  // Dataflow over the worker streams: every operation starts as soon as its
  // own inputs are done (an operation on its input's stream is ordered by
  // the stream, others wait on an event), instead of wave by wave.
  //   streams 0-3  D_j b_i -> b_j (.) D_j b_i -> (i: sum over j -> conv -> w)
  //   streams 4-6  b_j (.) b_i -> D_j (b_j (.) b_i)
  //   stream  9    D_1 (b_1 (.) b_0) (waits for stream 5)
  //   streams 7-8  Lap b_i -> e_i = a u_i + h nu Lap b_i
  // The viscous term is folded into e (w = e - h conv), off the chain of
  // sums that follows the last Hadamard product.
  auto sDb = [](int j, int i) { return 2 * i + j; };
  wk.fork();
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      Db[j][i] = MpsPtr(wk.run(sDb(j, i), [&] { return apply_impl(ctx, ctx->D[j], b[i], eps, chi); }));
  Q[0][0] = MpsPtr(wk.run(4, [&] { return hadamard_impl(ctx, b[0], b[0], eps, chi); }));
  Q[0][1] = MpsPtr(wk.run(5, [&] { return hadamard_impl(ctx, b[0], b[1], eps, chi); }));
  Q[1][1] = MpsPtr(wk.run(6, [&] { return hadamard_impl(ctx, b[1], b[1], eps, chi); }));
  for (int i = 0; i < 2; i++)
    Lb[i] = MpsPtr(wk.run(7 + i, [&] { return apply_impl(ctx, ctx->lap, b[i], eps, chi); }));
  // b_j (.) D_j b_i on the stream of D_j b_i
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++)
      P[j][i] = MpsPtr(wk.run(sDb(j, i), [&] { return hadamard_impl(ctx, b[j], Db[j][i].get(), eps, chi); }));
  // D_j (b_j (.) b_i): q(j, i) is Q00, Q01 (for (0,1) and (1,0)) or Q11
  wk.after(9, 5);  // before D_0 Q01 is queued on stream 5: waits for Q01 only
  DQ[0][0] = MpsPtr(wk.run(4, [&] { return apply_impl(ctx, ctx->D[0], Q[0][0].get(), eps, chi); }));
  DQ[0][1] = MpsPtr(wk.run(5, [&] { return apply_impl(ctx, ctx->D[0], Q[0][1].get(), eps, chi); }));
  DQ[1][0] = MpsPtr(wk.run(9, [&] { return apply_impl(ctx, ctx->D[1], Q[0][1].get(), eps, chi); }));
  DQ[1][1] = MpsPtr(wk.run(6, [&] { return apply_impl(ctx, ctx->D[1], Q[1][1].get(), eps, chi); }));
  // the sums of component i on stream sDb(0, i)
  const int sDQ[2][2] = {{4, 5}, {9, 6}};  // stream of DQ[j][i]
  for (int i = 0; i < 2; i++) {
    const int si = sDb(0, i);
    wk.after(si, sDb(1, i));
    ca[i] = MpsPtr(wk.run(si, [&] { return add2(ctx, 1.0, P[0][i].get(), 1.0, P[1][i].get()); }));
    // D_0 q + D_1 q on the stream of DQ[0][i], after DQ[1][i]
    wk.after(sDQ[0][i], sDQ[1][i]);
    cb[i] = MpsPtr(wk.run(sDQ[0][i], [&] { return add2(ctx, 1.0, DQ[0][i].get(), 1.0, DQ[1][i].get()); }));
    e[i] = MpsPtr(wk.run(7 + i, [&] { return add2(ctx, a_scale, u[i], h * nu, Lb[i].get()); }));
    wk.after(si, sDQ[0][i]);
    conv[i] = MpsPtr(wk.run(si, [&] { return add2(ctx, 0.5, ca[i].get(), 0.5, cb[i].get()); }));
    wk.after(si, 7 + i);
    w[i] = MpsPtr(wk.run(si, [&] { return add2(ctx, 1.0, e[i].get(), -h, conv[i].get()); }));
  }
  // every worker joins the context stream; all outputs and intermediates
  // are then released on it
  wk.join({Db[0][0].get(), Db[0][1].get(), Db[1][0].get(), Db[1][1].get(), Q[0][0].get(),
           Q[0][1].get(), Q[1][1].get(), Lb[0].get(), Lb[1].get(), P[0][0].get(), P[0][1].get(),
           P[1][0].get(), P[1][1].get(), DQ[0][0].get(), DQ[0][1].get(), DQ[1][0].get(),
           DQ[1][1].get(), ca[0].get(), ca[1].get(), cb[0].get(), cb[1].get(), conv[0].get(),
           conv[1].get(), e[0].get(), e[1].get(), w[0].get(), w[1].get()});
}

// ------------------------------------------------ stage graphs (params.graphs)
// The right-hand side of a stage issues thousands of launches over the
// worker streams and never waits for the device, so it can be captured once
// and replayed: a key's first occurrence runs eagerly (one-off shapes, such
// as a state just read from host memory, are never captured); the second
// runs eagerly (every product shape is then tuned) and is captured into a
// graph on graph-owned buffers; later occurrences copy their inputs in,
// launch the graph and copy the outputs out (device-to-device, a few MB).
// The kernels, their per-stream order and their arguments are those of the
// eager run, so the results are the same bit for bit.  h is part of the key:
// replays pay off with a fixed time step.
std::string stage_key(qtt_mps u[2], qtt_mps b[2], bool alias, double h, double nu, double a) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  put(&alias, sizeof alias);
  put(&h, sizeof h);
  put(&nu, sizeof nu);
  put(&a, sizeof a);
  for (int i = 0; i < (alias ? 2 : 4); i++) {
    const qtt_mps m = i < 2 ? u[i] : b[i - 2];
    put(m->cap.data(), m->cap.size() * sizeof(int));
  }
  return k;
}

void copy_mps_d2d(qtt_mps dst, qtt_mps src, cudaStream_t s) {
  if (dst->cap != src->cap) throw QttError(QTT_ERR_SHAPE, "stage graph: capacity mismatch");
  QTT_CUDA_CHECK(cudaMemcpyAsync(dst->data, src->data, src->off[src->n] * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
  QTT_CUDA_CHECK(cudaMemcpyAsync(dst->dims, src->dims, (src->n + 1) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, s));
}

void graph_release(StageGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  for (qtt_mps& m : G.in) {
    free_mps(m);
    m = nullptr;
  }
  for (qtt_mps& m : G.out) {
    free_mps(m);
    m = nullptr;
  }
}

void graphs_clear(qtt_ctx ctx) {
  if (ctx->graphs.empty() && ctx->step_graphs.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->graphs) graph_release(*kv.second);
  for (auto& kv : ctx->step_graphs) graph_release(*kv.second);
  ctx->graphs.clear();
  ctx->step_graphs.clear();
  ctx->graphs_captured = 0;
}

// Capture stage_w on graph-owned buffers shaped like this occurrence's
// inputs and outputs.  Any failure leaves the key marked `failed` (eager
// from then on) and the context as it was.
void capture_stage(qtt_ctx ctx, StageGraph& G, qtt_mps u[2], qtt_mps b[2], bool alias, double h,
                   double nu, double a_scale, MpsPtr w_eager[2]) {
  const int n = u[0]->n;
  G.in[0] = new_mps(ctx, n, u[0]->cap);
  G.in[1] = new_mps(ctx, n, u[1]->cap);
  if (!alias) {
    G.in[2] = new_mps(ctx, n, b[0]->cap);
    G.in[3] = new_mps(ctx, n, b[1]->cap);
  }
  G.out[0] = new_mps(ctx, n, w_eager[0]->cap);
  G.out[1] = new_mps(ctx, n, w_eager[1]->cap);
  if (!ctx->gstream)
    QTT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
  // nothing is executed by the capture; the buffers exist before any replay
  // because replays are ordered after this point on the context stream
  const cudaStream_t orig = ctx->stream;
  const long long n0 = ctx->launches.n;
  cudaGraph_t graph = nullptr;
  QTT_CUDA_CHECK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->gstream;
  t_capturing = true;
  t_body_launches = 0;
  try {
    qtt_mps gu[2] = {G.in[0], G.in[1]};
    qtt_mps gb[2] = {alias ? G.in[0] : G.in[2], alias ? G.in[1] : G.in[3]};
    MpsPtr w[2];
    stage_w(ctx, gu, gb, h, nu, w, a_scale);
    for (int i = 0; i < 2; i++) copy_mps_d2d(G.out[i], w[i].get(), ctx->stream);
    t_capturing = false;
  } catch (...) {
    t_capturing = false;
    t_body_launches = 0;
    cudaStreamEndCapture(ctx->gstream, &graph);
    if (graph) cudaGraphDestroy(graph);
    ctx->stream = orig;
    ctx->launches.n = n0;
    (void)cudaGetLastError();
    graph_release(G);
    G.failed = true;
    return;
  }
  const cudaError_t ec = cudaStreamEndCapture(ctx->gstream, &graph);
  ctx->stream = orig;
  // kernels outside the loop bodies run once per replay; the bodies' count
  // their passes on the device
  G.launches = ctx->launches.n - n0 - t_body_launches;
  t_body_launches = 0;
  ctx->launches.n = n0;
  cudaError_t ei = ec;
  if (ec == cudaSuccess) ei = cudaGraphInstantiate(&G.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    (void)cudaGetLastError();
    G.exec = nullptr;
    graph_release(G);
    G.failed = true;
  }
}

void stage_w_run(qtt_ctx ctx, qtt_mps u[2], qtt_mps b[2], double h, double nu, MpsPtr w[2],
                 double a_scale) {
  if (!ctx->p.graphs || g_prof.on || ctx->p.learned_trunc != QTT_LEARNED_OFF || ctx->dev_loops) {
    stage_w(ctx, u, b, h, nu, w, a_scale);
    return;
  }
  const bool alias = b[0] == u[0] && b[1] == u[1];
  const std::string key = stage_key(u, b, alias, h, nu, a_scale);
  if (ctx->graphs.size() > 256) {  // keys seen but never captured (a varying h)
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();)
      it = it->second->exec ? std::next(it) : ctx->graphs.erase(it);
  }
  std::unique_ptr<StageGraph>& slot = ctx->graphs[key];
  if (!slot) slot.reset(new StageGraph);
  StageGraph& G = *slot;
  if (!G.exec) {
    stage_w(ctx, u, b, h, nu, w, a_scale);
    if (G.seen++ >= 1 && !G.failed && ctx->graphs_captured < qtt_ctx_s::kMaxGraphs) {
      capture_stage(ctx, G, u, b, alias, h, nu, a_scale, w);
      if (!G.failed) ctx->graphs_captured++;
    }
    return;
  }
  const int n = u[0]->n;
  copy_mps_d2d(G.in[0], u[0], ctx->stream);
  copy_mps_d2d(G.in[1], u[1], ctx->stream);
  if (!alias) {
    copy_mps_d2d(G.in[2], b[0], ctx->stream);
    copy_mps_d2d(G.in[3], b[1], ctx->stream);
  }
  QTT_CUDA_CHECK(cudaGraphLaunch(G.exec, ctx->stream));
  ctx->launches.n += G.launches;
  ctx->graph_replays++;
  for (int i = 0; i < 2; i++) {
    w[i] = MpsPtr(new_mps(ctx, n, G.out[i]->cap));
    copy_mps_d2d(w[i].get(), G.out[i], ctx->stream);
  }
}

// A new step's slots: the current table becomes the previous one, the new
// current table starts empty.
void learned_next_step(qtt_ctx ctx) {
  ctx->tab ^= 1;
  ctx->slot = 0;
  const size_t cells = (size_t)qtt_ctx_s::kSlots * qtt_ctx_s::kBonds;
  QTT_CUDA_CHECK(cudaMemsetAsync(ctx->d_valid[ctx->tab], 0, cells * sizeof(int), stream_of(ctx)));
  QTT_CUDA_CHECK(cudaMemsetAsync(ctx->d_rank[ctx->tab], 0, cells * sizeof(int), stream_of(ctx)));
}

// The four stages and the final sum (Eqs. U1-U4); the inputs are left
// alone.  *nc: a projection of the step reached its CG or sweep cap (host
// loops; device-driven loops report on the device).
void rk4_core(qtt_ctx ctx, qtt_mps u[2], double dt, double nu, MpsPtr out[2], int* nc) {
  static const double HS[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  static const double BC[4][2] = {{0, 0}, {3.0, 0.25}, {1.5, 0.625}, {3.0, 0.25}};
  MpsPtr U[4][2];
  *nc = 0;
  // the running sum ((U_1 + U_2) + U_3) + U_4 is built on workers 10 and 11
  // (no stage uses them) as soon as each U_s exists, beside the later
  // stages: the same sums in the same order, one of them left after the
  // last projection instead of three
  static const bool ser = getenv("QTT_SERIAL") != nullptr;
  const bool side = !ser && ctx->workers[qtt_ctx_s::kWorkers - 1] != nullptr;
  MpsPtr acc[2];
  // Declared after U and acc, so destroyed before them: on every exit,
  // including an exception from a later stage, the context stream waits for
  // the running-sum work on workers 10 and 11 before U and acc are freed
  // (stream-ordered) on it.
  struct SideJoin {
    qtt_ctx ctx;
    bool on;
    void join() {
      if (!on) return;
      on = false;
      for (int i = 0; i < 2; i++) {
        if (cudaEventRecord(ctx->join_ev[10 + i], ctx->workers[10 + i]) == cudaSuccess)
          cudaStreamWaitEvent(ctx->stream, ctx->join_ev[10 + i], 0);
      }
    }
    ~SideJoin() { join(); }
  } side_join{ctx, side};
  auto accumulate = [&](int st) {
    if (side) {
      QTT_CUDA_CHECK(cudaEventRecord(ctx->sum_ev, ctx->stream));
      for (int i = 0; i < 2; i++) QTT_CUDA_CHECK(cudaStreamWaitEvent(ctx->workers[10 + i], ctx->sum_ev, 0));
    }
    for (int i = 0; i < 2; i++) {
      ctx->cur = side ? ctx->workers[10 + i] : nullptr;
      try {
        const qtt_mps prev = st == 1 ? U[0][i].get() : acc[i].get();
        acc[i] = MpsPtr(add2(ctx, 1.0, prev, 1.0, U[st][i].get()));
      } catch (...) {
        ctx->cur = nullptr;
        throw;
      }
      ctx->cur = nullptr;
    }
  };
  for (int st = 0; st < 4; st++) {
    MpsPtr bown[2];
    qtt_mps b[2] = {u[0], u[1]};
    if (st > 0) {
      Workers wk(ctx);
      wk.fork();
      for (int i = 0; i < 2; i++) {
        bown[i] = MpsPtr(wk.run(i, [&] { return add2(ctx, BC[st][0], U[st - 1][i].get(), BC[st][1], u[i]); }));
        b[i] = bown[i].get();
      }
      wk.join({b[0], b[1]});
    }
    const double h = HS[st] * dt;
    qtt_mps v1, v2;
    int cg = 0, sw = 0;
    if (ctx->p.rhs_form == QTT_RHS_IMPLICIT) {
      project_implicit_impl(ctx, u, b, h, nu, 0.25, &v1, &v2, &cg, &sw);
    } else {
      MpsPtr w[2];
      stage_w_run(ctx, u, b, h, nu, w, 0.25);
      project_stage(ctx, w[0].get(), w[1].get(), h, &v1, &v2, &cg, &sw);
    }
    *nc |= ctx->last_not_converged;
    U[st][0] = MpsPtr(v1);
    U[st][1] = MpsPtr(v2);
    if (st >= 1) accumulate(st);
  }
  side_join.join();
  QTT_CUDA_CHECK(cudaGetLastError());
  for (int i = 0; i < 2; i++) {
    acc[i]->stream = ctx->stream;
    out[i] = std::move(acc[i]);
  }
}

// Whole-step graph (params.graphs = 2): stages as in stage graphs, the
// projection's loops as WHILE nodes (capture_while), inputs and outputs
// through graph-owned buffers; key = the capacities of u_1, u_2 and dt, nu.
void capture_step(qtt_ctx ctx, StageGraph& G, qtt_mps u[2], double dt, double nu,
                  MpsPtr out_eager[2]) {
  const int n = u[0]->n;
  if (!ctx->d_stats) {
    QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_stats, 4 * sizeof(long long)));
    QTT_CUDA_CHECK(cudaMemset(ctx->d_stats, 0, 4 * sizeof(long long)));
    reg_alloc(ctx->d_stats, 4 * sizeof(long long));
    QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_loop, 4 * sizeof(int)));
    QTT_CUDA_CHECK(cudaMemset(ctx->d_loop, 0, 4 * sizeof(int)));
    reg_alloc(ctx->d_loop, 4 * sizeof(int));
  }
  for (int k = 0; k < 2; k++) {
    if (!ctx->bstream[k])
      QTT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->bstream[k], cudaStreamNonBlocking));
    for (int i = 0; i < 4; i++)
      if (!ctx->bworkers[k][i])
        QTT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->bworkers[k][i], cudaStreamNonBlocking));
  }
  if (!ctx->gstream)
    QTT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
  G.in[0] = new_mps(ctx, n, u[0]->cap);
  G.in[1] = new_mps(ctx, n, u[1]->cap);
  G.out[0] = new_mps(ctx, n, out_eager[0]->cap);
  G.out[1] = new_mps(ctx, n, out_eager[1]->cap);
  const cudaStream_t orig = ctx->stream;
  const long long n0 = ctx->launches.n;
  cudaGraph_t graph = nullptr;
  QTT_CUDA_CHECK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
  ctx->stream = ctx->gstream;
  ctx->dev_loops = true;
  t_capturing = true;
  t_body_launches = 0;
  try {
    qtt_mps gu[2] = {G.in[0], G.in[1]};
    MpsPtr o[2];
    int nc = 0;
    rk4_core(ctx, gu, dt, nu, o, &nc);
    for (int i = 0; i < 2; i++) copy_mps_d2d(G.out[i], o[i].get(), ctx->stream);
    t_capturing = false;
    ctx->dev_loops = false;
  } catch (...) {
    t_capturing = false;
    ctx->dev_loops = false;
    t_body_launches = 0;
    cudaStreamEndCapture(ctx->gstream, &graph);
    if (graph) cudaGraphDestroy(graph);
    ctx->stream = orig;
    ctx->launches.n = n0;
    (void)cudaGetLastError();
    graph_release(G);
    G.failed = true;
    return;
  }
  const cudaError_t ec = cudaStreamEndCapture(ctx->gstream, &graph);
  ctx->stream = orig;
  // kernels outside the loop bodies run once per replay; the bodies count
  // their passes on the device
  G.launches = ctx->launches.n - n0 - t_body_launches;
  t_body_launches = 0;
  ctx->launches.n = n0;
  cudaError_t ei = ec;
  if (ec == cudaSuccess) ei = cudaGraphInstantiate(&G.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    (void)cudaGetLastError();
    G.exec = nullptr;
    graph_release(G);
    G.failed = true;
  }
}

void rk4_impl(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (ctx->p.learned_trunc != QTT_LEARNED_OFF) learned_next_step(ctx);
  qtt_mps u[2] = {*u1, *u2};
  MpsPtr out[2];
  const bool step_graphs = ctx->p.graphs == 2 && !g_prof.on && ctx->p.learned_trunc == QTT_LEARNED_OFF;
  StageGraph* G = nullptr;
  if (step_graphs) {
    std::string key;
    auto put = [&](const void* p, size_t k) { key.append((const char*)p, k); };
    put(&dt, sizeof dt);
    put(&nu, sizeof nu);
    for (int i = 0; i < 2; i++) put(u[i]->cap.data(), u[i]->cap.size() * sizeof(int));
    if (ctx->step_graphs.size() > 64) {
      for (auto it = ctx->step_graphs.begin(); it != ctx->step_graphs.end();)
        it = it->second->exec ? std::next(it) : ctx->step_graphs.erase(it);
    }
    std::unique_ptr<StageGraph>& slot = ctx->step_graphs[key];
    if (!slot) slot.reset(new StageGraph);
    G = slot.get();
  }
  if (G && G->exec) {
    const int n = u[0]->n;
    copy_mps_d2d(G->in[0], u[0], ctx->stream);
    copy_mps_d2d(G->in[1], u[1], ctx->stream);
    QTT_CUDA_CHECK(cudaGraphLaunch(G->exec, ctx->stream));
    ctx->launches.n += G->launches;
    ctx->graph_replays++;
    ctx->stats_pending = true;
    for (int i = 0; i < 2; i++) {
      out[i] = MpsPtr(new_mps(ctx, n, G->out[i]->cap));
      copy_mps_d2d(out[i].get(), G->out[i], ctx->stream);
    }
    ctx->last_not_converged = 0;  // the device flag is read at the next sync
  } else {
    int nc = 0;
    rk4_core(ctx, u, dt, nu, out, &nc);
    if (G && G->seen++ >= 1 && !G->failed && ctx->graphs_captured < qtt_ctx_s::kMaxGraphs) {
      capture_step(ctx, *G, u, dt, nu, out);
      if (!G->failed) ctx->graphs_captured++;
    }
    ctx->last_not_converged = nc;
  }
  free_mps(*u1);
  free_mps(*u2);
  *u1 = out[0].release();
  *u2 = out[1].release();
}

// One penalised minimisation with a = u (scale 1) and the given b, h.
void euler_min(qtt_ctx ctx, qtt_mps u[2], qtt_mps b[2], double h, double nu, MpsPtr v[2]) {
  qtt_mps v1, v2;
  int cg = 0, sw = 0;
  if (ctx->p.rhs_form == QTT_RHS_IMPLICIT) {
    project_implicit_impl(ctx, u, b, h, nu, 1.0, &v1, &v2, &cg, &sw);
  } else {
    MpsPtr w[2];
    stage_w_run(ctx, u, b, h, nu, w, 1.0);
    project_stage(ctx, w[0].get(), w[1].get(), h, &v1, &v2, &cg, &sw);
  }
  v[0] = MpsPtr(v1);
  v[1] = MpsPtr(v2);
}

// Explicit Euler (App. B, Eq. "euler"): u^{s+1} = argmin Theta(v, u, u, dt).
void euler_impl(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (ctx->p.learned_trunc != QTT_LEARNED_OFF) learned_next_step(ctx);
  qtt_mps u[2] = {*u1, *u2};
  MpsPtr v[2];
  euler_min(ctx, u, u, dt, nu, v);
  const int nc = ctx->last_not_converged;
  free_mps(*u1);
  free_mps(*u2);
  *u1 = v[0].release();
  *u2 = v[1].release();
  ctx->last_not_converged = nc;
}

// Midpoint RK2 (App. B, Eqs. "midpoint_calc", "full_calc").
void rk2_impl(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (ctx->p.learned_trunc != QTT_LEARNED_OFF) learned_next_step(ctx);
  qtt_mps u[2] = {*u1, *u2};
  MpsPtr um[2], v[2];
  euler_min(ctx, u, u, 0.5 * dt, nu, um);
  int nc = ctx->last_not_converged;
  qtt_mps b[2] = {um[0].get(), um[1].get()};
  euler_min(ctx, u, b, dt, nu, v);
  nc |= ctx->last_not_converged;
  free_mps(*u1);
  free_mps(*u2);
  *u1 = v[0].release();
  *u2 = v[1].release();
  ctx->last_not_converged = nc;
}

// <a|b> by the left transfer matrices E_k = sum_s A_k[s]^T E_{k-1} B_k[s]
// (capacity shapes; the zero padding contributes nothing); the 1 x 1 E_n is
// copied to the host (synchronises).
double inner_impl(qtt_ctx ctx, qtt_mps A, qtt_mps B) {
  const int n = A->n;
  cudaStream_t s = stream_of(ctx);
  size_t emax = 1, tmax = 1;
  for (int k = 0; k <= n; k++) emax = std::max(emax, (size_t)A->cap[k] * B->cap[k]);
  for (int k = 0; k < n; k++) tmax = std::max(tmax, (size_t)A->cap[k] * 4 * B->cap[k + 1]);
  DBuf<double> E0(emax, s), E1(emax, s), Tb(tmax, s);
  launch_fill(E0.p, 1, 1.0, s);
  double* Ec = E0.p;
  double* En = E1.p;
  for (int k = 0; k < n; k++) {
    const int al = A->cap[k], ar = A->cap[k + 1], bl = B->cap[k], br = B->cap[k + 1];
    // T ((al x 4) x br) = E (al x bl) * B_k (bl x 4 br)
    gemm(gemm_plain(Ec, B->core(k), Tb.p, al, 4 * br, bl, bl, 4 * br, 4 * br), s);
    // E' (ar x br) = A_k^T ((al 4) x ar)^T * T ((al 4) x br)
    GemmF64 g = gemm_plain(A->core(k), Tb.p, En, ar, br, 4 * al, ar, br, br);
    g.tA = 1;
    gemm(g, s);
    std::swap(Ec, En);
  }
  double h = 0.0;
  QTT_CUDA_CHECK(cudaMemcpyAsync(&h, Ec, sizeof(double), cudaMemcpyDeviceToHost, s));
  QTT_CUDA_CHECK(cudaStreamSynchronize(s));
  return h;
}

// ---------------------------------------------------------------- dense I/O
qtt_mps from_dense_impl(qtt_ctx ctx, const double* F, double eps, int chi) {
  const int n = ctx->p.n;
  cudaStream_t s = stream_of(ctx);
  std::vector<int> ocap(n + 1, 1);
  for (int b = 1; b < n; b++) ocap[b] = std::min(chi, clampi(natural_cap(n, b)));
  MpsPtr Y(new_mps(ctx, n, ocap));
  launch_fill_int(Y->dims, n + 1, 1, s);
  const size_t tot = (size_t)1 << (2 * n);
  DBuf<double> T(tot, s);
  launch_check_finite(F, tot, ctx->d_err, s);
  launch_dense_to_omega(F, T.p, n, s);
  if (n == 1) {
    launch_copy(Y->core(0), T.p, 4, s);
    return Y.release();
  }
  // right-to-left TT-SVD: carry C (4^k x ocap[k]) -> reshape (4^(k-1) x 4 ocap[k])
  size_t cmax = 1, svw = 1;
  for (int k = 1; k < n; k++) {
    const size_t rows = (size_t)1 << (2 * k);  // 4^k
    cmax = std::max(cmax, rows * ocap[k]);
    svw = std::max(svw, svd_work_doubles(clampi(1LL << (2 * k)), 4 * ocap[k + 1]));
  }
  DBuf<double> C0(cmax, s), C1(cmax, s), W(svw, s);
  const double* Mp = T.p;
  double* Cn = C0.p;
  double* Co = C1.p;
  for (int k = n - 1; k >= 1; k--) {
    const int rows = clampi(1LL << (2 * k));  // 4^k rows (sites 0..k-1)
    SvdArgs a{};
    a.M = MatView{const_cast<double*>(Mp), 4 * ocap[k + 1], axis_prefix(rows, dconst(rows)),
                  axis_pair(4, dconst(4), ocap[k + 1], dref(Y->dims + k + 1))};
    a.US = MatView{Cn, ocap[k], axis_prefix(rows, dconst(rows)), axis_prefix(ocap[k], dconst(1))};
    a.VT = MatView{Y->core(k), 4 * ocap[k + 1], axis_prefix(ocap[k], dconst(1)),
                   axis_pair(4, dconst(4), ocap[k + 1], dref(Y->dims + k + 1))};
    a.eps = eps;
    a.chi = chi;
    a.rank_limit = dconst(1 << 30);
    a.r_out = Y->dims + k;
    a.work = W.p;
    a.work_len = (long long)W.n;
    a.err = ctx->d_err;
    launch_svd_f64(a, rows, 4 * ocap[k + 1], s);
    Mp = Cn;
    std::swap(Cn, Co);
  }
  launch_copy(Y->core(0), Mp, (size_t)4 * ocap[1], s);
  return Y.release();
}

void to_dense_impl(qtt_ctx ctx, qtt_mps A, double* F) {
  const int n = A->n;
  cudaStream_t s = stream_of(ctx);
  const size_t tot = (size_t)1 << (2 * n);
  size_t mx = 4 * (size_t)A->cap[1];
  for (int k = 1; k < n; k++) mx = std::max(mx, ((size_t)1 << (2 * (k + 1))) * A->cap[k + 1]);
  DBuf<double> L0(std::max(mx, tot), s), L1(std::max(mx, tot), s);
  launch_copy(L0.p, A->core(0), (size_t)4 * A->cap[1], s);
  double* cur = L0.p;
  double* nxt = L1.p;
  for (int k = 1; k < n; k++) {
    const int rows = clampi(1LL << (2 * k));
    gemm(gemm_plain(cur, A->core(k), nxt, rows, 4 * A->cap[k + 1], A->cap[k], A->cap[k],
                    4 * A->cap[k + 1], 4 * A->cap[k + 1]), s);
    std::swap(cur, nxt);
  }
  launch_omega_to_dense(cur, F, n, s);
}

// --------------------------------------------------------------- errors
qtt_status check_device_errors(qtt_ctx ctx) {
  int h = 0;
  long long st[4] = {0, 0, 0, 0};
  QTT_CUDA_CHECK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  const bool pending = ctx->stats_pending && ctx->d_stats;
  if (pending)
    QTT_CUDA_CHECK(cudaMemcpyAsync(st, ctx->d_stats, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  if (pending) {
    // counters of replayed steps whose projection loops ran on the device
    ctx->cg_iters += st[0];
    ctx->sweeps += st[1];
    ctx->launches.n += st[3];
    if (st[2]) ctx->last_not_converged = 1;
    QTT_CUDA_CHECK(cudaMemsetAsync(ctx->d_stats, 0, sizeof st, ctx->stream));
    ctx->stats_pending = false;
  }
  if (h) {
    QTT_CUDA_CHECK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    if (h & QTT_DEVERR_NUMERIC) {
      ctx->err = "non-finite value met on the device";
      return QTT_ERR_NUMERIC;
    }
    if (h & QTT_DEVERR_TIMEOUT) {
      ctx->err = "a bounded device-side wait gave up";
      return QTT_ERR_TIMEOUT;
    }
    ctx->err = "device-side shape error";
    return QTT_ERR_SHAPE;
  }
  return QTT_OK;
}

template <typename F>
qtt_status guarded(qtt_ctx ctx, F&& f) {
  if (!ctx) return QTT_ERR_ARG;
  CtxGuard g(ctx);
  try {
    return f();
  } catch (const QttError& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (const CudaError& e) {
    char buf[256];
    snprintf(buf, sizeof buf, "CUDA error %s at line %d: %s", cudaGetErrorString(e.e), e.line,
             e.what);
    ctx->err = buf;
    return QTT_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return QTT_ERR_ALLOC;
  }
}

bool valid_params(const qtt_params* p) {
  return p && p->n >= 1 && p->n <= 15 && p->L > 0 && p->eps >= 0 && p->chi_max >= 1 &&
         p->mu >= 0 && p->cg_tol >= 0 && p->cg_maxit >= 1 && p->sweep_tol >= 0 &&
         p->max_sweeps >= 1 && (p->precision == QTT_PREC_FP64 || p->precision == QTT_PREC_MIXED) &&
         p->learned_trunc >= QTT_LEARNED_OFF && p->learned_trunc <= QTT_LEARNED_ON &&
         (p->learned_trunc != QTT_LEARNED_LOG || p->precision == QTT_PREC_FP64) &&
         p->rf_oversample >= 0 && p->rf_oversample <= 256 && p->rf_min_width >= 1 &&
         p->graphs >= 0 && p->graphs <= 2 &&
         (p->fd_order == 0 || p->fd_order == 2 || p->fd_order == 4 || p->fd_order == 6 ||
          p->fd_order == 8) &&
         (p->rhs_form == QTT_RHS_EXPLICIT || p->rhs_form == QTT_RHS_IMPLICIT) &&
         (p->projection == QTT_PROJ_PENALTY ||
          (p->projection == QTT_PROJ_SPECTRAL && p->rhs_form == QTT_RHS_EXPLICIT && p->n <= 13));
}

void check_mps(qtt_ctx ctx, qtt_mps m) {
  if (!m) throw QttError(QTT_ERR_ARG, "null MPS");
  if (m->n != ctx->p.n) throw QttError(QTT_ERR_SHAPE, "MPS has a different n than the context");
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

qtt_status qtt_create(qtt_ctx* out, int device, void* stream, const qtt_params* params) {
  if (!out || !valid_params(params)) return QTT_ERR_ARG;
  *out = nullptr;
  auto ctx = new qtt_ctx_s;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->p = *params;
  ctx->dx = params->L / (double)(1 << params->n);
  qtt_status st = guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaSetDevice(device));
    cudaMemPool_t pool;
    QTT_CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    QTT_CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_err, sizeof(int)));
    for (int k = 0; k < qtt_ctx_s::kWorkers; k++) {
      QTT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->workers[k], cudaStreamNonBlocking));
      QTT_CUDA_CHECK(cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming));
    }
    QTT_CUDA_CHECK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
    QTT_CUDA_CHECK(cudaEventCreateWithFlags(&ctx->sum_ev, cudaEventDisableTiming));
    for (int e = 0; e < qtt_ctx_s::kFlowEvents; e++)
      QTT_CUDA_CHECK(cudaEventCreateWithFlags(&ctx->flow_ev[e], cudaEventDisableTiming));
    QTT_CUDA_CHECK(cudaMemset(ctx->d_err, 0, sizeof(int)));
    noalloc_prepare_current_device();
    {
      const size_t cells = (size_t)qtt_ctx_s::kSlots * qtt_ctx_s::kBonds;
      for (int t = 0; t < 2; t++) {
        QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_feat[t], cells * QTT_MLP_FEATURES * sizeof(float)));
        QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_rank[t], cells * sizeof(int)));
        QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_valid[t], cells * sizeof(int)));
        QTT_CUDA_CHECK(cudaMemset(ctx->d_rank[t], 0, cells * sizeof(int)));
        QTT_CUDA_CHECK(cudaMemset(ctx->d_valid[t], 0, cells * sizeof(int)));
        reg_alloc(ctx->d_feat[t], cells * QTT_MLP_FEATURES * sizeof(float));
        reg_alloc(ctx->d_rank[t], cells * sizeof(int));
        reg_alloc(ctx->d_valid[t], cells * sizeof(int));
      }
      QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_mlp, QTT_MLP_PARAMS * sizeof(float)));
      QTT_CUDA_CHECK(cudaMemset(ctx->d_mlp, 0, QTT_MLP_PARAMS * sizeof(float)));
      reg_alloc(ctx->d_mlp, QTT_MLP_PARAMS * sizeof(float));
      QTT_CUDA_CHECK(cudaMalloc((void**)&ctx->d_rf_counts, 4 * sizeof(long long)));
      QTT_CUDA_CHECK(cudaMemset(ctx->d_rf_counts, 0, 4 * sizeof(long long)));
      reg_alloc(ctx->d_rf_counts, 4 * sizeof(long long));
    }
    const int n = params->n;
    const double dx = ctx->dx;
    const int order = params->fd_order == 0 ? 2 : params->fd_order;
    if (order == 2) {
      // the paper's operators: D from App. A's carry table
      HostMpo D1 = diff_mpo(n, 1, dx), D2 = diff_mpo(n, 2, dx);
      ctx->D[0] = upload_mpo(ctx, D1);
      ctx->D[1] = upload_mpo(ctx, D2);
      // Laplacian D1 D1 + D2 D2 = (S1^{+2} + S1^{-2} + S2^{+2} + S2^{-2} - 4) / (4 dx^2)
      const double c2 = 1.0 / (4.0 * dx * dx);
      ctx->lap = upload_mpo(ctx, shift_sum_mpo(n, -4.0 * c2, {1, 1, 2, 2}, {2, -2, 2, -2},
                                               {c2, c2, c2, c2}));
      // projection blocks D_i^T D_j = -D_i D_j
      HostMpo Ds[2] = {D1, D2};
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
          if (i == j) {
            ctx->K[i][j] = upload_mpo(ctx, shift_sum_mpo(n, 2.0 * c2, {i + 1, i + 1}, {2, -2},
                                                         {-c2, -c2}));
          } else {
            ctx->K[i][j] = upload_mpo(ctx, mpo_scaled(mpo_mul(Ds[i], Ds[j]), -1.0));
          }
        }
    } else {
      // higher even orders (Sec. II.B): the same operators from central
      // differences of that order, built as translation machines
      HostMpo Ds[2] = {fd_mpo(n, 1, 1, order, dx), fd_mpo(n, 2, 1, order, dx)};
      ctx->D[0] = upload_mpo(ctx, Ds[0]);
      ctx->D[1] = upload_mpo(ctx, Ds[1]);
      ctx->lap = upload_mpo(ctx, fd_laplacian(n, order, dx));
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
          ctx->K[i][j] = upload_mpo(
              ctx, i == j ? mpo_scaled(fd_mpo(n, i + 1, 2, order, dx), -1.0)
                          : mpo_scaled(mpo_mul(Ds[i], Ds[j]), -1.0));
    }
    return QTT_OK;
  });
  if (st != QTT_OK) {
    qtt_destroy(ctx);
    return st;
  }
  *out = ctx;
  return QTT_OK;
}

qtt_status qtt_destroy(qtt_ctx ctx) {
  if (!ctx) return QTT_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  graphs_clear(ctx);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  for (cudaStream_t b : ctx->bstream)
    if (b) cudaStreamDestroy(b);
  for (auto& pr : ctx->bworkers)
    for (cudaStream_t b : pr)
      if (b) cudaStreamDestroy(b);
  for (void* q : {(void*)ctx->d_stats, (void*)ctx->d_loop})
    if (q) {
      reg_free(q);
      cudaFree(q);
    }
  for (int i = 0; i < 2; i++) mpo_release(ctx->D[i]);
  mpo_release(ctx->lap);
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) mpo_release(ctx->K[i][j]);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (int t = 0; t < 2; t++) {
    for (void* q : {(void*)ctx->d_feat[t], (void*)ctx->d_rank[t], (void*)ctx->d_valid[t]})
      if (q) {
        reg_free(q);
        cudaFree(q);
      }
  }
  for (void* q : {(void*)ctx->d_mlp, (void*)ctx->d_rf_counts})
    if (q) {
      reg_free(q);
      cudaFree(q);
    }
  for (int k = 0; k < qtt_ctx_s::kWorkers; k++) {
    if (ctx->workers[k]) cudaStreamDestroy(ctx->workers[k]);
    if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->sum_ev) cudaEventDestroy(ctx->sum_ev);
  for (int e = 0; e < qtt_ctx_s::kFlowEvents; e++)
    if (ctx->flow_ev[e]) cudaEventDestroy(ctx->flow_ev[e]);
  delete ctx;
  return QTT_OK;
}

qtt_status qtt_set_params(qtt_ctx ctx, const qtt_params* p) {
  if (!ctx || !valid_params(p) || p->n != ctx->p.n || p->L != ctx->p.L ||
      (p->fd_order == 0 ? 2 : p->fd_order) != (ctx->p.fd_order == 0 ? 2 : ctx->p.fd_order))
    return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    graphs_clear(ctx);  // captured with the previous eps / chi / precision
    ctx->p = *p;
    return QTT_OK;
  });
}

qtt_status qtt_sync(qtt_ctx ctx) {
  return guarded(ctx, [&]() -> qtt_status { return check_device_errors(ctx); });
}

const char* qtt_last_error(qtt_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

qtt_status qtt_from_dense(qtt_ctx ctx, const double* d_field, double eps, int chi_max,
                          qtt_mps* out) {
  if (!out || !d_field || eps < 0 || chi_max < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    *out = from_dense_impl(ctx, d_field, eps, chi_max);
    return QTT_OK;
  });
}

qtt_status qtt_to_dense(qtt_ctx ctx, qtt_mps mps, double* d_field_out) {
  if (!d_field_out) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, mps);
    to_dense_impl(ctx, mps, d_field_out);
    return check_device_errors(ctx);
  });
}

qtt_status qtt_mps_from_packed(qtt_ctx ctx, const double* cores, int cores_are_device,
                               const int* bonds, qtt_mps* out) {
  if (!out || !cores || !bonds) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    const int n = ctx->p.n;
    std::vector<int> cap(bonds, bonds + n + 1);
    if (cap[0] != 1 || cap[n] != 1) throw QttError(QTT_ERR_SHAPE, "end bonds must be 1");
    for (int b = 1; b < n; b++)
      if (cap[b] < 1 || cap[b] > (1 << 20)) throw QttError(QTT_ERR_SHAPE, "bad bond dimension");
    MpsPtr m(new_mps(ctx, n, cap));
    const cudaMemcpyKind kind = cores_are_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    QTT_CUDA_CHECK(cudaMemcpyAsync(m->data, cores, m->off[n] * sizeof(double), kind, ctx->stream));
    QTT_CUDA_CHECK(cudaMemcpyAsync(m->dims, cap.data(), (n + 1) * sizeof(int),
                                   cudaMemcpyHostToDevice, ctx->stream));
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    *out = m.release();
    return QTT_OK;
  });
}

qtt_status qtt_mps_upload_packed(qtt_ctx ctx, qtt_mps dst, const double* cores,
                                 int cores_are_device, const int* bonds) {
  if (!dst || !cores || !bonds) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, dst);
    const int n = dst->n;
    std::vector<int> d(bonds, bonds + n + 1);
    if (d[0] != 1 || d[n] != 1) throw QttError(QTT_ERR_SHAPE, "end bonds must be 1");
    for (int b = 1; b < n; b++)
      if (d[b] < 1 || d[b] > dst->cap[b])
        throw QttError(QTT_ERR_SHAPE, "bond dimension above the MPS's capacity");
    cudaStream_t s = ctx->stream;
    // capacity storage: rows (a, s) of length cap[k+1], the actual block in
    // the leading rows and columns, zero elsewhere
    QTT_CUDA_CHECK(cudaMemsetAsync(dst->data, 0, dst->off[n] * sizeof(double), s));
    const cudaMemcpyKind kind = cores_are_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t o = 0;
    for (int k = 0; k < n; k++) {
      QTT_CUDA_CHECK(cudaMemcpy2DAsync(dst->core(k), dst->cap[k + 1] * sizeof(double), cores + o,
                                       d[k + 1] * sizeof(double), d[k + 1] * sizeof(double),
                                       (size_t)d[k] * 4, kind, s));
      o += (size_t)d[k] * 4 * d[k + 1];
    }
    QTT_CUDA_CHECK(cudaMemcpyAsync(dst->dims, d.data(), (n + 1) * sizeof(int),
                                   cudaMemcpyHostToDevice, s));
    QTT_CUDA_CHECK(cudaStreamSynchronize(s));
    return QTT_OK;
  });
}

qtt_status qtt_mps_to_packed(qtt_ctx ctx, qtt_mps mps, double* cores, int cores_are_device,
                             size_t capacity, int* bonds) {
  if (!cores || !bonds) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, mps);
    const int n = mps->n;
    std::vector<int> d(n + 1);
    QTT_CUDA_CHECK(cudaMemcpyAsync(d.data(), mps->dims, (n + 1) * sizeof(int),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    size_t need = 0;
    for (int k = 0; k < n; k++) need += (size_t)d[k] * 4 * d[k + 1];
    if (need > capacity) throw QttError(QTT_ERR_ARG, "output capacity too small");
    // pack: rows (a, s) of length d[k+1] from capacity storage
    size_t o = 0;
    const cudaMemcpyKind kind = cores_are_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < n; k++) {
      QTT_CUDA_CHECK(cudaMemcpy2DAsync(cores + o, d[k + 1] * sizeof(double), mps->core(k),
                                       mps->cap[k + 1] * sizeof(double), d[k + 1] * sizeof(double),
                                       (size_t)d[k] * 4, kind, ctx->stream));
      o += (size_t)d[k] * 4 * d[k + 1];
    }
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b <= n; b++) bonds[b] = d[b];
    return check_device_errors(ctx);
  });
}

qtt_status qtt_mps_info(qtt_mps mps, int* n, int* bonds) {
  if (!mps) return QTT_ERR_ARG;
  qtt_ctx ctx = mps->ctx;
  return guarded(ctx, [&]() -> qtt_status {
    std::vector<int> d(mps->n + 1);
    QTT_CUDA_CHECK(cudaMemcpyAsync(d.data(), mps->dims, (mps->n + 1) * sizeof(int),
                                   cudaMemcpyDeviceToHost, mps->stream));
    QTT_CUDA_CHECK(cudaStreamSynchronize(mps->stream));
    if (n) *n = mps->n;
    if (bonds)
      for (int b = 0; b <= mps->n; b++) bonds[b] = d[b];
    return check_device_errors(ctx);
  });
}

void qtt_free_mps(qtt_mps mps) {
  if (!mps) return;
  cudaSetDevice(mps->ctx->device);
  free_mps(mps);
}

qtt_status qtt_mpo_get(qtt_ctx ctx, int which, qtt_mpo* out) {
  if (!ctx || !out) return QTT_ERR_ARG;
  qtt_mpo m = nullptr;
  if (which == 1) m = ctx->D[0];
  else if (which == 2) m = ctx->D[1];
  else if (which == 3) m = ctx->lap;
  else if (which >= 4 && which <= 7) m = ctx->K[(which - 4) >> 1][(which - 4) & 1];
  if (!m) return QTT_ERR_ARG;
  m->refs++;
  *out = m;
  return QTT_OK;
}

void qtt_free_mpo(qtt_mpo mpo) { mpo_release(mpo); }

qtt_status qtt_apply_mpo(qtt_ctx ctx, qtt_mpo mpo, qtt_mps in, double eps, int chi_max,
                         qtt_mps* out) {
  if (!mpo || !out || eps < 0 || chi_max < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, in);
    if (mpo->n != in->n) throw QttError(QTT_ERR_SHAPE, "MPO and MPS sizes differ");
    *out = apply_impl(ctx, mpo, in, eps, chi_max);
    return QTT_OK;
  });
}

qtt_status qtt_add(qtt_ctx ctx, int k, const double* coef, const qtt_mps* terms, double eps,
                   int chi_max, qtt_mps* out) {
  if (!out || !coef || !terms || k < 1 || k > 8 || eps < 0 || chi_max < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    for (int t = 0; t < k; t++) check_mps(ctx, terms[t]);
    *out = add_impl(ctx, k, coef, terms, eps, chi_max);
    return QTT_OK;
  });
}

qtt_status qtt_hadamard(qtt_ctx ctx, qtt_mps a, qtt_mps b, double eps, int chi_max, qtt_mps* out) {
  if (!out || eps < 0 || chi_max < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, a);
    check_mps(ctx, b);
    *out = hadamard_impl(ctx, a, b, eps, chi_max);
    return QTT_OK;
  });
}

qtt_status qtt_compress(qtt_ctx ctx, qtt_mps inout, double eps, int chi_max) {
  if (eps < 0 || chi_max < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, inout);
    qtt_mps y = compress_impl(ctx, inout, eps, chi_max);
    // swap contents so the caller's handle now holds the result
    std::swap(inout->cap, y->cap);
    std::swap(inout->off, y->off);
    std::swap(inout->data, y->data);
    std::swap(inout->dims, y->dims);
    free_mps(y);
    return QTT_OK;
  });
}

qtt_status qtt_project(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, double h, double mu, qtt_mps* v1,
                       qtt_mps* v2, int* cg_iters, int* sweeps) {
  if (!v1 || !v2 || !(h > 0) || !(mu >= 0)) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, w1);
    check_mps(ctx, w2);
    project_impl(ctx, w1, w2, h, mu, v1, v2, cg_iters, sweeps);
    qtt_status st = check_device_errors(ctx);
    if (st != QTT_OK) return st;
    if (ctx->last_not_converged) {
      ctx->err = "projection reached its CG or sweep cap";
      return QTT_ERR_NOT_CONVERGED;
    }
    return QTT_OK;
  });
}

qtt_status qtt_project_spectral(qtt_ctx ctx, qtt_mps w1, qtt_mps w2, qtt_mps* v1, qtt_mps* v2) {
  if (!ctx || !v1 || !v2) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, w1);
    check_mps(ctx, w2);
    project_spectral_impl(ctx, w1, w2, v1, v2);
    return QTT_OK;
  });
}

qtt_status qtt_rk4_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (!u1 || !u2 || !(dt > 0) || nu < 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, *u1);
    check_mps(ctx, *u2);
    rk4_impl(ctx, u1, u2, dt, nu);
    qtt_status st = check_device_errors(ctx);
    if (st != QTT_OK) return st;
    if (ctx->last_not_converged) {
      ctx->err = "a projection reached its CG or sweep cap";
      return QTT_ERR_NOT_CONVERGED;
    }
    return QTT_OK;
  });
}

qtt_status qtt_euler_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (!u1 || !u2 || !(dt > 0) || nu < 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, *u1);
    check_mps(ctx, *u2);
    euler_impl(ctx, u1, u2, dt, nu);
    qtt_status st = check_device_errors(ctx);
    if (st != QTT_OK) return st;
    if (ctx->last_not_converged) {
      ctx->err = "a projection reached its CG or sweep cap";
      return QTT_ERR_NOT_CONVERGED;
    }
    return QTT_OK;
  });
}

qtt_status qtt_rk2_step(qtt_ctx ctx, qtt_mps* u1, qtt_mps* u2, double dt, double nu) {
  if (!u1 || !u2 || !(dt > 0) || nu < 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, *u1);
    check_mps(ctx, *u2);
    rk2_impl(ctx, u1, u2, dt, nu);
    qtt_status st = check_device_errors(ctx);
    if (st != QTT_OK) return st;
    if (ctx->last_not_converged) {
      ctx->err = "a projection reached its CG or sweep cap";
      return QTT_ERR_NOT_CONVERGED;
    }
    return QTT_OK;
  });
}

qtt_status qtt_inner(qtt_ctx ctx, qtt_mps a, qtt_mps b, double* out) {
  if (!out) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, a);
    check_mps(ctx, b);
    *out = inner_impl(ctx, a, b);
    return check_device_errors(ctx);
  });
}

qtt_status qtt_tke_spectrum(qtt_ctx ctx, qtt_mps u1, qtt_mps u2, int kmax, double* h_E) {
  if (!ctx || !h_E || kmax < 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    check_mps(ctx, u1);
    check_mps(ctx, u2);
    const int n = u1->n;
    if (u2->n != n) throw QttError(QTT_ERR_SHAPE, "components on different grids");
    if (n > 12) throw QttError(QTT_ERR_SHAPE, "spectrum: n > 12");
    cudaStream_t s = stream_of(ctx);
    const size_t NN = (size_t)1 << (2 * n);
    DBuf<double> F1(NN, s), F2(NN, s), P(NN, s), E(kmax + 1, s);
    DBuf<double2> C1(NN, s), C2(NN, s);
    to_dense_impl(ctx, u1, F1.p);
    to_dense_impl(ctx, u2, F2.p);
    launch_tke_spectrum(F1.p, F2.p, n, C1.p, C2.p, P.p, E.p, kmax, s);
    QTT_CUDA_CHECK(cudaMemcpyAsync(h_E, E.p, (kmax + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA_CHECK(cudaStreamSynchronize(s));
    return check_device_errors(ctx);
  });
}

qtt_status qtt_mpo_diff(qtt_ctx ctx, int axis, int power, double dx, qtt_mpo* out) {
  if (!ctx || !out || (axis != 1 && axis != 2) || (power != 1 && power != 2) || !(dx > 0.0))
    return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    cudaSetDevice(ctx->device);
    const int n = ctx->p.n;
    const int order = ctx->p.fd_order == 0 ? 2 : ctx->p.fd_order;
    HostMpo m;
    if (order == 2 && power == 1) {
      m = diff_mpo(n, axis, dx);  // App. A's carry table
    } else if (order == 2) {
      const double c2 = 1.0 / (4.0 * dx * dx);  // (S^2 - 2 + S^-2) / (4 dx^2)
      m = shift_sum_mpo(n, -2.0 * c2, {axis, axis}, {2, -2}, {c2, c2});
    } else {
      m = fd_mpo(n, axis, power, order, dx);
    }
    *out = upload_mpo(ctx, m);
    return QTT_OK;
  });
}

qtt_status qtt_tc_stats(qtt_ctx ctx, long long* accepted, long long* fell_back) {
  if (!ctx || !accepted || !fell_back) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    long long h[2];
    QTT_CUDA_CHECK(cudaMemcpy(h, ctx->d_rf_counts + 2, sizeof h, cudaMemcpyDeviceToHost));
    *accepted = h[0];
    *fell_back = h[1];
    return check_device_errors(ctx);
  });
}

qtt_status qtt_gemm_tf32x3(qtt_ctx ctx, int M, int N, int K, const double* A, int lda, int tA,
                           const double* B, int ldb, int tB, double* C, int ldc) {
  if (!ctx || !A || !B || !C || M < 1 || N < 1 || K < 1) return QTT_ERR_ARG;
  if (lda < (tA ? M : K) || ldb < (tB ? K : N) || ldc < N) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    cudaStream_t s = stream_of(ctx);
    const int S = tc_gemm_splits(M, N, K);
    DBuf<float> scr(tc_gemm_scratch_floats(M, N, K, S), s);
    tc_gemm_f64(s, M, N, K, A, lda, tA, B, ldb, tB, C, ldc, ctx->d_err, scr.p, scr.n);
    return QTT_OK;
  });
}

qtt_status qtt_gemm_ozaki(qtt_ctx ctx, int M, int N, int K, const double* A, int lda, int tA,
                          long long sA, const double* B, int ldb, int tB, long long sB,
                          double* C, int ldc, long long sC, int batch, double alpha,
                          double beta) {
  if (!ctx || !A || !B || !C || M < 1 || N < 1 || K < 1 || batch < 1) return QTT_ERR_ARG;
  if (lda < (tA ? M : K) || ldb < (tB ? K : N) || ldc < N) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    GemmF64 g = gemm_plain(A, B, C, M, N, K, lda, ldb, ldc);
    g.tA = tA ? 1 : 0;
    g.tB = tB ? 1 : 0;
    g.nb1 = batch;
    g.sA1 = sA;
    g.sB1 = sB;
    g.sC1 = sC;
    g.alpha = alpha;
    g.beta = beta;
    if (!gemm_oz_eligible(g)) return QTT_ERR_SHAPE;
    const int S = gemm_oz_splits(g);
    DBuf<double> part(S > 1 ? (size_t)S * M * N : 0, stream_of(ctx));
    launch_gemm_oz(g, ctx->d_err, stream_of(ctx), true, part.p, part.n);
    return QTT_OK;
  });
}

qtt_status qtt_graph_stats(qtt_ctx ctx, long long* captured, long long* replays) {
  if (!ctx || !captured || !replays) return QTT_ERR_ARG;
  *captured = ctx->graphs_captured;
  *replays = ctx->graph_replays;
  return QTT_OK;
}

qtt_status qtt_profile_begin(qtt_ctx ctx) {
  return guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    std::lock_guard<std::mutex> g(g_prof.mu);
    for (auto& r : g_prof.recs) {
      g_prof.pool.push_back(r.e0);
      g_prof.pool.push_back(r.e1);
    }
    g_prof.recs.clear();
    svd_work_reset();
    g_prof.on = true;
    return QTT_OK;
  });
}

qtt_status qtt_profile_end(qtt_ctx ctx, char* buf, size_t cap) {
  if (!buf || cap == 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    g_prof.on = false;
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    std::lock_guard<std::mutex> g(g_prof.mu);
    struct Agg { long long n = 0; double ms = 0, flops = 0; };
    std::map<std::string, Agg> agg;
    for (auto& r : g_prof.recs) {
      float ms = 0.f;
      QTT_CUDA_CHECK(cudaEventElapsedTime(&ms, r.e0, r.e1));
      Agg& a = agg[r.name];
      a.n++;
      a.ms += ms;
      a.flops += r.flops;
      g_prof.pool.push_back(r.e0);
      g_prof.pool.push_back(r.e1);
    }
    g_prof.recs.clear();
    // the cluster SVDs count the arithmetic they actually did (sweeps are
    // data-dependent); that replaces the host's capacity-shape estimate
    unsigned long long work[2] = {0, 0};
    svd_work_read(work);
    if (agg.count("k_svd_cluster")) agg["k_svd_cluster"].flops = (double)work[0];
    if (agg.count("k_svd_cluster_f32")) agg["k_svd_cluster_f32"].flops = (double)work[1];
    std::string out = "{";
    bool first = true;
    for (auto& kv : agg) {
      char line[256];
      snprintf(line, sizeof line, "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e}",
               first ? "" : ", ", kv.first.c_str(), kv.second.n, kv.second.ms, kv.second.flops);
      out += line;
      first = false;
    }
    out += "}";
    if (out.size() + 1 > cap) return QTT_ERR_ARG;
    memcpy(buf, out.c_str(), out.size() + 1);
    return QTT_OK;
  });
}

qtt_status qtt_stats(qtt_ctx ctx, long long* cg_iters, long long* sweeps, long long* launches) {
  if (!ctx) return QTT_ERR_ARG;
  if (cg_iters) *cg_iters = ctx->cg_iters;
  if (sweeps) *sweeps = ctx->sweeps;
  if (launches) *launches = ctx->launches.n;
  return QTT_OK;
}

// ------------------------------------------------------- learned truncation
qtt_status qtt_learned_set(qtt_ctx ctx, const float* d_params) {
  if (!ctx || !d_params) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaMemcpyAsync(ctx->d_mlp, d_params, QTT_MLP_PARAMS * sizeof(float),
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->mlp_set = true;
    return QTT_OK;
  });
}

qtt_status qtt_learned_next_step(qtt_ctx ctx) {
  return guarded(ctx, [&]() -> qtt_status {
    learned_next_step(ctx);
    return QTT_OK;
  });
}

qtt_status qtt_learned_log(qtt_ctx ctx, float* h_feat, int* h_rank, int max_slots, int* n_slots) {
  if (!ctx || max_slots < 0 || (max_slots > 0 && (!h_feat || !h_rank))) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    const int ns = std::min(max_slots, (int)qtt_ctx_s::kSlots);
    const int nb = ctx->p.n + 1;
    std::vector<float> f((size_t)qtt_ctx_s::kSlots * qtt_ctx_s::kBonds * QTT_MLP_FEATURES);
    std::vector<int> r((size_t)qtt_ctx_s::kSlots * qtt_ctx_s::kBonds);
    const int t = ctx->tab;
    QTT_CUDA_CHECK(cudaMemcpy(f.data(), ctx->d_feat[t], f.size() * sizeof(float),
                              cudaMemcpyDeviceToHost));
    QTT_CUDA_CHECK(cudaMemcpy(r.data(), ctx->d_rank[t], r.size() * sizeof(int),
                              cudaMemcpyDeviceToHost));
    for (int sl = 0; sl < ns; sl++)
      for (int b = 0; b < nb; b++) {
        const size_t src = (size_t)sl * qtt_ctx_s::kBonds + b, dst = (size_t)sl * nb + b;
        h_rank[dst] = r[src];
        for (int j = 0; j < QTT_MLP_FEATURES; j++)
          h_feat[dst * QTT_MLP_FEATURES + j] = f[src * QTT_MLP_FEATURES + j];
      }
    if (n_slots) *n_slots = std::min(ctx->slot, (int)qtt_ctx_s::kSlots);
    return check_device_errors(ctx);
  });
}

qtt_status qtt_learned_stats(qtt_ctx ctx, long long* accepted, long long* fell_back) {
  return guarded(ctx, [&]() -> qtt_status {
    QTT_CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    long long h[2] = {0, 0};
    QTT_CUDA_CHECK(cudaMemcpy(h, ctx->d_rf_counts, sizeof h, cudaMemcpyDeviceToHost));
    if (accepted) *accepted = h[0];
    if (fell_back) *fell_back = h[1];
    return QTT_OK;
  });
}

qtt_status qtt_rf_omega(qtt_ctx ctx, unsigned long long key, int D, int w, double* d_out) {
  if (!ctx || !d_out || D < 1 || w < 1 || w > 1024) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    reg_alloc(d_out, (size_t)4 * D * w * sizeof(double));  // caller's buffer, this launch only
    try {
      launch_rf_omega(d_out, D, nullptr, w, nullptr, key, ctx->stream);
    } catch (...) {
      reg_free(d_out);
      throw;
    }
    reg_free(d_out);
    return QTT_OK;
  });
}

qtt_status qtt_mlp_forward(qtt_ctx ctx, const float* d_params, const float* d_X, int N,
                           float* d_out) {
  if (!ctx || !d_params || !d_X || !d_out || N < 0) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    launch_mlp_forward(d_params, d_X, N, d_out, ctx->stream);
    return QTT_OK;
  });
}

qtt_status qtt_mlp_loss_grad(qtt_ctx ctx, const float* d_params, const float* d_X,
                             const float* d_y, int N, float* d_grad, float* d_loss) {
  if (!ctx || !d_params || !d_X || !d_y || !d_grad || !d_loss || N < 1) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    cudaStream_t s = ctx->stream;
    DBuf<float> Z((size_t)N * QTT_MLP_HIDDEN, s), dout(N, s);
    launch_mlp_grad(d_params, d_X, d_y, N, Z.p, dout.p, d_grad, d_loss, s);
    return QTT_OK;
  });
}

qtt_status qtt_mlp_train(qtt_ctx ctx, float* d_params, const float* d_X, const float* d_y, int N,
                         int iters, float lr, float* d_loss_out) {
  if (!ctx || !d_params || !d_X || !d_y || N < 1 || iters < 0 || !(lr > 0.0f)) return QTT_ERR_ARG;
  return guarded(ctx, [&]() -> qtt_status {
    cudaStream_t s = ctx->stream;
    DBuf<float> Z((size_t)N * QTT_MLP_HIDDEN, s), dout(N, s), G(QTT_MLP_PARAMS, s),
        m(QTT_MLP_PARAMS, s), v(QTT_MLP_PARAMS, s), L(1, s);
    QTT_CUDA_CHECK(cudaMemsetAsync(m.p, 0, QTT_MLP_PARAMS * sizeof(float), s));
    QTT_CUDA_CHECK(cudaMemsetAsync(v.p, 0, QTT_MLP_PARAMS * sizeof(float), s));
    for (int t = 1; t <= iters; t++) {
      float* lp = d_loss_out ? d_loss_out + (t - 1) : L.p;
      launch_mlp_grad(d_params, d_X, d_y, N, Z.p, dout.p, G.p, lp, s);
      launch_adam(d_params, G.p, m.p, v.p, t, lr, s);
    }
    return QTT_OK;
  });
}

// ---------------------------------------------------------- batched steps
}  // extern "C"

struct qtt_batch_s {
  int device = 0;
  std::vector<qtt_ctx> ctx;
  std::vector<cudaStream_t> streams;
};

extern "C" {

qtt_status qtt_batch_create(qtt_batch* out, int device, int B, const qtt_params* per_traj) {
  if (!out || B < 1 || !per_traj) return QTT_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < B; i++)
    if (!valid_params(per_traj + i)) return QTT_ERR_ARG;
  auto b = new qtt_batch_s;
  b->device = device;
  qtt_status st = QTT_OK;
  if (cudaSetDevice(device) != cudaSuccess) st = QTT_ERR_CUDA;
  for (int i = 0; i < B && st == QTT_OK; i++) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      st = QTT_ERR_CUDA;
      break;
    }
    b->streams.push_back(s);
    qtt_ctx c = nullptr;
    st = qtt_create(&c, device, s, per_traj + i);
    if (st == QTT_OK) b->ctx.push_back(c);
  }
  if (st != QTT_OK) {
    qtt_batch_destroy(b);
    return st;
  }
  *out = b;
  return QTT_OK;
}

qtt_status qtt_batch_destroy(qtt_batch b) {
  if (!b) return QTT_ERR_ARG;
  for (qtt_ctx c : b->ctx) qtt_destroy(c);
  cudaSetDevice(b->device);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  delete b;
  return QTT_OK;
}

qtt_ctx qtt_batch_context(qtt_batch b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

qtt_status qtt_rk4_step_batched(qtt_batch b, qtt_mps* u1s, qtt_mps* u2s, const double* dts,
                                const double* nus) {
  if (!b || !u1s || !u2s || !dts || !nus) return QTT_ERR_ARG;
  const int B = (int)b->ctx.size();
  for (int i = 0; i < B; i++)
    if (!u1s[i] || !u2s[i] || u1s[i]->ctx != b->ctx[i] || u2s[i]->ctx != b->ctx[i])
      return QTT_ERR_ARG;
  std::vector<qtt_status> st(B, QTT_OK);
  std::vector<std::thread> th;
  th.reserve(B > 1 ? B - 1 : 0);
  for (int i = 1; i < B; i++)
    th.emplace_back([&, i] { st[i] = qtt_rk4_step(b->ctx[i], &u1s[i], &u2s[i], dts[i], nus[i]); });
  st[0] = qtt_rk4_step(b->ctx[0], &u1s[0], &u2s[0], dts[0], nus[0]);
  for (auto& t : th) t.join();
  for (int i = 0; i < B; i++)
    if (st[i] != QTT_OK) return st[i];
  return QTT_OK;
}

}  // extern "C"
