// Shared types of the QTT library: device-side dimension references, matrix
// views over capacity-padded storage, error handling and launch helpers.
//
// Storage model.  Every tensor (MPS core, environment, carry) lives in a
// buffer sized for its CAPACITY along each index; the ACTUAL extents (bond
// dimensions chosen by truncation on the device) are ints in device memory,
// and everything outside the actual extents is kept exactly zero.  Dense
// contractions therefore run over capacities without reading the actual
// dims (zeros contribute nothing), and only factorisations, which must see
// the true shape, read them.  No host synchronisation is needed to enqueue
// an operation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qtt.h"

#define QTT_MAX_N 20

// value = (p ? *p : 1) * c
struct DimRef {
  const int* p;
  int c;
};
static inline DimRef dconst(int c) { return DimRef{nullptr, c}; }
static inline DimRef dref(const int* p, int c = 1) { return DimRef{p, c}; }
__device__ __forceinline__ int dval(const DimRef& d) { return d.p ? (*d.p) * d.c : d.c; }

// One matrix index made of (hi, lo) with storage index hi * lcap + lo; the
// actual entries are hi < hact, lo < lact.  Compact index jc maps to
// (jc / lact) * lcap + jc % lact.
struct Axis {
  int hcap, lcap;
  DimRef hact, lact;
};
static inline Axis axis_prefix(int cap, DimRef act) { return Axis{cap, 1, act, dconst(1)}; }
static inline Axis axis_pair(int hcap, DimRef hact, int lcap, DimRef lact) {
  return Axis{hcap, lcap, hact, lact};
}
__device__ __forceinline__ int axis_len(const Axis& a) { return dval(a.hact) * dval(a.lact); }
__device__ __forceinline__ int axis_full(const Axis& a, int jc, int lact) {
  return (jc / lact) * a.lcap + (jc % lact);
}
__device__ __forceinline__ bool axis_actual(const Axis& a, int j, int hact, int lact) {
  return (j / a.lcap) < hact && (j % a.lcap) < lact;
}

// Row-major matrix over capacity storage: element (i, j) at ptr[i * ld + j].
struct MatView {
  double* ptr;
  int ld;
  Axis rows, cols;
};

// Device-side error flags (bit mask), read at synchronisation points.
// A guard that finds an inconsistent shape sets QTT_DEVERR_SHAPE and
// touches nothing.
enum : int {
  QTT_DEVERR_NUMERIC = 1,
  QTT_DEVERR_SHAPE = 2,
  QTT_DEVERR_TIMEOUT = 4,
};

struct LaunchCounter {
  long long n = 0;
};
extern thread_local LaunchCounter* g_launch_counter;
extern thread_local int* g_dev_err;
// Called after every kernel launch: counts it and, when the environment
// variable QTT_DEBUG_SYNC is set, waits for it and reports a failure by
// kernel name (a debugging aid that localises device-side faults).
void post_launch(const char* name, cudaStream_t s, double flops = 0.0);
// With QTT_PROFILE_SHAPES set in the environment the profiler separates one
// kernel's launches by problem shape: shape_name returns `base[tag]` as a
// stable, interned string (callers build the tag only when shape_profiling()).
bool shape_profiling();
const char* shape_name(const char* base, const char* tag);
// Called just before every kernel launch (records a start event when the
// context is profiling).
void pre_launch(cudaStream_t s);
static inline void count_launch() {
  if (g_launch_counter) g_launch_counter->n++;
}

#define QTT_CUDA_CHECK(expr)                                   \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) throw CudaError(_e, #expr, __LINE__); \
  } while (0)

struct CudaError {
  cudaError_t e;
  const char* what;
  int line;
  CudaError(cudaError_t e_, const char* w, int l) : e(e_), what(w), line(l) {}
};

struct QttError {
  qtt_status st;
  std::string msg;
  QttError(qtt_status s, std::string m) : st(s), msg(std::move(m)) {}
};

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Host-side registry of the library's device allocations.  Every launch
// checks, before it is enqueued, that each buffer range it will touch
// (computed from the capacities it is given) lies inside one registered
// allocation; a violation throws instead of launching.  Pointers the
// registry does not know (caller-owned buffers) are not checked.
void reg_alloc(const void* p, size_t bytes);
void reg_free(const void* p);
// throws QttError(QTT_ERR_SHAPE) if [p, p + count) leaves its allocation
void check_range(const void* p, long long count_elems, size_t elem_bytes, const char* what);
