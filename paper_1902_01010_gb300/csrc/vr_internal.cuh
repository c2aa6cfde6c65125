// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "vr.h"

namespace vr {

typedef unsigned long long u64;

constexpr int64_t kLattice = 1LL << 21;
constexpr int64_t kHalf = 1LL << 20;

// Device status block (allocated once per context by vr_create).
struct DevStatus {
  int error;          // first device-side error code (VR_ERR_*), 0 = none
  int error_where;    // kernel id that raised it
  long long aux[6];   // counters read back by the host (sizes, flags)
  long long info[8];  // diagnostics (e.g. degenerate cells, candidate counts)
};

}  // namespace vr

namespace vr {
struct Timers;  // per-kernel event timers (vr_api.cu)
struct Tuning;  // launch shapes chosen by the autotuner (tuning.cuh)
}

struct vr_ctx {
  int device;
  int sm_count;
  char err[512];
  vr::DevStatus *d_status;  // device
  long long *h_pinned;      // pinned host staging (64 entries)
  vr::Timers *timers;       // NULL unless timing is enabled
  vr::Tuning *tune;         // NULL until vr_autotune or vr_tuning_force is called
  cudaStream_t side;        // second stream for work that overlaps the caller's stream
  cudaEvent_t ev_fork, ev_join;
  cudaStream_t side2;       // third stream: the cell-tree build beside the f_l stage
  cudaEvent_t ev_fork2, ev_join2;
  cudaEvent_t ev_flbig, ev_tail;  // f_l of the largest halos done; their R and fit done
  int log_level;            // vr_set_log_level: 0 silent, 1 errors, 2 errors and calls
};

namespace vr {

// ------------------------------------------------------------------ errors
vr_status set_error(vr_ctx *ctx, vr_status st, const char *fmt, ...);
vr_status check_cuda(vr_ctx *ctx, cudaError_t e, const char *what);
// Level-2 log line of an entry point's call (vr_set_log_level); returns st.
vr_status log_call(vr_ctx *ctx, const char *name, int64_t n, vr_status st);
#define VR_CUDA(ctx, call)                                    \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return vr::check_cuda(ctx, _e, #call); \
  } while (0)
// Counts one kernel launch (every launch site calls it).
void count_launch();
#define VR_LAUNCHED(ctx, name)                                          \
  do {                                                                  \
    vr::count_launch();                                                 \
    cudaError_t _e = cudaGetLastError();                                \
    if (_e != cudaSuccess) return vr::check_cuda(ctx, _e, name);        \
  } while (0)

// Event timing around one launch when the context has timing enabled.
void timer_begin(vr_ctx *ctx, const char *name, cudaStream_t s);
void timer_end(vr_ctx *ctx, const char *name, cudaStream_t s);
#define VR_TIMED(ctx, name, s, ...) \
  do {                              \
    vr::timer_begin(ctx, name, s);  \
    __VA_ARGS__;                    \
    vr::timer_end(ctx, name, s);    \
  } while (0)

// Device-side error report (first one wins).
__device__ __forceinline__ void raise_error(DevStatus *st, int code, int where) {
  if (atomicCAS(&st->error, 0, code) == 0) st->error_where = where;
}

// ---------------------------------------------------------------- workspace
// Bump allocator over the caller's workspace. In "dry" mode (base == nullptr) it only
// measures, so the same carving code yields vr_workspace_size().
struct Arena {
  char *base;
  size_t off;
  size_t cap;
  explicit Arena(void *b = nullptr, size_t c = 0) : base((char *)b), off(0), cap(c) {}
  bool dry() const { return base == nullptr; }
  template <class T>
  T *take(size_t count) {
    size_t b = (off + 255) & ~(size_t)255;
    off = b + count * sizeof(T);
    return dry() ? nullptr : (T *)(base + b);
  }
  bool ok() const { return dry() || off <= cap; }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int grid_for(int64_t n, int block, int64_t cap = 1 << 30) {
  int64_t g = ceil_div(n > 0 ? n : 1, block);
  return (int)(g < cap ? g : cap);
}

// -------------------------------------------------------------- primitives
// Exclusive prefix sum of n values (in and out may alias). Scratch from `ar`.
template <class T>
size_t scan_scratch_bytes(int64_t n);
template <class T>
cudaError_t exclusive_scan(const T *in, T *out, int64_t n, void *scratch, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [begin_bit, end_bit).
// Ping-pongs between (k0, v0) and (k1, v1); returns the buffer index (0 or 1) holding
// the result via *which.
template <class K>
size_t radix_scratch_bytes(int64_t n);
template <class K>
cudaError_t radix_sort_pairs(K *k0, uint32_t *v0, K *k1, uint32_t *v1, int64_t n, int begin_bit,
                             int end_bit, void *scratch, cudaStream_t s, int *which);

// ------------------------------------------------------------------ geometry
__host__ __device__ __forceinline__ int min_image(int d) {
  // d in (-2^21, 2^21) -> [-2^20, 2^20]
  if (d >= (int)kHalf) d -= (int)kLattice;
  else if (d < -(int)kHalf) d += (int)kLattice;
  return d;
}

// Spreads the low 21 bits of x so that bit i moves to bit 3i.
__host__ __device__ __forceinline__ u64 spread3(u64 x) {
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}
__host__ __device__ __forceinline__ u64 morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---------------------------------------------------------- shared helpers
struct HaloSeg;  // defined in halos.cuh
vr_status params_check(vr_ctx *ctx, const vr_params *p);

}  // namespace vr
