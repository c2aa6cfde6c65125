// Context, parameters, errors and workspace sizing of the C ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <string>
#include <unordered_map>
#include <vector>

#include "tuning.cuh"
#include "vr_internal.cuh"
#include "vr_workspace.h"

namespace vr {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct Timer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open = nullptr;
  double ms = 0.0;
  long long launches = 0;
};
struct Timers {
  std::unordered_map<std::string, Timer> by_name;
};

static cudaEvent_t take_event(Timer &t) {
  if (!t.pool.empty()) {
    cudaEvent_t e = t.pool.back();
    t.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void timer_begin(vr_ctx *ctx, const char *name, cudaStream_t s) {
  if (!ctx || !ctx->timers) return;
  Timer &t = ctx->timers->by_name[name];
  t.open = take_event(t);
  cudaEventRecord(t.open, s);
}

void timer_end(vr_ctx *ctx, const char *name, cudaStream_t s) {
  if (!ctx || !ctx->timers) return;
  Timer &t = ctx->timers->by_name[name];
  if (!t.open) return;
  cudaEvent_t e = take_event(t);
  cudaEventRecord(e, s);
  t.pending.push_back({t.open, e});
  t.open = nullptr;
}

static void timers_collect(Timers *T) {
  for (auto &kv : T->by_name) {
    Timer &t = kv.second;
    for (auto &pr : t.pending) {
      cudaEventSynchronize(pr.second);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      t.ms += ms;
      t.launches += 1;
      t.pool.push_back(pr.first);
      t.pool.push_back(pr.second);
    }
    t.pending.clear();
  }
}

static void timers_free(Timers *T) {
  if (!T) return;
  timers_collect(T);
  for (auto &kv : T->by_name)
    for (cudaEvent_t e : kv.second.pool) cudaEventDestroy(e);
  delete T;
}

vr_status set_error(vr_ctx *ctx, vr_status st, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
    if (ctx->log_level >= 1) fprintf(stderr, "vr: %s (status %d)\n", ctx->err, (int)st);
  }
  return st;
}

vr_status check_cuda(vr_ctx *ctx, cudaError_t e, const char *what) {
  return set_error(ctx, VR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

vr_status log_call(vr_ctx *ctx, const char *name, int64_t n, vr_status st) {
  if (ctx && ctx->log_level >= 2)
    fprintf(stderr, "vr: %s n=%lld status %d\n", name, (long long)n, (int)st);
  return st;
}

vr_status params_check(vr_ctx *ctx, const vr_params *p) {
  if (!p) return set_error(ctx, VR_ERR_INVALID_ARG, "params is NULL");
  if (p->nse < 1 || p->nse > 1024)
    return set_error(ctx, VR_ERR_INVALID_ARG, "nse must be in [1, 1024]");
  if (p->nv < 1 || p->nv > 64 || p->nv > p->nse)
    return set_error(ctx, VR_ERR_INVALID_ARG, "nv must be in [1, min(64, nse)]");
  if (!(p->f_cell > 0.0) || p->f_cell > 1.0)
    return set_error(ctx, VR_ERR_INVALID_ARG, "f_cell must be in (0, 1]");
  if (p->ncell_min < 1) return set_error(ctx, VR_ERR_INVALID_ARG, "ncell_min must be >= 1");
  if (p->nmin < 1) return set_error(ctx, VR_ERR_INVALID_ARG, "nmin must be >= 1");
  if (p->nsearch_min < 2) return set_error(ctx, VR_ERR_INVALID_ARG, "nsearch_min must be >= 2");
  if (!(p->v_ratio >= 1.0)) return set_error(ctx, VR_ERR_INVALID_ARG, "v_ratio must be >= 1");
  if (!(p->theta_op >= 0.0) || !(p->theta_op < 1.5707963267948966))
    return set_error(ctx, VR_ERR_INVALID_ARG, "theta_op must be in [0, pi/2)");
  if (p->fit_nbins_min < 2 || p->fit_nbins_max < p->fit_nbins_min || p->fit_nbins_max > 1024)
    return set_error(ctx, VR_ERR_INVALID_ARG, "fit bins must satisfy 2 <= min <= max <= 1024");
  if (p->fit_iters < 0 || p->fit_iters > 10000)
    return set_error(ctx, VR_ERR_INVALID_ARG, "fit_iters must be in [0, 10000]");
  if (p->split_rule != 0 && p->split_rule != 1)
    return set_error(ctx, VR_ERR_INVALID_ARG, "split_rule must be 0 or 1");
  return VR_OK;
}

vr_status check_ws(vr_ctx *ctx, const Arena &ar, size_t ws_bytes) {
  if (ar.off > ws_bytes)
    return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need %zu bytes, got %zu",
                     ar.off, ws_bytes);
  return VR_OK;
}

// Reads the device status block; returns its error as a vr_status.
vr_status read_status(vr_ctx *ctx, cudaStream_t s, DevStatus *out) {
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(DevStatus),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  DevStatus st;
  memcpy(&st, ctx->h_pinned, sizeof(DevStatus));
  if (out) *out = st;
  if (st.error != 0) {
    vr_status code = (vr_status)st.error;
    const char *what = "device error";
    switch (st.error_where) {
      case 1: what = "halo spans half the box or more, or holds more than 2^22 particles"; break;
      case 2: what = "k-NN candidate search exceeded its bound"; break;
      case 3: what = "background cell tree exceeded its depth bound"; break;
      case 5: what = "link-count table of the two-stage linking is full"; break;
      default: break;
    }
    // clear for the next call
    VR_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 2, s));
    return set_error(ctx, code, "%s (kernel site %d)", what, st.error_where);
  }
  return VR_OK;
}

}  // namespace vr

using namespace vr;

extern "C" {

void vr_params_default(vr_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nse = 256;
  p->nv = 32;
  p->f_cell = 0.01;
  p->ncell_min = 100;
  p->nmin = 20;
  p->nsearch_min = 160;
  p->ell_th = 2.5;
  p->v_ratio = 2.0;
  p->theta_op = 0.1 * 3.14159265358979323846;
  p->use_lv = 1;
  p->use_vr_theta = 1;
  p->split_rule = 0;
  p->fit_nbins_min = 10;
  p->fit_nbins_max = 200;
  p->fit_iters = 100;
}

vr_status vr_create(vr_ctx **out, int device) {
  if (!out) return VR_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return VR_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return VR_ERR_CUDA;
  vr_ctx *c = (vr_ctx *)calloc(1, sizeof(vr_ctx));
  if (!c) return VR_ERR_CUDA;
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->d_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->h_pinned, 64 * sizeof(long long)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_flbig, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tail, cudaEventDisableTiming) != cudaSuccess) {
    vr_destroy(c);
    return VR_ERR_CUDA;
  }
  *out = c;
  return VR_OK;
}

void vr_destroy(vr_ctx *ctx) {
  if (!ctx) return;
  timers_free(ctx->timers);
  delete ctx->tune;
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->side2) cudaStreamDestroy(ctx->side2);
  if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
  if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_flbig) cudaEventDestroy(ctx->ev_flbig);
  if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  free(ctx);
}

const char *vr_last_error(const vr_ctx *ctx) { return ctx ? ctx->err : "no context"; }

vr_status vr_set_log_level(vr_ctx *ctx, int level) {
  if (!ctx || level < 0 || level > 2) return VR_ERR_INVALID_ARG;
  ctx->log_level = level;
  return VR_OK;
}

vr_status vr_sync(vr_ctx *ctx, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  return read_status(ctx, (cudaStream_t)stream, nullptr);
}

vr_status vr_workspace_size(vr_ctx *ctx, int64_t n, const vr_params *p, size_t *bytes) {
  if (!ctx || !bytes || n < 0 || n >= (1LL << 31))
    return set_error(ctx, VR_ERR_INVALID_ARG, "bad arguments to vr_workspace_size");
  vr_params d;
  if (!p) {
    vr_params_default(&d);
    p = &d;
  }
  vr_status st = params_check(ctx, p);
  if (st != VR_OK) return st;
  size_t a = ws_fof3d(n);
  size_t b = ws_substructure(n, p);
  *bytes = (a > b ? a : b) + 4096;
  return VR_OK;
}

vr_status vr_timing_enable(vr_ctx *ctx, int enable) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  if (enable && !ctx->timers) ctx->timers = new Timers();
  if (!enable && ctx->timers) {
    timers_free(ctx->timers);
    ctx->timers = nullptr;
  }
  return VR_OK;
}

vr_status vr_timing_read(vr_ctx *ctx, const char *name, double *ms, int64_t *launches) {
  if (!ctx || !name || !ms || !launches) return VR_ERR_INVALID_ARG;
  *ms = 0.0;
  *launches = 0;
  if (!ctx->timers) return VR_OK;
  timers_collect(ctx->timers);
  auto it = ctx->timers->by_name.find(name);
  if (it != ctx->timers->by_name.end()) {
    *ms = it->second.ms;
    *launches = it->second.launches;
  }
  return VR_OK;
}

vr_status vr_timing_reset(vr_ctx *ctx) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  if (!ctx->timers) return VR_OK;
  timers_collect(ctx->timers);
  for (auto &kv : ctx->timers->by_name) {
    kv.second.ms = 0.0;
    kv.second.launches = 0;
  }
  return VR_OK;
}

int64_t vr_launch_count(void) { return (int64_t)g_launches.load(); }

vr_status vr_autotune(vr_ctx *ctx, int enable) {
  if (!ctx || (enable != 0 && enable != 1)) return VR_ERR_INVALID_ARG;
  if (!ctx->tune) ctx->tune = new Tuning();
  Tuning *t = ctx->tune;
  t->on = enable;
  for (int k = 0; k < kVBins; ++k) {
    t->vtuned[k] = 0;
    t->vshape[k] = 0;
  }
  t->ltuned = 0;
  t->lshape = 0;
  return VR_OK;
}

vr_status vr_tuning_force(vr_ctx *ctx, int velden_shape, int link_shape) {
  if (!ctx || velden_shape < -1 || velden_shape >= kNVShapes || link_shape < -1 ||
      link_shape >= kNLShapes)
    return set_error(ctx, VR_ERR_INVALID_ARG, "shape index out of range");
  if (!ctx->tune) ctx->tune = new Tuning();
  ctx->tune->force_v = velden_shape;
  ctx->tune->force_l = link_shape;
  return VR_OK;
}

vr_status vr_tuning_report(const vr_ctx *ctx, char *buf, size_t len) {
  if (!ctx || !buf || len == 0) return VR_ERR_INVALID_ARG;
  Tuning none;
  const Tuning *t = ctx->tune ? ctx->tune : &none;
  std::string o = "{\"f_l\": {\"bins\": [\"> 65536\", \"4097-65536\", \"N_se+1-4096\"], "
                  "\"shapes\": [";
  char tmp[160];
  for (int j = 0; j < kNVShapes; ++j) {
    snprintf(tmp, sizeof(tmp), "%s{\"batch\": %d, \"maxreg\": %d, \"warps\": %d}", j ? ", " : "",
             kVShapes[j].batch, kVShapes[j].maxreg, kVShapes[j].warps);
    o += tmp;
  }
  o += "], \"chosen\": [";
  for (int k = 0; k < kVBins; ++k) {
    snprintf(tmp, sizeof(tmp), "%s%d", k ? ", " : "", vshape_for(ctx, k));
    o += tmp;
  }
  o += "], \"measured\": [";
  for (int k = 0; k < kVBins; ++k) {
    o += k ? ", [" : "[";
    for (int j = 0; j < kNVShapes; ++j) {
      snprintf(tmp, sizeof(tmp), "%s%.4f", j ? ", " : "", t->vtuned[k] ? t->vms[k][j] : -1.0);
      o += tmp;
    }
    o += "]";
  }
  o += "]}, \"link6\": {\"warps\": [";
  for (int j = 0; j < kNLShapes; ++j) {
    snprintf(tmp, sizeof(tmp), "%s%d", j ? ", " : "", kLWarps[j]);
    o += tmp;
  }
  snprintf(tmp, sizeof(tmp), "], \"chosen\": %d, \"measured\": [", lshape_for(ctx));
  o += tmp;
  for (int j = 0; j < kNLShapes; ++j) {
    snprintf(tmp, sizeof(tmp), "%s%.4f", j ? ", " : "", t->ltuned ? t->lms[j] : -1.0);
    o += tmp;
  }
  snprintf(tmp, sizeof(tmp), "]}, \"tuning_on\": %d, \"forced\": [%d, %d]}", t->on, t->force_v,
           t->force_l);
  o += tmp;
  if (o.size() + 1 > len) return VR_ERR_INVALID_ARG;
  memcpy(buf, o.c_str(), o.size() + 1);
  return VR_OK;
}

}  // extern "C"
