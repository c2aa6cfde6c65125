// C-ABI entry points of the substructure stages (Sec. 2.2): argument checks, workspace
// carving and stage sequencing. The kernels live in halos.cu, velden.cu, background.cu,
// ellfit.cu and fof6d.cu.
#include <math.h>

#include <vector>

#include "stages.h"
#include "tuning.cuh"
#include "vr_workspace.h"

namespace vr {

size_t ws_substructure(int64_t n, const vr_params *p) {
  // the f_l stage and the cell trees run side by side in the batched form: both regions
  size_t a = velden_bytes(n, p->nmin, p->nse), b = background_bytes(n, p), c = fof6d_bytes(n, p->nmin);
  size_t m = a + b;
  m = m > c ? m : c;
  const size_t t = halo_seg_temp_bytes(n, p->nmin);
  m = m > t ? m : t;
  const size_t cl = clean_bytes(n), gr = grow_bytes(n, p->nmin),
               co = cores_bytes(n, p->nmin) + coregrow_bytes(n, p->nmin);
  m = m > cl ? m : cl;
  m = m > gr ? m : gr;
  m = m > co ? m : co;
  return halo_seg_bytes(n, p->nmin) + m + 4096;
}

namespace {

// A workspace below the documented size is refused before any launch.
vr_status ws_upfront(vr_ctx *ctx, int64_t n, const vr_params *p, size_t ws_bytes) {
  const size_t need = ws_substructure(n, p);
  if (ws_bytes < need)
    return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small: need %zu bytes, got %zu",
                     need, ws_bytes);
  return VR_OK;
}

vr_status common_checks(vr_ctx *ctx, int64_t n, const vr_params *p) {
  if (n < 0 || n >= (1LL << 31)) return set_error(ctx, VR_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  return params_check(ctx, p);
}

// Per-halo linking lengths of the substructure search: lx2 = lx_sub^2 for every
// searched halo, lv2 = (alpha_lv sigma_host)^2.
__global__ void k_link_lengths(double *hs, int64_t H, double lx_sub, double alpha_lv) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  double *row = hs + h * VR_HALO_COLS;
  if (row[VR_H_SEARCHED] == 0.0) return;
  row[VR_H_LX2] = __dmul_rn(lx_sub, lx_sub);
  double t = __dmul_rn(alpha_lv, row[VR_H_SIGMA]);
  row[VR_H_LV2] = __dmul_rn(t, t);
}

}  // namespace
}  // namespace vr

using namespace vr;

extern "C" {

vr_status vr_velden(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                    const int32_t *label, const vr_params *p, float *f_l, void *ws,
                    size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !f_l || !ws) return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  st = fill_f32(ctx, f_l, n, NAN, s);
  if (st != VR_OK) return st;
  st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g);
  if (st != VR_OK) return st;
  return run_velden(ctx, g, p, ar, f_l, s);
}

vr_status vr_outlier_ratio(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *f_l,
                           int64_t n, const int32_t *label, const vr_params *p, float *R,
                           float *ell, double *halo_stats, int64_t *nhalo, void *ws,
                           size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (nhalo) *nhalo = 0;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !f_l || !label || !R || !ell || !halo_stats || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = fill_f32(ctx, R, n, NAN, s)) != VR_OK) return st;
  if ((st = fill_f32(ctx, ell, n, NAN, s)) != VR_OK) return st;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  Background bg;
  if ((st = run_background(ctx, g, p, ar, f_l, R, halo_stats, &bg, s)) != VR_OK) return st;
  if ((st = run_fit(ctx, g, bg, p, R, halo_stats, ell, s)) != VR_OK) return st;
  if (nhalo) *nhalo = g.H;
  return read_status(ctx, s, nullptr);
}

vr_status vr_fof6d(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *ell,
                   int64_t n, const int32_t *label, const double *halo_params, int64_t nhalo,
                   const vr_params *p, int32_t *label6, void *ws, size_t ws_bytes,
                   void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !halo_params || !label6 || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = fill_i32(ctx, label6, n, -1, s)) != VR_OK) return st;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  if (nhalo != g.H)
    return set_error(ctx, VR_ERR_INVALID_ARG, "nhalo = %lld but the labels define %lld halos",
                     (long long)nhalo, (long long)g.H);
  return run_fof6d(ctx, g, p, ar, ell, halo_params, nhalo, label6, s);
}

vr_status vr_fof6d_field(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                         const int32_t *label, double lx, double alpha_v, const vr_params *p,
                         int32_t *label6, double *halo_stats, int64_t *nhalo, void *ws,
                         size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (nhalo) *nhalo = 0;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !label6 || !halo_stats || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(lx > 0.0) || !(alpha_v > 0.0))
    return set_error(ctx, VR_ERR_INVALID_ARG, "lx and alpha_v must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = fill_i32(ctx, label6, n, -1, s)) != VR_OK) return st;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  if ((st = run_halo_frame(ctx, g, p->nsearch_min, halo_stats, s)) != VR_OK) return st;
  if ((st = field_lengths(ctx, g.H, lx * lx, alpha_v, halo_stats, s)) != VR_OK) return st;
  vr_params q = *p;
  q.use_lv = 1;
  q.use_vr_theta = 0;
  if ((st = run_fof6d(ctx, g, &q, ar, nullptr, halo_stats, g.H, label6, s)) != VR_OK) return st;
  if (nhalo) *nhalo = g.H;
  return read_status(ctx, s, nullptr);
}

void vr_grow_params_default(vr_grow_params *g) {
  if (!g) return;
  g->gamma_ell = 1.0;
  g->gamma_x = 2.0;
  g->gamma_vr = 1.0;
  g->gamma_theta = 1.0;
  g->f_merge = 0.25;
}

vr_status vr_grow_groups(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *ell,
                         int64_t n, const int32_t *label, const double *halo_params,
                         int64_t nhalo, const vr_params *p, const vr_grow_params *gp,
                         int32_t *label6, void *ws, size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !ell || !label || !halo_params || !gp || !label6 || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(gp->gamma_ell > 0.0) || !(gp->gamma_x > 0.0) || !(gp->gamma_vr > 0.0) ||
      !(gp->gamma_theta > 0.0) || !(gp->f_merge >= 0.0))
    return set_error(ctx, VR_ERR_INVALID_ARG, "gamma factors must be > 0 and f_merge >= 0");
  if (!(p->theta_op * gp->gamma_theta < 1.5707963267948966))
    return set_error(ctx, VR_ERR_INVALID_ARG, "gamma_theta * theta_op must be < pi/2");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  if (nhalo != g.H)
    return set_error(ctx, VR_ERR_INVALID_ARG, "nhalo = %lld but the labels define %lld halos",
                     (long long)nhalo, (long long)g.H);
  if ((st = run_grow(ctx, g, p, gp, ar, ell, halo_params, nhalo, label6, s)) != VR_OK) return st;
  return read_status(ctx, s, nullptr);
}

void vr_core_params_default(vr_core_params *c) {
  if (!c) return;
  c->alpha_x = 0.8;
  c->alpha_v = 1.0;
  c->n_loop = 5;
  c->f_c = 0.02;
  c->alpha_n = 1.2;
}

vr_status vr_core_search(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                         const int32_t *label, const int32_t *label6, double lx, double alpha_v,
                         const vr_params *p, const vr_core_params *cp, int32_t *core,
                         int32_t *level, int64_t *ncores, double *halo_stats, int64_t *nhalo,
                         void *ws, size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (ncores) *ncores = 0;
  if (nhalo) *nhalo = 0;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !cp || !core || !level || !halo_stats || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(lx > 0.0) || !(alpha_v > 0.0) || !(cp->alpha_x > 0.0) || !(cp->alpha_v > 0.0) ||
      cp->n_loop < 0 || cp->n_loop > 1000 || !(cp->f_c >= 0.0) || !(cp->alpha_n > 0.0))
    return set_error(ctx, VR_ERR_INVALID_ARG, "bad core search parameters");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  if ((st = run_halo_frame(ctx, g, p->nsearch_min, halo_stats, s)) != VR_OK) return st;
  if ((st = run_cores(ctx, g, p, cp, lx, alpha_v, ar, label6, halo_stats, core, level, ncores,
                      s)) != VR_OK)
    return st;
  if (nhalo) *nhalo = g.H;
  return read_status(ctx, s, nullptr);
}

void vr_core_grow_params_default(vr_core_grow_params *g) {
  if (!g) return;
  g->beta_c = 1.0;  // Table 1, beta_C
  g->mode = 2;      // Table A1, Use_phase_tensor_core_growth
}

vr_status vr_core_grow(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                       const int32_t *label, const int32_t *label6, double lx, double alpha_v,
                       const vr_params *p, const vr_core_params *cp, const vr_core_grow_params *gp,
                       int32_t *core, int32_t *level, int32_t *grown, int64_t *nkept,
                       double *halo_stats, int64_t *nhalo, void *ws, size_t ws_bytes,
                       void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (nkept) *nkept = 0;
  if (nhalo) *nhalo = 0;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !cp || !gp || !core || !level || !grown || !halo_stats || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(lx > 0.0) || !(alpha_v > 0.0) || !(cp->alpha_x > 0.0) || !(cp->alpha_v > 0.0) ||
      cp->n_loop < 0 || cp->n_loop > 1000 || !(cp->f_c >= 0.0) || !(cp->alpha_n > 0.0))
    return set_error(ctx, VR_ERR_INVALID_ARG, "bad core search parameters");
  if (!(gp->beta_c >= 0.0) || gp->mode < 0 || gp->mode > 2)
    return set_error(ctx, VR_ERR_INVALID_ARG, "bad core growth parameters");
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  if ((st = run_halo_frame(ctx, g, p->nsearch_min, halo_stats, s)) != VR_OK) return st;
  CoreExtra ex;
  ex.searched = ar.take<int32_t>(n);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  if ((st = run_cores(ctx, g, p, cp, lx, alpha_v, ar, label6, halo_stats, core, level, nullptr,
                      s, &ex)) != VR_OK)
    return st;
  if ((st = run_core_grow(ctx, g, cp, gp, ar, core, level, ex, grown, nkept, s)) != VR_OK)
    return st;
  if (nhalo) *nhalo = g.H;
  return read_status(ctx, s, nullptr);
}

vr_status vr_clean_groups(vr_ctx *ctx, const float *ell, int64_t n, const vr_params *p,
                          double beta, int32_t *label6, int64_t *ngroups, void *ws,
                          size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (ngroups) *ngroups = 0;
  if (n == 0) return VR_OK;
  if (!ell || !label6 || !ws) return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(beta >= 0.0)) return set_error(ctx, VR_ERR_INVALID_ARG, "beta must be >= 0");
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  return run_clean(ctx, ell, n, p, beta, label6, ngroups, ar, (cudaStream_t)stream);
}

vr_status vr_find_substructure(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                               const int32_t *label, double lx_sub, double alpha_lv,
                               const vr_params *p, int batched, float *f_l, float *R,
                               float *ell, int32_t *label6, double *halo_stats, int64_t *nhalo,
                               void *ws, size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  vr_status st = common_checks(ctx, n, p);
  if (st != VR_OK) return st;
  if (nhalo) *nhalo = 0;
  if (n == 0) return VR_OK;
  if (!pos || !vel || !label || !f_l || !R || !ell || !label6 || !halo_stats || !ws)
    return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (!(lx_sub > 0.0) || !(alpha_lv > 0.0))
    return set_error(ctx, VR_ERR_INVALID_ARG, "lx_sub and alpha_lv must be positive");
  if (batched != 0 && batched != 1)
    return set_error(ctx, VR_ERR_INVALID_ARG, "batched must be 0 (one launch per halo) or 1");
  const bool plain = batched == 0;
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar(ws, ws_bytes);
  if ((st = ws_upfront(ctx, n, p, ws_bytes)) != VR_OK) return st;
  HaloSeg g;
  if ((st = fill_f32(ctx, f_l, n, NAN, s)) != VR_OK) return st;
  if ((st = fill_f32(ctx, R, n, NAN, s)) != VR_OK) return st;
  if ((st = fill_f32(ctx, ell, n, NAN, s)) != VR_OK) return st;
  if ((st = fill_i32(ctx, label6, n, -1, s)) != VR_OK) return st;
  if ((st = build_halos(ctx, pos, vel, n, label, p->nmin, p->nse, ar, s, &g)) != VR_OK) return st;
  std::vector<uint32_t> hoff_host;
  if (plain && g.H > 0) {
    hoff_host.resize(g.H + 1);
    VR_CUDA(ctx, cudaMemcpyAsync(hoff_host.data(), g.hoff, (g.H + 1) * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
  }
  const uint32_t *hh = plain ? hoff_host.data() : nullptr;
  const size_t mark = ar.off;
  Background bg;
  if (plain) {
    if ((st = run_velden(ctx, g, p, ar, f_l, s, hh)) != VR_OK) return st;
    ar.off = mark;
    if ((st = run_background(ctx, g, p, ar, f_l, R, halo_stats, &bg, s, hh)) != VR_OK) return st;
  } else {
    // the halo frames and cell trees need only the segmentation: they run on a third
    // stream while the f_l kernels run on `s` (separate workspace regions); R waits for both
    VR_CUDA(ctx, cudaEventRecord(ctx->ev_fork2, s));
    VR_CUDA(ctx, cudaStreamWaitEvent(ctx->side2, ctx->ev_fork2, 0));
    if ((st = run_background(ctx, g, p, ar, nullptr, R, halo_stats, &bg, ctx->side2)) != VR_OK)
      return st;
    VR_CUDA(ctx, cudaEventRecord(ctx->ev_join2, ctx->side2));
    if ((st = run_velden(ctx, g, p, ar, f_l, s, nullptr, ctx->ev_flbig)) != VR_OK) return st;
    // R and the fit of the halos above kVBinEdge0 members (the first f_l launch) run on
    // the side stream while the f_l kernels of the smaller halos finish on s; the two
    // halves write disjoint halos and members
    const uint32_t edge = kVBinEdge0, all = 0xffffffffu;
    VR_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_flbig, 0));
    VR_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_join2, 0));
    if ((st = background_ratio(ctx, g, bg, f_l, R, ctx->side, edge, all)) != VR_OK) return st;
    if ((st = run_fit(ctx, g, bg, p, R, halo_stats, ell, ctx->side, nullptr, edge, all)) != VR_OK)
      return st;
    VR_CUDA(ctx, cudaEventRecord(ctx->ev_tail, ctx->side));
    VR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join2, 0));
    if ((st = background_ratio(ctx, g, bg, f_l, R, s, 0u, edge)) != VR_OK) return st;
    if ((st = run_fit(ctx, g, bg, p, R, halo_stats, ell, s, nullptr, 0u, edge)) != VR_OK) return st;
    VR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_tail, 0));
  }
  if (plain && (st = run_fit(ctx, g, bg, p, R, halo_stats, ell, s, hh)) != VR_OK) return st;
  ar.off = mark;
  if (g.H > 0) {
    k_link_lengths<<<grid_for(g.H, 256), 256, 0, s>>>(halo_stats, g.H, lx_sub, alpha_lv);
    VR_LAUNCHED(ctx, "k_link_lengths");
  }
  if ((st = run_fof6d(ctx, g, p, ar, ell, halo_stats, g.H, label6, s, plain)) != VR_OK) return st;
  if (nhalo) *nhalo = g.H;
  return log_call(ctx, "vr_find_substructure", n, read_status(ctx, s, nullptr));
}

}  // extern "C"
