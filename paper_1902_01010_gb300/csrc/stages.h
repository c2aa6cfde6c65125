// Stage entry points shared between the substructure translation units.
#pragma once
#include "halos.cuh"
#include "background.cuh"

namespace vr {
size_t velden_bytes(int64_t n, int nmin, int nse);
// hoff_host / plain: non-NULL / true selects one launch per halo (the plain form).
// ev_big (batched form): recorded on s once the f_l of every halo above kVBinEdge0
// members is written.
vr_status run_velden(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar, float *f_l,
                     cudaStream_t s, const uint32_t *hoff_host = nullptr,
                     cudaEvent_t ev_big = nullptr);
vr_status fill_f32(vr_ctx *ctx, float *a, int64_t n, float val, cudaStream_t s);
vr_status fill_i32(vr_ctx *ctx, int32_t *a, int64_t n, int32_t val, cudaStream_t s);
// Batched form: halos of szlo < N_H <= szhi only.
vr_status run_fit(vr_ctx *ctx, const HaloSeg &g, const Background &bg, const vr_params *p,
                  const float *R, double *halo_stats, float *ell, cudaStream_t s,
                  const uint32_t *hoff_host = nullptr, uint32_t szlo = 0,
                  uint32_t szhi = 0xffffffffu);
size_t fof6d_bytes(int64_t n, int nmin);
// Halo table rows (label, N_H, frame, sigma_v) for every halo, one CTA per halo.
vr_status run_halo_frame(vr_ctx *ctx, const HaloSeg &g, int nsearch_min, double *halo_stats,
                         cudaStream_t s);
// Field 6DFOF lengths: LX2 = lx2, LV2 = (alpha_v sigma_v)^2, SEARCHED = 1 for every halo.
vr_status field_lengths(vr_ctx *ctx, int64_t H, double lx2, double alpha_v, double *hs,
                        cudaStream_t s);
vr_status run_fof6d(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar,
                    const float *ell, const double *hp, int64_t nhalo, int32_t *label6,
                    cudaStream_t s, bool plain = false);
size_t grow_bytes(int64_t n, int nmin);
// Two-stage linking: relaxed growth of the stage-1 groups in label6 (in/out).
vr_status run_grow(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, const vr_grow_params *gp,
                   Arena &ar, const float *ell, const double *hp, int64_t nhalo, int32_t *label6,
                   cudaStream_t s);
size_t cores_bytes(int64_t n, int nmin);
// Optional extra outputs of the core search for core growth: `searched` (caller's device
// array [n]) gets the last loop at which each particle was in a searching halo's
// background (-1 if never); `prim` / `last` point to per-halo arrays in the arena (the
// primary core's label and level, -1 for halos without one), valid while the arena
// region is not reused.
struct CoreExtra {
  int32_t *searched = nullptr;
  const int *prim = nullptr;
  const int *last = nullptr;
};
// Core search (Eq. coreloop) on a segmentation whose halo rows hold SIGMA.
vr_status run_cores(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, const vr_core_params *cp,
                    double lx, double alpha_v, Arena &ar, const int32_t *label6, double *hs,
                    int32_t *core, int32_t *level, int64_t *ncores, cudaStream_t s,
                    CoreExtra *ex = nullptr);
size_t coregrow_bytes(int64_t n, int nmin);
// Core cleaning (Eq. coresig) and core growth (Eqs. coremeanphase-coredist) after
// run_cores(..., ex): grown [n] out (-1 where no core), *nkept = cores kept.
vr_status run_core_grow(vr_ctx *ctx, const HaloSeg &g, const vr_core_params *cp,
                        const vr_core_grow_params *gp, Arena &ar, const int32_t *core,
                        const int32_t *level, const CoreExtra &ex, int32_t *grown,
                        int64_t *nkept, cudaStream_t s);
size_t clean_bytes(int64_t n);
// Significance cleaning of groups (Eq. ellsig); synchronises the stream.
vr_status run_clean(vr_ctx *ctx, const float *ell, int64_t n, const vr_params *p, double beta,
                    int32_t *label6, int64_t *ngroups, Arena &ar, cudaStream_t s);
}  // namespace vr
