// Launch shapes picked by the autotuner (vr_autotune). A shape only lays the same work
// out differently over warps and registers: the arithmetic and its order are unchanged,
// so every shape gives bit-identical results.
#pragma once
#include "vr_internal.cuh"

namespace vr {

// f_l launches by halo size (members): above 65536, (4096, 65536], (N_se, 4096].
constexpr int kVBins = 3;
constexpr uint32_t kVBinEdge0 = 65536u, kVBinEdge1 = 4096u;

// f_l kernel shapes: candidates computed side by side, register cap, warps per block.
struct VShape {
  int batch, maxreg, warps;
};
constexpr int kNVShapes = 5;
constexpr VShape kVShapes[kNVShapes] = {{4, 80, 4}, {4, 80, 8}, {4, 80, 2}, {2, 80, 4}, {8, 96, 4}};

// 6D linker shapes: warps (32-candidate tiles) per block.
constexpr int kNLShapes = 3;
constexpr int kLWarps[kNLShapes] = {4, 2, 8};

struct Tuning {
  int on = 0;                       // measure each untuned bin at its next launch
  int vshape[kVBins] = {0, 0, 0};   // chosen f_l shape per bin (0 = default)
  int vtuned[kVBins] = {0, 0, 0};
  float vms[kVBins][kNVShapes] = {};
  int lshape = 0, ltuned = 0;       // chosen linker shape
  float lms[kNLShapes] = {};
  int force_v = -1, force_l = -1;   // every launch uses this shape (tests), -1 = off
};

// Shape index for f_l bin k / the linker under the context's tuning state.
inline int vshape_for(const vr_ctx *ctx, int k) {
  const Tuning *t = ctx ? ctx->tune : nullptr;
  if (!t) return 0;
  if (t->force_v >= 0) return t->force_v;
  return t->vtuned[k] ? t->vshape[k] : 0;
}
inline int lshape_for(const vr_ctx *ctx) {
  const Tuning *t = ctx ? ctx->tune : nullptr;
  if (!t) return 0;
  if (t->force_l >= 0) return t->force_l;
  return t->ltuned ? t->lshape : 0;
}
// True when the f_l bin k / the linker is to be measured at this launch.
inline bool vmeasure(const vr_ctx *ctx, int k) {
  const Tuning *t = ctx ? ctx->tune : nullptr;
  return t && t->on && t->force_v < 0 && !t->vtuned[k];
}
inline bool lmeasure(const vr_ctx *ctx) {
  const Tuning *t = ctx ? ctx->tune : nullptr;
  return t && t->on && t->force_l < 0 && !t->ltuned;
}

}  // namespace vr
