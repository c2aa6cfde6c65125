// Halo segmentation shared by the substructure stages.
#pragma once
#include "vr_internal.cuh"

namespace vr {

// Halos are 3D groups with at least nmin members (Sec. 2.2, N >= N_min), numbered in
// increasing label order. Members are stored per halo in one contiguous run of "slots",
// ordered by the Morton code of their unwrapped position inside the halo's bounding box
// (spatial locality for the neighbour searches).
struct HaloSeg {
  int64_t n = 0;       // particles
  int64_t H = 0;       // halos (host copy)
  int64_t NHP = 0;     // halo particles (host copy)
  int64_t nbig = 0;    // halos with more than nsmall members (host copy)
  uint32_t *hoff;      // [H+1] first slot of each halo
  uint32_t *hlabel;    // [H] halo label (minimum particle index)
  uint32_t *horder;    // [H] halos by decreasing size (work order of per-halo kernels)
  uint32_t *hid;       // [NHP] halo of each slot
  int4 *u;             // [NHP] unwrapped position (x, y, z) and local index w
  float4 *v;           // [NHP] velocity (x, y, z) and particle index (w, as int bits)
  // work array kept for later stages
  uint32_t *scratch_u32_a;  // [n + 1]
};

// Carves and builds the segmentation (one stream synchronisation to read H and NHP).
// The outputs take halo_seg_bytes(n, nmin) and stay; the build needs a further
// halo_seg_temp_bytes(n, nmin), released (arena offset restored) on return.
size_t halo_seg_bytes(int64_t n, int nmin);
size_t halo_seg_temp_bytes(int64_t n, int nmin);
vr_status build_halos(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                      const int32_t *label, int nmin, int nsmall, Arena &ar, cudaStream_t s,
                      HaloSeg *out);

}  // namespace vr
