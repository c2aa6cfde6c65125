// Background-cell tree shared by the ratio, fit and linking stages.
#pragma once
#include "halos.cuh"

namespace vr {

// Node of a halo's entropy kd-tree. Child indices are relative to the halo's first node.
struct CellNode {
  int lo[3], hi[3];  // half-open region [lo, hi) per axis (unwrapped lattice units)
  uint32_t beg, end; // member range in the working permutation
  int axis;          // split axis, -1 for a leaf
  int split;         // split coordinate: left = {x < split}
  int left, right;
};

// Node slots reserved per searched halo: kNodeFactor * ceil(N_H / (N_cell + 1)) + 16.
// Median splits give at most about 4 N_H / N_cell nodes; coordinate ties can add more.
constexpr int kNodeFactor = 8;

struct Background {
  uint32_t *nodeoff;  // [H+1] first node slot of each halo (0-width for unsearched halos)
  uint32_t *leaf_of;  // [NHP] absolute node index of each member's leaf
  CellNode *nodes;
  double *mom;        // [nodes][13]: mass, xbar[3], vbar[3], sigma (xx yy zz xy xz yz)
};

int64_t max_nodes(int64_t n, const vr_params *p);
size_t background_bytes(int64_t n, const vr_params *p);
// Halo frames, cell trees and moments, then R (Eq. fvbg). With f_l == NULL (batched form
// only) the R kernel is left to background_ratio, so that the tree build can run beside
// the f_l stage on another stream.
vr_status run_background(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar,
                         const float *f_l, float *R, double *halo_stats, Background *out,
                         cudaStream_t s, const uint32_t *hoff_host = nullptr);
// R of the members of halos with szlo < N_H <= szhi.
vr_status background_ratio(vr_ctx *ctx, const HaloSeg &g, const Background &bg, const float *f_l,
                           float *R, cudaStream_t s, uint32_t szlo = 0,
                           uint32_t szhi = 0xffffffffu);
}  // namespace vr
