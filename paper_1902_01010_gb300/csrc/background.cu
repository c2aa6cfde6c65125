// Background velocity model and outlier ratio (Sec. 2.2).
//
//  k_halo_frame   one CTA per halo: FP64 mean velocity and dispersion tensor about it
//                 (divided by N_H), sigma_host = |Sigma|^(1/6), halo table row.
//  k_cells_build  one CTA per searched halo: entropy kd-tree (Eq. S) down to cells of at
//                 most N_cell members, built node by node in global working arrays;
//                 split value = element floor(n/2) of the node in (coordinate, local
//                 index) order found by an 8-bit radix select; FP64 cell moments
//                 (Eqs. meanpos, meanvel, meandispvel) per leaf.
//  k_ratio        one thread per member: own cell plus the cells across its six faces
//                 (point location by descending the tree), inverse-distance weights
//                 (Eq. cellinterp), FP64 Cholesky, ln f_bg (Eq. fvbg), R = ln f_l - ln f_bg.
// Readings of points the paper leaves open (fixed identically in the oracle): bins
// n_b = max(2, floor(n^(1/3))) over [min, max] with bin = (x - min) n_b / (max - min + 1);
// argmax S with ties within 1e-12 going to the lower axis; an axis whose split leaves
// the left side empty is skipped for the next-best one; regions are half-open boxes;
// a face neighbour is the leaf containing the member's position moved to lo - 1 (or hi)
// along that axis, skipped outside the root region and counted once.
#include <math.h>

#include <vector>

#include "halos.cuh"
#include "vr_workspace.h"
#include "background.cuh"

namespace vr {

namespace {

constexpr int kFrameT = 256;       // threads per halo-frame CTA
constexpr int kSmallT = 256;       // threads per tree-building CTA, halos below kBigHalo
constexpr int kBigT = 1024;        // threads per tree-building CTA, halos of kBigHalo or more
constexpr int64_t kBigHalo = 65536;
constexpr int kMaxBins = 162;      // floor((2^22)^(1/3)) + 1

__device__ __forceinline__ int64_t ncell_of(int64_t nh, double f_cell, int ncell_min) {
  int64_t nc = (int64_t)floor(__dmul_rn(f_cell, (double)nh));
  if (nc < ncell_min) {
    nc = ncell_min;
    if (nh / 8 < nc) nc = nh / 8;
  }
  return nc < 1 ? 1 : nc;
}

__device__ __forceinline__ int64_t icbrt_dev(int64_t n) {
  int64_t m = (int64_t)cbrt((double)n);
  while (m > 0 && m * m * m > n) --m;
  while ((m + 1) * (m + 1) * (m + 1) <= n) ++m;
  return m;
}

// ---- block reductions (256 threads) ----
template <int NT, class T, class Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T *sbuf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sbuf[w] = v;
  __syncthreads();
  T r = sbuf[0];
  for (int k = 1; k < NT / 32; ++k) r = op(r, sbuf[k]);
  __syncthreads();
  return r;
}

struct MinOp { __device__ int operator()(int a, int b) const { return a < b ? a : b; } };
struct MaxOp { __device__ int operator()(int a, int b) const { return a > b ? a : b; } };
struct AddD { __device__ double operator()(double a, double b) const { return a + b; } };
struct AddI { __device__ int operator()(int a, int b) const { return a + b; } };

__device__ __forceinline__ int coord(const int4 &p, int a) { return a == 0 ? p.x : (a == 1 ? p.y : p.z); }

}  // namespace

// Halo table row for every halo (searched or not): FP64 frame and sigma_host.
__global__ void __launch_bounds__(kFrameT) k_halo_frame(const uint32_t *__restrict__ hoff,
                                                    const uint32_t *__restrict__ hlabel,
                                                    const uint32_t *__restrict__ horder, int64_t first,
                                                    int64_t last, const float4 *__restrict__ v,
                                                    int nsearch_min, double *__restrict__ hs_out) {
  __shared__ double sd[kFrameT / 32];
  if (first + (int64_t)blockIdx.x >= last) return;
  const int64_t h = horder[first + blockIdx.x];  // largest halos first
  const uint32_t b = hoff[h], e = hoff[h + 1];
  const double nh = (double)(e - b);
  double s[3] = {0, 0, 0};
  for (uint32_t m = b + threadIdx.x; m < e; m += kFrameT) {
    float4 q = v[m];
    s[0] += (double)q.x;
    s[1] += (double)q.y;
    s[2] += (double)q.z;
  }
  double mean[3];
  for (int k = 0; k < 3; ++k) mean[k] = block_reduce<kFrameT>(s[k], AddD(), sd) / nh;
  double c[6] = {0, 0, 0, 0, 0, 0};
  for (uint32_t m = b + threadIdx.x; m < e; m += kFrameT) {
    float4 q = v[m];
    double d0 = (double)q.x - mean[0], d1 = (double)q.y - mean[1], d2 = (double)q.z - mean[2];
    c[0] += d0 * d0; c[1] += d1 * d1; c[2] += d2 * d2;
    c[3] += d0 * d1; c[4] += d0 * d2; c[5] += d1 * d2;
  }
  double S[6];
  for (int k = 0; k < 6; ++k) S[k] = block_reduce<kFrameT>(c[k], AddD(), sd) / nh;
  if (threadIdx.x == 0) {
    double det = S[0] * (S[1] * S[2] - S[5] * S[5]) - S[3] * (S[3] * S[2] - S[5] * S[4]) +
                 S[4] * (S[3] * S[5] - S[1] * S[4]);
    double *row = hs_out + h * VR_HALO_COLS;
    row[VR_H_LABEL] = (double)hlabel[h];
    row[VR_H_NH] = nh;
    row[VR_H_SEARCHED] = (e - b) >= (uint32_t)nsearch_min ? 1.0 : 0.0;
    row[VR_H_RBAR] = NAN;
    row[VR_H_SIGR] = NAN;
    row[VR_H_VFX] = mean[0];
    row[VR_H_VFY] = mean[1];
    row[VR_H_VFZ] = mean[2];
    row[VR_H_SIGMA] = det > 0.0 ? pow(det, 1.0 / 6.0) : 0.0;
    row[VR_H_LX2] = NAN;
    row[VR_H_LV2] = NAN;
    row[VR_H_NCELLS] = 0.0;
  }
}

vr_status run_halo_frame(vr_ctx *ctx, const HaloSeg &g, int nsearch_min, double *halo_stats,
                         cudaStream_t s) {
  if (g.H == 0) return VR_OK;
  VR_TIMED(ctx, "halo_frame", s, k_halo_frame<<<(unsigned)g.H, kFrameT, 0, s>>>(
      g.hoff, g.hlabel, g.horder, 0, g.H, g.v, nsearch_min, halo_stats));
  VR_LAUNCHED(ctx, "k_halo_frame");
  return VR_OK;
}

// Node-capacity bound per halo (node table slots), 0 for halos not searched.
__global__ void k_node_caps(const uint32_t *__restrict__ hoff, int64_t H, int nsearch_min,
                            double f_cell, int ncell_min, uint32_t *__restrict__ caps) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h > H) return;
  if (h == H) {
    caps[H] = 0;
    return;
  }
  int64_t nh = hoff[h + 1] - hoff[h];
  if (nh < nsearch_min) {
    caps[h] = 0;
    return;
  }
  int64_t nc = ncell_of(nh, f_cell, ncell_min);
  caps[h] = (uint32_t)(kNodeFactor * ((nh + nc) / (nc + 1)) + 16);
}

constexpr int kStackCap = 128;  // depth of a warp's node stack
// Per-warp scratch of the tree build (dynamic shared memory, one per warp): axis
// histograms, the radix digit counts of a median selection and the warp's node stack.
struct WarpTree {
  int hist[3][kMaxBins];
  uint32_t dig[256];
  int stack[kStackCap];
};
constexpr int kPendCap = 256;  // nodes handed from the block to its warps

// The digit holding the need-th (1-based) key of a warp's 256 digit counts and the
// number of keys in the digits below it (warp-uniform).
__device__ __forceinline__ int warp_digit(const uint32_t *dig, int lane, uint32_t need,
                                          uint32_t *below) {
  uint32_t c[8], tot = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    c[i] = dig[8 * lane + i];
    tot += c[i];
  }
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const unsigned m = __ballot_sync(0xffffffffu, inc >= need);
  const int L = m ? __ffs(m) - 1 : 31;
  uint32_t run = inc - tot, bel = run;
  int bin = 8 * lane + 7;
  bool done = false;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (!done && run + c[i] >= need) {
      bin = 8 * lane + i;
      bel = run;
      done = true;
    }
    run += c[i];
  }
  *below = __shfl_sync(0xffffffffu, bel, L);
  return __shfl_sync(0xffffffffu, bin, L);
}

// Splits the subtree rooted at node `root` of one halo with a single warp, depth first:
// the same rules as the block path (entropy of n_b bins per axis, axis order by S with
// ties within 1e-12 to the lower axis, split at element floor(n/2) in (coordinate, local
// index) order, left = {x < split}, an axis leaving the left side empty skipped, stable
// partition), with warp shuffles and per-warp shared counts instead of block barriers.
// New nodes are numbered by an atomic counter; results do not depend on the numbering.
__device__ void warp_build(int root, uint32_t base, uint32_t cap, int64_t ncell, int split_rule,
                           const int4 *__restrict__ u, uint32_t *__restrict__ perm,
                           uint32_t *__restrict__ tmp, CellNode *__restrict__ nodes,
                           int *s_count, WarpTree &wt, DevStatus *st) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
  int sp = 0;
  if (lane == 0) wt.stack[0] = root;
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    const int id = wt.stack[--sp];
    __syncwarp();
    CellNode *nd = &nodes[base + id];
    const uint32_t nb_ = nd->beg, ne_ = nd->end;
    const int64_t n = ne_ - nb_;
    if (n <= ncell) {
      if (lane == 0) nd->axis = -1;
      continue;
    }
    int amin[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, amax[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    for (uint32_t i = nb_ + lane; i < ne_; i += 32) {
      const int4 p = u[perm[i]];
      amin[0] = min(amin[0], p.x); amin[1] = min(amin[1], p.y); amin[2] = min(amin[2], p.z);
      amax[0] = max(amax[0], p.x); amax[1] = max(amax[1], p.y); amax[2] = max(amax[2], p.z);
    }
    for (int o = 16; o; o >>= 1)
      for (int a = 0; a < 3; ++a) {
        amin[a] = min(amin[a], __shfl_xor_sync(FULL, amin[a], o));
        amax[a] = max(amax[a], __shfl_xor_sync(FULL, amax[a], o));
      }
    const int64_t nbins = max((int64_t)2, icbrt_dev(n));
    for (int k = lane; k < 3 * kMaxBins; k += 32) (&wt.hist[0][0])[k] = 0;
    __syncwarp();
    for (uint32_t i = nb_ + lane; i < ne_; i += 32) {
      const int4 p = u[perm[i]];
      for (int a = 0; a < 3; ++a)
        if (amax[a] > amin[a]) {
          const int64_t bin = ((int64_t)(coord(p, a) - amin[a]) * nbins) / ((int64_t)amax[a] - amin[a] + 1);
          atomicAdd(&wt.hist[a][bin], 1);
        }
    }
    __syncwarp();
    // Shannon entropy per axis (Eq. S); every lane ends with the same sums
    double S[3];
    int ok[3];
    for (int a = 0; a < 3; ++a) {
      ok[a] = amax[a] > amin[a];
      double part = 0.0;
      if (ok[a])
        for (int b = lane; b < nbins; b += 32) {
          const int c = wt.hist[a][b];
          if (c > 0) {
            const double f = (double)c / (double)n;
            part -= f * log(f);
          }
        }
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
      S[a] = ok[a] ? part / log((double)nbins) : 0.0;
    }
    int order[3], norder = 0, used[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r) {
      int best = -1;
      for (int a = 0; a < 3; ++a) {
        if (!ok[a] || used[a]) continue;
        if (best < 0) { best = a; continue; }
        if (split_rule == 0 ? (S[a] > S[best] + 1e-12) : (S[a] < S[best] - 1e-12)) best = a;
      }
      if (best < 0) break;
      used[best] = 1;
      order[norder++] = best;
    }
    bool split_done = false;
    for (int r = 0; r < norder && !split_done; ++r) {
      const int a = order[r];
      const int lo_a = amin[a];
      auto node_key = [&](uint32_t i) {
        const int4 p = u[perm[i]];
        return ((unsigned long long)(coord(p, a) - lo_a) << 22) | (unsigned)p.w;
      };
      // element of rank floor(n/2) by 8-bit radix selection from the top digit
      int bits = 22;
      {
        unsigned int ext = (unsigned int)(amax[a] - lo_a);
        while (ext) { ++bits; ext >>= 1; }
      }
      unsigned long long prefix = 0ULL;
      uint32_t rank = (uint32_t)(n / 2);
      for (int d = (bits + 7) / 8 - 1; d >= 0; --d) {
        const int sh = 8 * d;
        for (int k = lane; k < 256; k += 32) wt.dig[k] = 0u;
        __syncwarp();
        for (uint32_t i = nb_ + lane; i < ne_; i += 32) {
          const unsigned long long key = node_key(i);
          const unsigned long long hk = (sh + 8 >= 64) ? 0ULL : (key >> (sh + 8));
          const unsigned long long hp = (sh + 8 >= 64) ? 0ULL : (prefix >> (sh + 8));
          if (hk == hp) atomicAdd(&wt.dig[(key >> sh) & 0xffu], 1u);
        }
        __syncwarp();
        uint32_t below;
        const int dg = warp_digit(wt.dig, lane, rank + 1u, &below);
        prefix |= (unsigned long long)dg << sh;
        rank -= below;
        __syncwarp();
      }
      const int xs = lo_a + (int)(prefix >> 22);
      int cl = 0;
      for (uint32_t i = nb_ + lane; i < ne_; i += 32) cl += coord(u[perm[i]], a) < xs ? 1 : 0;
      for (int o = 16; o; o >>= 1) cl += __shfl_xor_sync(FULL, cl, o);
      const int nleft = cl;
      if (nleft == 0) continue;  // left side empty: next axis
      // stable partition: chunks of 32 in the node's order, left block then right block
      uint32_t offl = 0, offr = 0;
      for (uint32_t cb = nb_; cb < ne_; cb += 32) {
        const uint32_t i = cb + lane;
        const bool okm = i < ne_;
        uint32_t pm = 0;
        bool isl = false;
        if (okm) {
          pm = perm[i];
          isl = coord(u[pm], a) < xs;
        }
        const unsigned bl = __ballot_sync(FULL, okm && isl);
        const unsigned br = __ballot_sync(FULL, okm && !isl);
        if (okm) {
          if (isl) tmp[nb_ + offl + __popc(bl & lt)] = pm;
          else tmp[nb_ + nleft + offr + __popc(br & lt)] = pm;
        }
        offl += __popc(bl);
        offr += __popc(br);
      }
      __syncwarp();
      for (uint32_t i = nb_ + lane; i < ne_; i += 32) perm[i] = tmp[i];
      __syncwarp();
      int c0 = 0;
      if (lane == 0) {
        c0 = sp + 2 <= kStackCap ? atomicAdd(s_count, 2) : (int)cap;  // stack full: error
        if ((uint32_t)(c0 + 2) > cap) {
          raise_error(st, VR_ERR_UNSUPPORTED, 3);
          nd->axis = -1;
          c0 = -1;
        } else {
          CellNode *L = &nodes[base + c0], *R = &nodes[base + c0 + 1];
          for (int k = 0; k < 3; ++k) {
            L->lo[k] = R->lo[k] = nd->lo[k];
            L->hi[k] = R->hi[k] = nd->hi[k];
          }
          L->hi[a] = xs;
          R->lo[a] = xs;
          L->beg = nb_;
          L->end = nb_ + nleft;
          R->beg = nb_ + nleft;
          R->end = ne_;
          L->axis = R->axis = -1;
          nd->axis = a;
          nd->split = xs;
          nd->left = c0;
          nd->right = c0 + 1;
          wt.stack[sp] = c0 + 1;
          wt.stack[sp + 1] = c0;
        }
      }
      c0 = __shfl_sync(FULL, c0, 0);
      if (c0 >= 0) sp += 2;
      __syncwarp();
      split_done = true;
    }
    if (!split_done && lane == 0) nd->axis = -1;
    __syncwarp();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_cells_build(
    const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ horder,
    const uint32_t *__restrict__ nodeoff, int64_t first, int64_t last,
    const int4 *__restrict__ u, const float4 *__restrict__ v, int nsearch_min, double f_cell,
    int ncell_min, int split_rule, uint32_t *__restrict__ perm, uint32_t *__restrict__ tmp,
    CellNode *__restrict__ nodes, double *__restrict__ mom, uint32_t *__restrict__ leaf_of,
    double *__restrict__ hs_out, DevStatus *st) {
  __shared__ int s_hist[3][kMaxBins];
  __shared__ uint32_t s_dig[256];
  __shared__ int s_ri[NT / 32];
  __shared__ double s_rd[NT / 32];
  __shared__ int s_order[3];
  __shared__ int s_norder;
  __shared__ unsigned long long s_prefix;
  __shared__ int s_rank;
  __shared__ int s_count;
  __shared__ uint32_t s_scan[NT];
  __shared__ int s_pend[kPendCap];
  __shared__ int s_npend;
  extern __shared__ __align__(16) unsigned char tree_smem[];
  __shared__ uint32_t s_wl[NT / 32], s_wr[NT / 32];
  __shared__ int s_nleaves;
  if (first + (int64_t)blockIdx.x >= last) return;
  const int64_t h = horder[first + blockIdx.x];  // largest halos first
  const uint32_t hb = hoff[h], he = hoff[h + 1];
  const int64_t nh = he - hb;
  if (nh < nsearch_min) return;
  if ((NT == kBigT) != (nh >= kBigHalo)) return;  // each size class has its own launch
  const int64_t ncell = ncell_of(nh, f_cell, ncell_min);
  const uint32_t base = nodeoff[h], cap = nodeoff[h + 1] - base;
  const int t = threadIdx.x;
  for (uint32_t m = hb + t; m < he; m += NT) perm[m] = m;
  // root region: [min, max + 1)
  {
    int mn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, mx[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
    for (uint32_t m = hb + t; m < he; m += NT) {
      int4 p = u[m];
      mn[0] = min(mn[0], p.x); mn[1] = min(mn[1], p.y); mn[2] = min(mn[2], p.z);
      mx[0] = max(mx[0], p.x); mx[1] = max(mx[1], p.y); mx[2] = max(mx[2], p.z);
    }
    for (int a = 0; a < 3; ++a) {
      int lo = block_reduce<NT>(mn[a], MinOp(), s_ri);
      int hi = block_reduce<NT>(mx[a], MaxOp(), s_ri);
      if (t == 0) {
        nodes[base].lo[a] = lo;
        nodes[base].hi[a] = hi + 1;
      }
    }
    if (t == 0) {
      nodes[base].beg = hb;
      nodes[base].end = he;
      nodes[base].axis = -1;
      s_count = 1;
    }
  }
  if (t == 0) s_npend = 0;
  __syncthreads();
  // nodes of at most `tw` members are split by single warps afterwards (whole subtrees);
  // larger ones by the whole block, one at a time
  const int64_t tw = max((int64_t)1024, nh / (2 * (NT / 32)));
  for (int cur = 0; cur < s_count; ++cur) {
    CellNode *nd = &nodes[base + cur];
    const uint32_t nb_ = nd->beg, ne_ = nd->end;
    const int64_t n = ne_ - nb_;
    __syncthreads();
    if (n <= ncell) {
      if (t == 0) nd->axis = -1;
      __syncthreads();
      continue;
    }
    const bool hand = n <= tw && s_npend < kPendCap;  // read by every thread before the write
    __syncthreads();
    if (hand) {
      if (t == 0) s_pend[s_npend++] = cur;
      __syncthreads();
      continue;
    }
    // extent of the node's members per axis
    int mn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, mx[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
#pragma unroll 4
    for (uint32_t i = nb_ + t; i < ne_; i += NT) {
      int4 p = u[perm[i]];
      mn[0] = min(mn[0], p.x); mn[1] = min(mn[1], p.y); mn[2] = min(mn[2], p.z);
      mx[0] = max(mx[0], p.x); mx[1] = max(mx[1], p.y); mx[2] = max(mx[2], p.z);
    }
    int amin[3], amax[3];
    for (int a = 0; a < 3; ++a) {
      amin[a] = block_reduce<NT>(mn[a], MinOp(), s_ri);
      amax[a] = block_reduce<NT>(mx[a], MaxOp(), s_ri);
    }
    const int64_t nbins = max((int64_t)2, icbrt_dev(n));
    for (int k = t; k < 3 * kMaxBins; k += NT) (&s_hist[0][0])[k] = 0;
    __syncthreads();
#pragma unroll 4
    for (uint32_t i = nb_ + t; i < ne_; i += NT) {
      int4 p = u[perm[i]];
      for (int a = 0; a < 3; ++a) {
        if (amax[a] > amin[a]) {
          int64_t bin = ((int64_t)(coord(p, a) - amin[a]) * nbins) / ((int64_t)amax[a] - amin[a] + 1);
          atomicAdd(&s_hist[a][bin], 1);
        }
      }
    }
    __syncthreads();
    // Shannon entropy per axis (Eq. S): every thread sums the bins it owns, then a block
    // reduction; thread 0 orders the axes.
    double Sa[3];
    for (int a = 0; a < 3; ++a) {
      double part = 0.0;
      if (amax[a] > amin[a]) {
        for (int b = t; b < nbins; b += NT) {
          int c = s_hist[a][b];
          if (c > 0) {
            double f = (double)c / (double)n;
            part -= f * log(f);
          }
        }
      }
      Sa[a] = block_reduce<NT>(part, AddD(), s_rd);
    }
    if (t == 0) {
      double S[3];
      int ok[3];
      for (int a = 0; a < 3; ++a) {
        ok[a] = amax[a] > amin[a];
        S[a] = ok[a] ? Sa[a] / log((double)nbins) : 0.0;
      }
      int used[3] = {0, 0, 0}, no = 0;
      for (int r = 0; r < 3; ++r) {
        int best = -1;
        for (int a = 0; a < 3; ++a) {
          if (!ok[a] || used[a]) continue;
          if (best < 0) { best = a; continue; }
          if (split_rule == 0 ? (S[a] > S[best] + 1e-12) : (S[a] < S[best] - 1e-12)) best = a;
        }
        if (best < 0) break;
        used[best] = 1;
        s_order[no++] = best;
      }
      s_norder = no;
    }
    __syncthreads();
    bool split_done = false;
    const int norder = s_norder;
    for (int r = 0; r < norder && !split_done; ++r) {
      const int a = s_order[r];
      const int lo_a = amin[a];
      // element of rank floor(n/2) by key ((x - lo) << 22 | local index); keys are unique
      auto node_key = [&](uint32_t i) {
        int4 p = u[perm[i]];
        return ((unsigned long long)(coord(p, a) - lo_a) << 22) | (unsigned)p.w;
      };
      {
        // large node: 8-bit radix selection from the top digit
        int bits = 22;
        {
          unsigned int ext = (unsigned int)(amax[a] - lo_a);
          while (ext) { ++bits; ext >>= 1; }
        }
        int ndig = (bits + 7) / 8;
        if (t == 0) {
          s_prefix = 0ULL;
          s_rank = (int)(n / 2);
        }
        __syncthreads();
        for (int d = ndig - 1; d >= 0; --d) {
          if (t < 256) s_dig[t] = 0;
          __syncthreads();
          const int sh = 8 * d;
          const unsigned long long pre = s_prefix;
#pragma unroll 4
          for (uint32_t i = nb_ + t; i < ne_; i += NT) {
            unsigned long long key = node_key(i);
            unsigned long long hiK = (sh + 8 >= 64) ? 0ULL : (key >> (sh + 8));
            unsigned long long hiP = (sh + 8 >= 64) ? 0ULL : (pre >> (sh + 8));
            if (hiK == hiP) atomicAdd(&s_dig[(key >> sh) & 0xffu], 1u);
          }
          __syncthreads();
          // exclusive scan of the 256 digit counts (thread t < 256 owns digit t): warp
          // scans, then the 8 warp totals
          const uint32_t c = t < 256 ? s_dig[t] : 0u;
          uint32_t incl = c;
          for (int o = 1; o < 32; o <<= 1) {
            uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
            if ((t & 31) >= o) incl += x;
          }
          if (t < 256 && (t & 31) == 31) s_scan[t >> 5] = incl;
          __syncthreads();
          uint32_t wbase = 0;
          if (t < 256)
            for (int w = 0; w < (t >> 5); ++w) wbase += s_scan[w];
          incl += wbase;
          const uint32_t excl = incl - c;
          const int rk = s_rank;
          __syncthreads();
          if (t < 256 && (int)excl <= rk && rk < (int)incl) {
            s_prefix = pre | ((unsigned long long)t << sh);
            s_rank = rk - (int)excl;
          }
          __syncthreads();
        }
      }
      const int xs = lo_a + (int)(s_prefix >> 22);
      // left = {x < xs}
      int cl = 0;
#pragma unroll 4
      for (uint32_t i = nb_ + t; i < ne_; i += NT) cl += coord(u[perm[i]], a) < xs ? 1 : 0;
      const int nleft = block_reduce<NT>(cl, AddI(), s_ri);
      if (nleft == 0) continue;  // left side empty: next axis
      // stable partition into tmp (left block, then right block, each in the node's
      // order): per chunk, every warp's ballot counts are scanned across the warps, so
      // the member order, and with it every later FP64 sum, does not depend on warp
      // scheduling
      {
        const unsigned lt = (1u << (t & 31)) - 1u;
        const int w = t >> 5, lane = t & 31;
        uint32_t offl = 0, offr = 0;
        for (uint32_t cb = nb_; cb < ne_; cb += NT) {
          const uint32_t i = cb + t;
          const bool ok = i < ne_;
          uint32_t pm = 0;
          bool isl = false;
          if (ok) {
            pm = perm[i];
            isl = coord(u[pm], a) < xs;
          }
          const unsigned bl = __ballot_sync(0xffffffffu, ok && isl);
          const unsigned br = __ballot_sync(0xffffffffu, ok && !isl);
          if (lane == 0) {
            s_wl[w] = (uint32_t)__popc(bl);
            s_wr[w] = (uint32_t)__popc(br);
          }
          __syncthreads();
          // inclusive scan of the per-warp counts, redone by every warp
          uint32_t xl = lane < NT / 32 ? s_wl[lane] : 0u, xr = lane < NT / 32 ? s_wr[lane] : 0u;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yl = __shfl_up_sync(0xffffffffu, xl, o);
            const uint32_t yr = __shfl_up_sync(0xffffffffu, xr, o);
            if (lane >= o) {
              xl += yl;
              xr += yr;
            }
          }
          const uint32_t basel = offl + __shfl_sync(0xffffffffu, xl, w) - (uint32_t)__popc(bl);
          const uint32_t baser = offr + __shfl_sync(0xffffffffu, xr, w) - (uint32_t)__popc(br);
          offl += __shfl_sync(0xffffffffu, xl, 31);
          offr += __shfl_sync(0xffffffffu, xr, 31);
          if (ok) {
            if (isl) tmp[nb_ + basel + __popc(bl & lt)] = pm;
            else tmp[nb_ + nleft + baser + __popc(br & lt)] = pm;
          }
          __syncthreads();  // s_wl / s_wr are rewritten by the next chunk
        }
      }
      __syncthreads();
#pragma unroll 4
      for (uint32_t i = nb_ + t; i < ne_; i += NT) perm[i] = tmp[i];
      __syncthreads();
      if (t == 0) {
        int c0 = s_count;
        if ((uint32_t)(c0 + 2) > cap) {
          raise_error(st, VR_ERR_UNSUPPORTED, 3);
          nd->axis = -1;
        } else {
          CellNode *L = &nodes[base + c0], *R = &nodes[base + c0 + 1];
          for (int k = 0; k < 3; ++k) {
            L->lo[k] = R->lo[k] = nd->lo[k];
            L->hi[k] = R->hi[k] = nd->hi[k];
          }
          L->hi[a] = xs;
          R->lo[a] = xs;
          L->beg = nb_;
          L->end = nb_ + nleft;
          R->beg = nb_ + nleft;
          R->end = ne_;
          L->axis = R->axis = -1;
          nd->axis = a;
          nd->split = xs;
          nd->left = c0;
          nd->right = c0 + 1;
          s_count = c0 + 2;
        }
      }
      split_done = true;
      __syncthreads();
    }
    if (!split_done && t == 0) nd->axis = -1;
    __syncthreads();
  }
  // the handed-over nodes: one warp builds each subtree
  __syncthreads();
  {
    WarpTree &wt = reinterpret_cast<WarpTree *>(tree_smem)[t >> 5];
    const int np = s_npend;
    for (int k = t >> 5; k < np; k += NT / 32)
      warp_build(s_pend[k], base, cap, ncell, split_rule, u, perm, tmp, nodes, &s_count, wt, st);
  }
  // leaves: FP64 moments and membership, one warp per leaf (leaves taken round-robin by
  // the block's warps; warp-shuffle reductions, so no block barrier per leaf)
  if (t == 0) s_nleaves = 0;
  __syncthreads();
  const int count = s_count;
  {
    const int lane = t & 31, wid = t >> 5;
    const unsigned FULL = 0xffffffffu;
    for (int cur = wid; cur < count; cur += NT / 32) {
      const CellNode *nd = &nodes[base + cur];
      if (nd->axis >= 0) continue;  // the same node for the whole warp
      if (lane == 0) atomicAdd(&s_nleaves, 1);
      const uint32_t b = nd->beg, e = nd->end;
      const double M = (double)(e - b);
      long long sx[3] = {0, 0, 0};
      double sv[3] = {0, 0, 0};
      for (uint32_t i = b + lane; i < e; i += 32) {
        const uint32_t m = perm[i];
        leaf_of[m] = base + cur;
        const int4 p = u[m];
        const float4 q = v[m];
        sx[0] += p.x; sx[1] += p.y; sx[2] += p.z;
        sv[0] += (double)q.x; sv[1] += (double)q.y; sv[2] += (double)q.z;
      }
      for (int o = 16; o; o >>= 1)
        for (int k = 0; k < 3; ++k) {
          sx[k] += __shfl_xor_sync(FULL, sx[k], o);
          sv[k] += __shfl_xor_sync(FULL, sv[k], o);
        }
      double xm[3], vm[3];
      for (int k = 0; k < 3; ++k) {
        xm[k] = (double)sx[k] / M;
        vm[k] = sv[k] / M;
      }
      double c[6] = {0, 0, 0, 0, 0, 0};
      for (uint32_t i = b + lane; i < e; i += 32) {
        const float4 q = v[perm[i]];
        const double d0 = (double)q.x - vm[0], d1 = (double)q.y - vm[1], d2 = (double)q.z - vm[2];
        c[0] += d0 * d0; c[1] += d1 * d1; c[2] += d2 * d2;
        c[3] += d0 * d1; c[4] += d0 * d2; c[5] += d1 * d2;
      }
      for (int o = 16; o; o >>= 1)
        for (int k = 0; k < 6; ++k) c[k] += __shfl_xor_sync(FULL, c[k], o);
      if (lane == 0) {
        double *out = mom + 13 * (int64_t)(base + cur);
        out[0] = M;
        for (int k = 0; k < 3; ++k) { out[1 + k] = xm[k]; out[4 + k] = vm[k]; }
        for (int k = 0; k < 6; ++k) out[7 + k] = c[k] / M;
      }
    }
  }
  __syncthreads();
  const int nleaves = s_nleaves;
  if (t == 0) hs_out[h * VR_HALO_COLS + VR_H_NCELLS] = (double)nleaves;
}

// Leaf containing point p, or -1 outside the root region.
__device__ __forceinline__ int locate(const CellNode *__restrict__ nodes, uint32_t base, const int *p) {
  const CellNode &r = nodes[base];
  for (int a = 0; a < 3; ++a)
    if (p[a] < r.lo[a] || p[a] >= r.hi[a]) return -1;
  uint32_t id = base;
  for (int guard = 0; guard < 4096; ++guard) {
    const CellNode &nd = nodes[id];
    if (nd.axis < 0) return (int)id;
    id = base + (p[nd.axis] < nd.split ? nd.left : nd.right);
  }
  return -1;
}

// Cholesky of (xx, yy, zz, xy, xz, yz); false if not positive definite.
__device__ __forceinline__ bool chol3(const double *s, double *L) {
  double a00 = s[0], a11 = s[1], a22 = s[2], a10 = s[3], a20 = s[4], a21 = s[5];
  if (!(a00 > 0.0)) return false;
  double l00 = sqrt(a00);
  double l10 = a10 / l00, l20 = a20 / l00;
  double d1 = a11 - l10 * l10;
  if (!(d1 > 0.0)) return false;
  double l11 = sqrt(d1);
  double l21 = (a21 - l20 * l10) / l11;
  double d2 = a22 - l20 * l20 - l21 * l21;
  if (!(d2 > 0.0)) return false;
  double l22 = sqrt(d2);
  L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = l22;
  return true;
}

__global__ void k_ratio(const uint32_t *__restrict__ hid, const uint32_t *__restrict__ nodeoff,
                        int64_t m0, int64_t m1, const int4 *__restrict__ u, const float4 *__restrict__ v,
                        const float *__restrict__ f_l, const CellNode *__restrict__ nodes,
                        const double *__restrict__ mom, const uint32_t *__restrict__ leaf_of,
                        float *__restrict__ R, unsigned long long *__restrict__ ndegen,
                        const uint32_t *__restrict__ hoff, uint32_t szlo, uint32_t szhi) {
  int64_t m = m0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // members [m0, m1)
  if (m >= m1) return;
  const uint32_t h = hid[m];
  const uint32_t base = nodeoff[h];
  if (nodeoff[h + 1] == base) return;  // halo not searched
  const uint32_t nh = hoff[h + 1] - hoff[h];
  if (nh <= szlo || nh > szhi) return;  // another launch's halo
  const int4 p = u[m];
  const float4 q = v[m];
  const uint32_t own = leaf_of[m];
  const CellNode &nd = nodes[own];
  int cells[7];
  int nc = 0;
  cells[nc++] = (int)own;
  for (int a = 0; a < 3; ++a) {
    for (int side = 0; side < 2; ++side) {
      int pp[3] = {p.x, p.y, p.z};
      pp[a] = side == 0 ? nd.lo[a] - 1 : nd.hi[a];
      int c = locate(nodes, base, pp);
      if (c < 0) continue;
      bool dup = false;
      for (int k = 0; k < nc; ++k) dup |= cells[k] == c;
      if (!dup) cells[nc++] = c;
    }
  }
  double w[7];
  int zero = -1;
  for (int k = 0; k < nc; ++k) {
    const double *c = mom + 13 * (int64_t)cells[k];
    double dx = (double)p.x - c[1], dy = (double)p.y - c[2], dz = (double)p.z - c[3];
    const double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 == 0.0) {
      zero = k;
      break;
    }
    w[k] = rsqrt(d2);  // 1 / |x - xbar|
  }
  double vb[3] = {0, 0, 0}, sg[6] = {0, 0, 0, 0, 0, 0};
  if (zero >= 0) {
    const double *c = mom + 13 * (int64_t)cells[zero];
    for (int k = 0; k < 3; ++k) vb[k] = c[4 + k];
    for (int k = 0; k < 6; ++k) sg[k] = c[7 + k];
  } else {
    double ws = 0.0;
    for (int k = 0; k < nc; ++k) ws += w[k];
    for (int k = 0; k < nc; ++k) {
      const double *c = mom + 13 * (int64_t)cells[k];
      double f = w[k] / ws;
      for (int j = 0; j < 3; ++j) vb[j] += f * c[4 + j];
      for (int j = 0; j < 6; ++j) sg[j] += f * c[7 + j];
    }
  }
  double L[6];
  const int pidx = __float_as_int(q.w);
  if (!chol3(sg, L)) {
    R[pidx] = NAN;
    atomicAdd(ndegen, 1ULL);
    return;
  }
  double d0 = (double)q.x - vb[0], d1 = (double)q.y - vb[1], d2 = (double)q.z - vb[2];
  double y0 = d0 / L[0];
  double y1 = (d1 - L[1] * y0) / L[2];
  double y2 = (d2 - L[3] * y0 - L[4] * y1) / L[5];
  double qf = y0 * y0 + y1 * y1 + y2 * y2;
  const double ln2pi = 1.8378770664093453;  // ln(2 pi)
  double lnfbg = -0.5 * qf - 1.5 * ln2pi - log(L[0] * L[2] * L[5]);  // ln det L
  R[pidx] = (float)(log((double)f_l[pidx]) - lnfbg);
}

size_t background_bytes(int64_t n, const vr_params *p) {
  Arena ar;
  int64_t hmax = n / (p->nmin > 0 ? p->nmin : 1) + 2;
  ar.take<uint32_t>(hmax + 1);                       // nodeoff
  ar.take<uint32_t>(n);                              // perm
  ar.take<uint32_t>(n);                              // tmp
  ar.take<uint32_t>(n);                              // leaf_of
  int64_t nodes = max_nodes(n, p);
  ar.take<CellNode>(nodes);
  ar.take<double>(13 * nodes);
  ar.take<char>(scan_scratch_bytes<uint32_t>(hmax + 1));
  return ar.off;
}

int64_t max_nodes(int64_t n, const vr_params *p) {
  // smallest N_cell over searched halos is that of the smallest searched halo
  int64_t ns = p->nsearch_min;
  int64_t nc = (int64_t)floor(p->f_cell * (double)ns);
  if (nc < p->ncell_min) {
    nc = p->ncell_min;
    if (ns / 8 < nc) nc = ns / 8;
  }
  if (nc < 1) nc = 1;
  return kNodeFactor * ((n + nc) / (nc + 1)) + 16 * (n / ns + 1) + 16;
}

vr_status run_background(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar,
                         const float *f_l, float *R, double *halo_stats, Background *out,
                         cudaStream_t s, const uint32_t *hoff_host) {
  const int64_t H = g.H;
  int64_t hmax = g.n / (p->nmin > 0 ? p->nmin : 1) + 2;
  Background &bg = *out;
  bg.nodeoff = ar.take<uint32_t>(hmax + 1);
  uint32_t *perm = ar.take<uint32_t>(g.n);
  uint32_t *tmp = ar.take<uint32_t>(g.n);
  bg.leaf_of = ar.take<uint32_t>(g.n);
  int64_t cap = max_nodes(g.n, p);
  bg.nodes = ar.take<CellNode>(cap);
  bg.mom = ar.take<double>(13 * cap);
  void *scr = ar.take<char>(scan_scratch_bytes<uint32_t>(hmax + 1));
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  if (H == 0) return VR_OK;
  if (hoff_host) {
    for (int64_t i = 0; i < H; ++i) {
      k_halo_frame<<<1, kFrameT, 0, s>>>(g.hoff, g.hlabel, g.horder, i, i + 1, g.v, p->nsearch_min,
                                         halo_stats);
      VR_LAUNCHED(ctx, "k_halo_frame");
    }
  } else {
    vr_status st = run_halo_frame(ctx, g, p->nsearch_min, halo_stats, s);
    if (st != VR_OK) return st;
  }
  k_node_caps<<<grid_for(H + 1, 256), 256, 0, s>>>(g.hoff, H, p->nsearch_min, p->f_cell,
                                                   p->ncell_min, bg.nodeoff);
  VR_LAUNCHED(ctx, "k_node_caps");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(bg.nodeoff, bg.nodeoff, H + 1, scr, s));
  const size_t smem_big = sizeof(WarpTree) * (kBigT / 32), smem_small = sizeof(WarpTree) * (kSmallT / 32);
  VR_CUDA(ctx, cudaFuncSetAttribute(k_cells_build<kBigT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big));
  VR_CUDA(ctx, cudaFuncSetAttribute(k_cells_build<kSmallT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_small));
  auto build = [&](bool bigc, cudaStream_t st, int64_t a, int64_t z, unsigned grid) {
    if (bigc)
      k_cells_build<kBigT><<<grid, kBigT, smem_big, st>>>(g.hoff, g.horder, bg.nodeoff, a, z, g.u, g.v,
                                                   p->nsearch_min, p->f_cell, p->ncell_min,
                                                   p->split_rule, perm, tmp, bg.nodes, bg.mom,
                                                   bg.leaf_of, halo_stats, ctx->d_status);
    else
      k_cells_build<kSmallT><<<grid, kSmallT, smem_small, st>>>(g.hoff, g.horder, bg.nodeoff, a, z, g.u,
                                                       g.v, p->nsearch_min, p->f_cell,
                                                       p->ncell_min, p->split_rule, perm, tmp,
                                                       bg.nodes, bg.mom, bg.leaf_of, halo_stats,
                                                       ctx->d_status);
  };
  unsigned long long *ndeg = (unsigned long long *)&ctx->d_status->info[0];
  if (hoff_host) {
    // one launch per searched halo, in the size order, with the CTA size of its class
    std::vector<uint32_t> ord(H);
    VR_CUDA(ctx, cudaMemcpyAsync(ord.data(), g.horder, H * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < H; ++i) {
      const int64_t nh = hoff_host[ord[i] + 1] - hoff_host[ord[i]];
      if (nh < p->nsearch_min) continue;
      build(nh >= kBigHalo, s, i, i + 1, 1);
      VR_LAUNCHED(ctx, nh >= kBigHalo ? "k_cells_build<big>" : "k_cells_build");
    }
    for (int64_t h = 0; h < H; ++h) {
      const int64_t a = hoff_host[h], z = hoff_host[h + 1];
      if (z - a < p->nsearch_min) continue;
      k_ratio<<<grid_for(z - a, 256), 256, 0, s>>>(g.hid, bg.nodeoff, a, z, g.u, g.v, f_l, bg.nodes,
                                                  bg.mom, bg.leaf_of, R, ndeg, g.hoff, 0u,
                                                  0xffffffffu);
      VR_LAUNCHED(ctx, "k_ratio");
    }
    return VR_OK;
  }
  // Halos of kBigHalo members or more (the first entries of the size order) run with
  // 1024-thread CTAs on the context's side stream while all other halos run with
  // 256-thread CTAs on stream s; the two launches overlap.
  const int64_t nbig_max = g.NHP / kBigHalo + 1;
  const unsigned big_grid = (unsigned)(nbig_max < H ? nbig_max : H);
  VR_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
  VR_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  VR_TIMED(ctx, "cells_build_big", ctx->side, build(true, ctx->side, 0, H, big_grid));
  VR_LAUNCHED(ctx, "k_cells_build<big>");
  VR_TIMED(ctx, "cells_build", s, build(false, s, 0, H, (unsigned)H));
  VR_LAUNCHED(ctx, "k_cells_build");
  VR_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
  VR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
  if (f_l) return background_ratio(ctx, g, bg, f_l, R, s);
  return VR_OK;
}

vr_status background_ratio(vr_ctx *ctx, const HaloSeg &g, const Background &bg, const float *f_l,
                           float *R, cudaStream_t s, uint32_t szlo, uint32_t szhi) {
  if (g.H == 0) return VR_OK;
  unsigned long long *ndeg = (unsigned long long *)&ctx->d_status->info[0];
  VR_TIMED(ctx, "ratio", s, k_ratio<<<grid_for(g.NHP, 256), 256, 0, s>>>(g.hid, bg.nodeoff, 0, g.NHP, g.u, g.v, f_l, bg.nodes,
                                               bg.mom, bg.leaf_of, R, ndeg, g.hoff, szlo, szhi));
  VR_LAUNCHED(ctx, "k_ratio");
  return VR_OK;
}

}  // namespace vr
