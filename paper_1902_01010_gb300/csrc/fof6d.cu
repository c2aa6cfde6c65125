// Phase-space linking of outliers (Sec. 2.2, Eq. linkingcriteria; with use_lv the
// velocity term of Eq. fof6d is added).
//
// The same linker serves the field 6DFOF of Sec. 2.1 (Eq. fof6d): every halo member is a
// candidate, lx is the 3D linking length and lv = alpha_v sigma_v per halo.
//
// GB300 design: candidates (ell >= ell_th, or all members) are compacted per halo in the
// halo's Morton order, so 32 consecutive candidates form a compact "tile" with an integer
// bounding box. One warp owns one tile and walks the later tiles of its halo, 32 box
// tests at a time across the lanes: a box gap of at least the spatial linking length
// skips a tile pair outright; otherwise the 32 x 32 pairs are tested from shared memory. The predicate is FP64 with every operation rounded
// explicitly (no fused multiply-add), in the fixed order stated in vr.h, so it decides
// exactly as an FP64 reference fed the same inputs. Linked pairs are merged by the
// lock-free union-find; labels are the minimum particle index of each group, and groups
// smaller than N_min get -1.
#include <math.h>

#include <vector>

#include "halos.cuh"
#include "vr_workspace.h"
#include "unionfind.cuh"

namespace vr {

namespace {

__global__ void k_cand_flags(const uint32_t *__restrict__ hid, int64_t nhp,
                             const float4 *__restrict__ v, const float *__restrict__ ell,
                             const double *__restrict__ hp, int64_t nhalo, double ell_th,
                             uint32_t *__restrict__ flag) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m > nhp) return;
  if (m == nhp) {
    flag[nhp] = 0;
    return;
  }
  uint32_t h = hid[m];
  bool c = h < (uint64_t)nhalo && hp[(int64_t)h * VR_HALO_COLS + VR_H_SEARCHED] != 0.0;
  if (c && ell) {
    float e = ell[__float_as_int(v[m].w)];
    c = (double)e >= ell_th;  // false for NaN
  }
  flag[m] = c ? 1u : 0u;
}

__global__ void k_cand_compact(const uint32_t *__restrict__ flag_scan, const uint32_t *__restrict__ hid,
                               int64_t nhp, const int4 *__restrict__ u, const float4 *__restrict__ v,
                               int4 *__restrict__ cu, float4 *__restrict__ cv,
                               uint32_t *__restrict__ chid) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  uint32_t a = flag_scan[m], b = flag_scan[m + 1];
  if (b == a) return;
  cu[a] = u[m];
  cv[a] = v[m];
  chid[a] = hid[m];
}

// Per halo: first candidate (coff), number of tiles (into toff before its scan).
__global__ void k_cand_halos(const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ flag_scan,
                             int64_t H, uint32_t *__restrict__ coff, uint32_t *__restrict__ toff) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h > H) return;
  uint32_t c0 = flag_scan[hoff[h]];
  coff[h] = c0;
  if (h == H) {
    toff[H] = 0;
    return;
  }
  uint32_t c1 = flag_scan[hoff[h + 1]];
  toff[h] = (c1 - c0 + 31) / 32;
}

__global__ void k_tile_fill(const uint32_t *__restrict__ toff, int64_t H, uint32_t *__restrict__ thalo) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  for (uint32_t k = toff[h]; k < toff[h + 1]; ++k) thalo[k] = (uint32_t)h;
}

__global__ void k_tile_boxes(const uint32_t *__restrict__ toff, const uint32_t *__restrict__ coff,
                             const uint32_t *__restrict__ thalo, int64_t ntiles,
                             const int4 *__restrict__ cu, int4 *__restrict__ tmin,
                             int4 *__restrict__ tmax) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ntiles) return;
  uint32_t h = thalo[k];
  uint32_t c0 = coff[h] + 32u * ((uint32_t)k - toff[h]), c1 = min(c0 + 32u, coff[h + 1]);
  int4 lo = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0);
  int4 hi = make_int4(-0x7fffffff, -0x7fffffff, -0x7fffffff, 0);
  for (uint32_t c = c0; c < c1; ++c) {
    int4 p = cu[c];
    lo.x = min(lo.x, p.x); lo.y = min(lo.y, p.y); lo.z = min(lo.z, p.z);
    hi.x = max(hi.x, p.x); hi.y = max(hi.y, p.y); hi.z = max(hi.z, p.z);
  }
  tmin[k] = lo;
  tmax[k] = hi;
}

__device__ __forceinline__ long long gap1(int alo, int ahi, int blo, int bhi) {
  if (blo > ahi) return (long long)blo - ahi;
  if (alo > bhi) return (long long)alo - bhi;
  return 0;
}

struct Link6 {
  double lx2, lv2, vf0, vf1, vf2, vr2, cos2;
  int use_lv, use_vt;
};

// The link predicate, evaluated in the fixed order stated in vr.h with explicit
// rounding of every FP64 operation.
__device__ __forceinline__ bool link6(long long dx2, float4 a, float4 b, const Link6 &L) {
  double q = __ddiv_rn((double)dx2, L.lx2);
  if (L.use_lv) {
    double d0 = __dsub_rn((double)a.x, (double)b.x), d1 = __dsub_rn((double)a.y, (double)b.y),
           d2 = __dsub_rn((double)a.z, (double)b.z);
    double dv2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    q = __dadd_rn(q, __ddiv_rn(dv2, L.lv2));
  }
  if (!(q < 1.0)) return false;
  if (L.use_vt) {
    double ui0 = __dsub_rn((double)a.x, L.vf0), ui1 = __dsub_rn((double)a.y, L.vf1),
           ui2 = __dsub_rn((double)a.z, L.vf2);
    double uj0 = __dsub_rn((double)b.x, L.vf0), uj1 = __dsub_rn((double)b.y, L.vf1),
           uj2 = __dsub_rn((double)b.z, L.vf2);
    double si = __dadd_rn(__dadd_rn(__dmul_rn(ui0, ui0), __dmul_rn(ui1, ui1)), __dmul_rn(ui2, ui2));
    double sj = __dadd_rn(__dadd_rn(__dmul_rn(uj0, uj0), __dmul_rn(uj1, uj1)), __dmul_rn(uj2, uj2));
    if (!(si > 0.0 && sj > 0.0)) return false;
    if (!(si <= __dmul_rn(L.vr2, sj) && sj <= __dmul_rn(L.vr2, si))) return false;
    double dot = __dadd_rn(__dadd_rn(__dmul_rn(ui0, uj0), __dmul_rn(ui1, uj1)), __dmul_rn(ui2, uj2));
    if (!(dot >= 0.0)) return false;
    if (!(__dmul_rn(dot, dot) >= __dmul_rn(__dmul_rn(L.cos2, si), sj))) return false;
  }
  return true;
}

// One warp per tile i: pairs with every later tile of the same halo (and inside tile i).
// The lanes test the boxes of 32 later tiles at once; each tile that comes within the
// spatial linking length is staged in shared memory and its 32 members are read back by
// every lane. The predicate is first evaluated in FP32 with every operand a rounded copy
// of the FP64 one: its relative error is below 8 * 2^-24 < 5e-7, so a result outside
// [1 - 1e-5, 1 + 1e-5] decides the FP64 comparison too; pairs inside that band, and every
// pair when V_r / Theta_op are on, take the exact FP64 path. The FP32 route is used only
// when lx2 and lv2 are normal FP32 numbers.
__global__ void __launch_bounds__(128) k_link6(const uint32_t *__restrict__ toff,
                                               const uint32_t *__restrict__ coff,
                                               const uint32_t *__restrict__ thalo, int64_t t0,
                                               int64_t t1, const int4 *__restrict__ cu,
                                               const float4 *__restrict__ cv,
                                               const int4 *__restrict__ tmin,
                                               const int4 *__restrict__ tmax,
                                               const double *__restrict__ hp, double vr2,
                                               double cos2, int use_lv, int use_vt, int *parent) {
  __shared__ int4 s_u[4][32];
  __shared__ float4 s_v[4][32];
  __shared__ int s_r[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t ti = t0 + (int64_t)blockIdx.x * (blockDim.x / 32) + w;  // tiles [t0, t1)
  if (ti >= t1) return;
  const uint32_t h = thalo[ti];
  const double *row = hp + (int64_t)h * VR_HALO_COLS;
  Link6 L;
  L.lx2 = row[VR_H_LX2];
  L.lv2 = row[VR_H_LV2];
  L.vf0 = row[VR_H_VFX];
  L.vf1 = row[VR_H_VFY];
  L.vf2 = row[VR_H_VFZ];
  L.vr2 = vr2;
  L.cos2 = cos2;
  L.use_lv = use_lv;
  L.use_vt = use_vt;
  const bool fast = L.lx2 > 1e-30 && L.lx2 < 1e30 && (!use_lv || (L.lv2 > 1e-30 && L.lv2 < 1e30));
  const float ilx2 = fast ? (float)(1.0 / L.lx2) : 0.0f;
  const float ilv2 = fast && use_lv ? (float)(1.0 / L.lv2) : 0.0f;
  const uint32_t c0h = coff[h], c1h = coff[h + 1], th0 = toff[h], th1 = toff[h + 1];
  const uint32_t ia = c0h + 32u * ((uint32_t)ti - th0);
  const uint32_t na = min(32u, c1h - ia);
  const bool va = (uint32_t)lane < na;
  const int4 pa = cu[va ? ia + lane : ia];
  const float4 qa = cv[va ? ia + lane : ia];
  const int4 alo = tmin[ti], ahi = tmax[ti];
  // the spatial term alone must be < 1: dx2 < lx2
  for (uint32_t base = (uint32_t)ti; base < th1; base += 32) {
    const uint32_t tj = base + lane;
    bool hit = false;
    if (tj < th1) {
      const int4 blo = tmin[tj], bhi = tmax[tj];
      const long long gx = gap1(alo.x, ahi.x, blo.x, bhi.x), gy = gap1(alo.y, ahi.y, blo.y, bhi.y),
                      gz = gap1(alo.z, ahi.z, blo.z, bhi.z);
      hit = (double)(gx * gx + gy * gy + gz * gz) < L.lx2;
    }
    unsigned hm = __ballot_sync(FULL, hit);
    while (hm) {
      const uint32_t tb = base + (uint32_t)(__ffs(hm) - 1);
      hm &= hm - 1;
      const uint32_t ib = c0h + 32u * (tb - th0);
      const uint32_t nbb = min(32u, c1h - ib);
      __syncwarp();
      // current roots of both tiles' members: a tile pair whose members all share one set
      // has nothing left to link (sets only ever merge, so an equal pair of roots, even
      // stale ones, proves the two members connected)
      const int ra = va ? uf_find(parent, (int)(ia + lane)) : -1;
      const int rb = (uint32_t)lane < nbb ? uf_find(parent, (int)(ib + lane)) : -1;
      if ((uint32_t)lane < nbb) {
        s_u[w][lane] = cu[ib + lane];
        s_v[w][lane] = cv[ib + lane];
        s_r[w][lane] = rb;
      }
      const int r0 = __shfl_sync(FULL, ra, 0);
      if (__all_sync(FULL, (!va || ra == r0) && ((uint32_t)lane >= nbb || rb == r0))) continue;
      __syncwarp();
      if (!va) continue;
      int rk = ra;  // a member of this lane's set, for the connected-pair skip below
      for (uint32_t k = tb == (uint32_t)ti ? (uint32_t)lane + 1 : 0; k < nbb; ++k) {
        const int4 p = s_u[w][k];
        const float4 q = s_v[w][k];
        const long long dx = (long long)pa.x - p.x, dy = (long long)pa.y - p.y,
                        dz = (long long)pa.z - p.z;
        const long long dx2 = dx * dx + dy * dy + dz * dz;
        // exact pre-test: dx2 >= lx2 gives dx2 / lx2 >= 1 after rounding, so q >= 1
        if ((double)dx2 >= L.lx2) continue;
        bool link;
        if (fast) {
          float qf = (float)dx2 * ilx2;
          if (use_lv) {
            const float d0 = qa.x - q.x, d1 = qa.y - q.y, d2 = qa.z - q.z;
            qf += ((d0 * d0 + d1 * d1) + d2 * d2) * ilv2;
          }
          if (qf >= 1.0f + 1e-5f) continue;  // also +inf; NaN falls through to FP64
          link = (qf <= 1.0f - 1e-5f && !use_vt) ? true : link6(dx2, qa, q, L);
        } else {
          link = link6(dx2, qa, q, L);
        }
        if (link && s_r[w][k] != rk) {
          uf_unite(parent, (int)(ia + lane), (int)(ib + k));
          rk = min(rk, s_r[w][k]);  // now in this lane's set
        }
      }
    }
  }
}

// Field halos (Eq. fof6d): lx2 and lv2 = (alpha_v sigma_v)^2 for every halo, and every
// halo marked for linking.
__global__ void k_field_lengths(int64_t H, double lx2, double alpha_v, double *__restrict__ hs) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  double *row = hs + h * VR_HALO_COLS;
  const double lv = alpha_v * row[VR_H_SIGMA];
  row[VR_H_LX2] = lx2;
  row[VR_H_LV2] = lv * lv;
  row[VR_H_SEARCHED] = 1.0;
}

__global__ void k_cand_init(int64_t nc, int *__restrict__ parent, int *__restrict__ minidx,
                            int *__restrict__ size) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  parent[c] = (int)c;
  minidx[c] = 0x7fffffff;
  size[c] = 0;
}

__global__ void k_cand_roots(int *parent, const float4 *__restrict__ cv, int64_t nc,
                             int *__restrict__ minidx, int *__restrict__ size) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int r = uf_find(parent, (int)c);
  atomicMin(&minidx[r], __float_as_int(cv[c].w));
  atomicAdd(&size[r], 1);
}

__global__ void k_cand_label(int *parent, const float4 *__restrict__ cv, int64_t nc,
                             const int *__restrict__ minidx, const int *__restrict__ size,
                             int nmin, int32_t *__restrict__ label6) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int r = uf_find(parent, (int)c);
  label6[__float_as_int(cv[c].w)] = size[r] >= nmin ? minidx[r] : -1;
}

__global__ void k_fill_i32(int32_t *__restrict__ a, int64_t n, int32_t val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = val;
}

}  // namespace

size_t fof6d_bytes(int64_t n, int nmin) {
  Arena ar;
  int64_t hmax = n / (nmin > 0 ? nmin : 1) + 2;
  int64_t tmaxn = n / 32 + hmax + 2;
  ar.take<uint32_t>(n + 1);  // flag scan
  ar.take<int4>(n);          // cu
  ar.take<float4>(n);        // cv
  ar.take<uint32_t>(n);      // chid
  ar.take<uint32_t>(hmax + 1);  // coff
  ar.take<uint32_t>(hmax + 1);  // toff
  ar.take<uint32_t>(tmaxn);     // thalo
  ar.take<int4>(tmaxn);
  ar.take<int4>(tmaxn);
  ar.take<int>(n);  // parent
  ar.take<int>(n);  // minidx
  ar.take<int>(n);  // size
  size_t a = scan_scratch_bytes<uint32_t>(n + 1);
  ar.take<char>(a);
  return ar.off;
}

vr_status field_lengths(vr_ctx *ctx, int64_t H, double lx2, double alpha_v, double *hs,
                        cudaStream_t s) {
  if (H == 0) return VR_OK;
  k_field_lengths<<<grid_for(H, 256), 256, 0, s>>>(H, lx2, alpha_v, hs);
  VR_LAUNCHED(ctx, "k_field_lengths");
  return VR_OK;
}

vr_status fill_i32(vr_ctx *ctx, int32_t *a, int64_t n, int32_t val, cudaStream_t s) {
  k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(a, n, val);
  VR_LAUNCHED(ctx, "k_fill_i32");
  return VR_OK;
}

vr_status run_fof6d(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar,
                    const float *ell, const double *hp, int64_t nhalo, int32_t *label6,
                    cudaStream_t s, bool plain) {
  if (g.H == 0) return VR_OK;
  const int64_t H = g.H, nhp = g.NHP;
  int64_t hmax = g.n / (p->nmin > 0 ? p->nmin : 1) + 2;
  int64_t tmaxn = g.n / 32 + hmax + 2;
  uint32_t *flag = ar.take<uint32_t>(g.n + 1);
  int4 *cu = ar.take<int4>(g.n);
  float4 *cv = ar.take<float4>(g.n);
  uint32_t *chid = ar.take<uint32_t>(g.n);
  uint32_t *coff = ar.take<uint32_t>(hmax + 1);
  uint32_t *toff = ar.take<uint32_t>(hmax + 1);
  uint32_t *thalo = ar.take<uint32_t>(tmaxn);
  int4 *tmin = ar.take<int4>(tmaxn);
  int4 *tmax = ar.take<int4>(tmaxn);
  int *parent = ar.take<int>(g.n);
  int *minidx = ar.take<int>(g.n);
  int *size = ar.take<int>(g.n);
  void *scr = ar.take<char>(scan_scratch_bytes<uint32_t>(g.n + 1));
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int T = 256;
  k_cand_flags<<<grid_for(nhp + 1, T), T, 0, s>>>(g.hid, nhp, g.v, ell, hp, nhalo, p->ell_th, flag);
  VR_LAUNCHED(ctx, "k_cand_flags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(flag, flag, nhp + 1, scr, s));
  k_cand_compact<<<grid_for(nhp, T), T, 0, s>>>(flag, g.hid, nhp, g.u, g.v, cu, cv, chid);
  VR_LAUNCHED(ctx, "k_cand_compact");
  k_cand_halos<<<grid_for(H + 1, T), T, 0, s>>>(g.hoff, flag, H, coff, toff);
  VR_LAUNCHED(ctx, "k_cand_halos");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(toff, toff, H + 1, scr, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 35, flag + nhp, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 36, toff + H, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  uint32_t nc = 0, ntiles = 0;
  memcpy(&nc, ctx->h_pinned + 35, 4);
  memcpy(&ntiles, ctx->h_pinned + 36, 4);
  if (nc == 0) return VR_OK;
  k_tile_fill<<<grid_for(H, T), T, 0, s>>>(toff, H, thalo);
  VR_LAUNCHED(ctx, "k_tile_fill");
  k_tile_boxes<<<grid_for(ntiles, T), T, 0, s>>>(toff, coff, thalo, ntiles, cu, tmin, tmax);
  VR_LAUNCHED(ctx, "k_tile_boxes");
  k_cand_init<<<grid_for(nc, T), T, 0, s>>>(nc, parent, minidx, size);
  VR_LAUNCHED(ctx, "k_cand_init");
  const double vr2 = p->v_ratio * p->v_ratio;
  const double ct = cos(p->theta_op);
  const double cos2 = ct * ct;
  if (plain) {  // one launch per halo
    std::vector<uint32_t> th(H + 1);
    VR_CUDA(ctx, cudaMemcpyAsync(th.data(), toff, (H + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t h = 0; h < H; ++h) {
      if (th[h + 1] == th[h]) continue;
      k_link6<<<grid_for(th[h + 1] - th[h], 4), 128, 0, s>>>(toff, coff, thalo, th[h], th[h + 1], cu,
                                                              cv, tmin, tmax, hp, vr2, cos2,
                                                              p->use_lv, p->use_vr_theta, parent);
      VR_LAUNCHED(ctx, "k_link6");
    }
  } else {
    VR_TIMED(ctx, "link6", s, k_link6<<<grid_for(ntiles, 4), 128, 0, s>>>(toff, coff, thalo, 0, ntiles, cu, cv, tmin,
                                                                       tmax, hp, vr2, cos2, p->use_lv,
                                                                       p->use_vr_theta, parent));
    VR_LAUNCHED(ctx, "k_link6");
  }
  k_cand_roots<<<grid_for(nc, T), T, 0, s>>>(parent, cv, nc, minidx, size);
  VR_LAUNCHED(ctx, "k_cand_roots");
  k_cand_label<<<grid_for(nc, T), T, 0, s>>>(parent, cv, nc, minidx, size, p->nmin, label6);
  VR_LAUNCHED(ctx, "k_cand_label");
  (void)chid;
  return VR_OK;
}

}  // namespace vr
