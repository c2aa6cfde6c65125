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

#include "stages.h"
#include "tuning.cuh"
#include "vr_workspace.h"
#include "unionfind.cuh"

namespace vr {

namespace {

// Candidates: members of linked halos with ell >= ell_th (every member when ell is NULL),
// and every member already in a group when `tag` is given.
__global__ void k_cand_flags(const uint32_t *__restrict__ hid, int64_t nhp,
                             const float4 *__restrict__ v, const float *__restrict__ ell,
                             const double *__restrict__ hp, int64_t nhalo, double ell_th,
                             const int32_t *__restrict__ tag, const uint8_t *__restrict__ mask,
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
    const int pi = __float_as_int(v[m].w);
    c = (double)ell[pi] >= ell_th || (tag && tag[pi] >= 0);  // false for NaN
  }
  if (c && mask) c = mask[__float_as_int(v[m].w)] != 0;
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
//
// The same walk serves the relaxed pass of the two-stage linking (MODE > 0, lx2 scaled
// by gamma_x^2): MODE 1 unites linked pairs of untagged candidates, MODE 2 counts links
// between an untagged candidate's component and a tagged candidate's group, MODE 3
// counts links between candidates of two different grown groups (counts in a hash table
// keyed by the pair).
enum { kLink = 0, kUntagged = 1, kToGroup = 2, kCross = 3 };

struct GrowArgs {
  double gx;             // gamma_x
  const int *tag;        // [nc] stage-1 label of the candidate's particle, -1 untagged
  const int *croot;      // [nc] root of the candidate's untagged component
  const int *grown;      // [nc] grown group label, -1 none
  u64 *hkey;             // hash table keys (kEmptyKey = free)
  uint32_t *hcnt;        // hash table counts
  u64 hmask;             // capacity - 1 (a power of two)
  DevStatus *st;
};

constexpr u64 kEmptyKey = ~0ULL;

// Adds one to the count of `key` (open addressing, linear probing, bounded).
__device__ __forceinline__ void hash_add(const GrowArgs &G, u64 key) {
  const u64 h0 = (key * 0x9E3779B97F4A7C15ull) >> 16;
  for (u64 probe = 0; probe < 4096; ++probe) {
    const u64 i = (h0 + probe) & G.hmask;
    u64 k = __ldcg(G.hkey + i);
    if (k == kEmptyKey) k = atomicCAS((unsigned long long *)(G.hkey + i), kEmptyKey, key);
    if (k == kEmptyKey || k == key) {
      atomicAdd(G.hcnt + i, 1u);
      return;
    }
  }
  raise_error(G.st, VR_ERR_UNSUPPORTED, 5);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_link6(const uint32_t *__restrict__ toff,
                                               const uint32_t *__restrict__ coff,
                                               const uint32_t *__restrict__ thalo, int64_t t0,
                                               int64_t t1, const int4 *__restrict__ cu,
                                               const float4 *__restrict__ cv,
                                               const int4 *__restrict__ tmin,
                                               const int4 *__restrict__ tmax,
                                               const double *__restrict__ hp, double vr2,
                                               double cos2, int use_lv, int use_vt, int *parent,
                                               GrowArgs G) {
  __shared__ int4 s_u[8][32];  // one row per warp (up to 8 warps per block)
  __shared__ float4 s_v[8][32];
  __shared__ int s_r[8][32];
  __shared__ int s_x[8][32];
  __shared__ int s_y[8][32];
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
  if (MODE != kLink) L.lx2 = __dmul_rn(__dmul_rn(L.lx2, G.gx), G.gx);
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
  const int xa = MODE == kLink || !va ? -1 : (MODE == kCross ? G.grown[ia + lane] : G.tag[ia + lane]);
  const int ya = MODE == kToGroup && va ? G.croot[ia + lane] : -1;
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
      constexpr bool kUnion = MODE == kLink || MODE == kUntagged;
      const int ra = kUnion && va ? uf_find(parent, (int)(ia + lane)) : -1;
      const int rb = kUnion && (uint32_t)lane < nbb ? uf_find(parent, (int)(ib + lane)) : -1;
      if ((uint32_t)lane < nbb) {
        s_u[w][lane] = cu[ib + lane];
        s_v[w][lane] = cv[ib + lane];
        s_r[w][lane] = rb;
        if (MODE != kLink) s_x[w][lane] = MODE == kCross ? G.grown[ib + lane] : G.tag[ib + lane];
        if (MODE == kToGroup) s_y[w][lane] = G.croot[ib + lane];
      }
      if (kUnion) {
        const int r0 = __shfl_sync(FULL, ra, 0);
        if (__all_sync(FULL, (!va || ra == r0) && ((uint32_t)lane >= nbb || rb == r0))) continue;
      }
      __syncwarp();
      if (!va) continue;
      int rk = ra;  // a member of this lane's set, for the connected-pair skip below
      for (uint32_t k = tb == (uint32_t)ti ? (uint32_t)lane + 1 : 0; k < nbb; ++k) {
        // pairs this mode has no use for, before any arithmetic
        if (MODE == kUntagged && (xa >= 0 || s_x[w][k] >= 0)) continue;
        if (MODE == kToGroup && (xa < 0) == (s_x[w][k] < 0)) continue;
        if (MODE == kCross && (xa < 0 || s_x[w][k] < 0 || xa == s_x[w][k])) continue;
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
        if (!link) continue;
        if (kUnion) {
          if (s_r[w][k] != rk) {
            uf_unite(parent, (int)(ia + lane), (int)(ib + k));
            rk = min(rk, s_r[w][k]);  // now in this lane's set
          }
        } else if (MODE == kToGroup) {
          const u64 c = (u64)(uint32_t)(xa < 0 ? ya : s_y[w][k]);
          const u64 g = (u64)(uint32_t)(xa < 0 ? s_x[w][k] : xa);
          hash_add(G, (c << 32) | g);
        } else {
          const int b = s_x[w][k];
          hash_add(G, ((u64)(uint32_t)min(xa, b) << 32) | (u64)(uint32_t)max(xa, b));
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

// Hash table capacity for the two-stage counts: a power of two >= n / 2.
int64_t grow_table_cap(int64_t n) {
  int64_t c = 1024;
  while (c < n / 2) c <<= 1;
  return c;
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

namespace {

// Candidates compacted per halo in slot order, with their tiles and tile boxes.
struct Cands {
  uint32_t nc = 0, ntiles = 0;
  int4 *cu;
  float4 *cv;
  uint32_t *chid;  // halo of each candidate
  uint32_t *coff, *toff, *thalo;
  int4 *tmin, *tmax;
  int *parent, *minidx, *size;
};

vr_status prep_cands(vr_ctx *ctx, const HaloSeg &g, int nmin, Arena &ar, const float *ell,
                     double ell_thr, const int32_t *tag, const double *hp, int64_t nhalo,
                     cudaStream_t s, Cands *C, const uint8_t *mask = nullptr) {
  const int64_t H = g.H, nhp = g.NHP;
  int64_t hmax = g.n / (nmin > 0 ? nmin : 1) + 2;
  int64_t tmaxn = g.n / 32 + hmax + 2;
  uint32_t *flag = ar.take<uint32_t>(g.n + 1);
  C->cu = ar.take<int4>(g.n);
  C->cv = ar.take<float4>(g.n);
  uint32_t *chid = C->chid = ar.take<uint32_t>(g.n);
  C->coff = ar.take<uint32_t>(hmax + 1);
  C->toff = ar.take<uint32_t>(hmax + 1);
  C->thalo = ar.take<uint32_t>(tmaxn);
  C->tmin = ar.take<int4>(tmaxn);
  C->tmax = ar.take<int4>(tmaxn);
  C->parent = ar.take<int>(g.n);
  C->minidx = ar.take<int>(g.n);
  C->size = ar.take<int>(g.n);
  void *scr = ar.take<char>(scan_scratch_bytes<uint32_t>(g.n + 1));
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int T = 256;
  k_cand_flags<<<grid_for(nhp + 1, T), T, 0, s>>>(g.hid, nhp, g.v, ell, hp, nhalo, ell_thr, tag,
                                                  mask, flag);
  VR_LAUNCHED(ctx, "k_cand_flags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(flag, flag, nhp + 1, scr, s));
  k_cand_compact<<<grid_for(nhp, T), T, 0, s>>>(flag, g.hid, nhp, g.u, g.v, C->cu, C->cv, chid);
  VR_LAUNCHED(ctx, "k_cand_compact");
  k_cand_halos<<<grid_for(H + 1, T), T, 0, s>>>(g.hoff, flag, H, C->coff, C->toff);
  VR_LAUNCHED(ctx, "k_cand_halos");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(C->toff, C->toff, H + 1, scr, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 35, flag + nhp, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 36, C->toff + H, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  memcpy(&C->nc, ctx->h_pinned + 35, 4);
  memcpy(&C->ntiles, ctx->h_pinned + 36, 4);
  if (C->nc == 0) return VR_OK;
  k_tile_fill<<<grid_for(H, T), T, 0, s>>>(C->toff, H, C->thalo);
  VR_LAUNCHED(ctx, "k_tile_fill");
  k_tile_boxes<<<grid_for(C->ntiles, T), T, 0, s>>>(C->toff, C->coff, C->thalo, C->ntiles, C->cu,
                                                    C->tmin, C->tmax);
  VR_LAUNCHED(ctx, "k_tile_boxes");
  k_cand_init<<<grid_for(C->nc, T), T, 0, s>>>(C->nc, C->parent, C->minidx, C->size);
  VR_LAUNCHED(ctx, "k_cand_init");
  return VR_OK;
}

// ------------------------------------------------------- two-stage linking kernels

// Stage-1 label of each candidate and stage-1 group sizes (indexed by label).
__global__ void k_grow_tags(const float4 *__restrict__ cv, int64_t nc,
                            const int32_t *__restrict__ label6, int *__restrict__ tag,
                            int *__restrict__ n0) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int t = label6[__float_as_int(cv[c].w)];
  tag[c] = t;
  if (t >= 0) atomicAdd(&n0[t], 1);
}

__global__ void k_grow_roots(int *parent, int64_t nc, int *__restrict__ croot) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) croot[c] = uf_find(parent, (int)c);
}

__global__ void k_hash_clear(u64 *__restrict__ key, uint32_t *__restrict__ cnt, int64_t cap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap) return;
  key[i] = kEmptyKey;
  cnt[i] = 0;
}

// Per untagged component: the group with the most links (ties: the smaller label), as
// (count << 32 | ~label) maximised.
__global__ void k_grow_attach(const u64 *__restrict__ key, const uint32_t *__restrict__ cnt,
                              int64_t cap, unsigned long long *__restrict__ best) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || key[i] == kEmptyKey) return;
  const uint32_t c = (uint32_t)(key[i] >> 32), g = (uint32_t)key[i];
  atomicMax(&best[c], ((unsigned long long)cnt[i] << 32) | (unsigned long long)(~g));
}

__global__ void k_grow_label(const int *__restrict__ tag, const int *__restrict__ croot,
                             const unsigned long long *__restrict__ best, int64_t nc,
                             int *__restrict__ grown) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  if (tag[c] >= 0) {
    grown[c] = tag[c];
    return;
  }
  const unsigned long long b = best[croot[c]];
  grown[c] = b ? (int)(~(uint32_t)b) : -1;
}

__global__ void k_iota(int *__restrict__ a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int)i;
}

// Joins of grown groups A < B with more than f_merge N_o links between them (either).
__global__ void k_grow_merge(const u64 *__restrict__ key, const uint32_t *__restrict__ cnt,
                             int64_t cap, const int *__restrict__ n0, double f_merge, int *gpar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || key[i] == kEmptyKey) return;
  const int a = (int)(key[i] >> 32), b = (int)(uint32_t)key[i];
  const double c = (double)cnt[i];
  if (c > f_merge * (double)n0[a] || c > f_merge * (double)n0[b]) uf_unite(gpar, a, b);
}

__global__ void k_grow_min(int *gpar, const int *__restrict__ grown, const float4 *__restrict__ cv,
                           int64_t nc, int *__restrict__ minidx) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || grown[c] < 0) return;
  atomicMin(&minidx[uf_find(gpar, grown[c])], __float_as_int(cv[c].w));
}

__global__ void k_grow_out(int *gpar, const int *__restrict__ grown, const float4 *__restrict__ cv,
                           int64_t nc, const int *__restrict__ minidx, int32_t *__restrict__ label6) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || grown[c] < 0) return;
  label6[__float_as_int(cv[c].w)] = minidx[uf_find(gpar, grown[c])];
}

// ------------------------------------------------------------- core search kernels

// Initial background: members of halos of >= nsearch_min members outside substructure.
__global__ void k_core_init(const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ hid,
                            const float4 *__restrict__ v, int64_t nhp, int nsearch_min,
                            const int32_t *__restrict__ label6, uint8_t *__restrict__ mask) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const uint32_t h = hid[m];
  const int pi = __float_as_int(v[m].w);
  mask[pi] = (hoff[h + 1] - hoff[h] >= (uint32_t)nsearch_min && (!label6 || label6[pi] < 0)) ? 1 : 0;
}

// Loop l: lengths and thresholds of every halo still searching (Eq. coreloop, by repeated
// multiplication), written into the rows the linker reads.
__global__ void k_core_rows(int64_t H, const uint32_t *__restrict__ hoff, int l, double lx2,
                            double alpha_v, double av, double f_c, double an, int nsearch_min,
                            int *__restrict__ active, double *__restrict__ lv,
                            double *__restrict__ thr, unsigned long long *__restrict__ best,
                            double *__restrict__ hs) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  double *row = hs + h * VR_HALO_COLS;
  if (l == 0) {
    active[h] = hoff[h + 1] - hoff[h] >= (uint32_t)nsearch_min;
    lv[h] = alpha_v * row[VR_H_SIGMA];
    thr[h] = f_c * (double)(hoff[h + 1] - hoff[h]);
  } else {
    lv[h] = lv[h] * av;
    thr[h] = thr[h] * an;
  }
  best[h] = 0;
  row[VR_H_SEARCHED] = active[h] ? 1.0 : 0.0;
  row[VR_H_LX2] = lx2;
  row[VR_H_LV2] = lv[h] * lv[h];
}

__device__ __forceinline__ bool core_ok(int size, int nmin, double thr) {
  return size >= nmin && (double)size >= thr;
}

// The largest qualifying group of each halo: max of (size << 32 | ~label).
__global__ void k_core_best(int *parent, const uint32_t *__restrict__ chid, int64_t nc,
                            const int *__restrict__ minidx, const int *__restrict__ size, int nmin,
                            const double *__restrict__ thr, unsigned long long *__restrict__ best) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || uf_find(parent, (int)c) != (int)c) return;
  const uint32_t h = chid[c];
  if (!core_ok(size[c], nmin, thr[h])) return;
  atomicMax(&best[h], ((unsigned long long)(uint32_t)size[c] << 32) |
                          (unsigned long long)(~(uint32_t)minidx[c]));
}

// Members of the largest group stay in the background; members of other qualifying
// groups become cores of level l; the rest leave the background. Halos without a
// qualifying group keep their background (their last primary core).
__global__ void k_core_mark(int *parent, const uint32_t *__restrict__ chid,
                            const float4 *__restrict__ cv, int64_t nc,
                            const int *__restrict__ minidx, const int *__restrict__ size, int nmin,
                            const double *__restrict__ thr,
                            const unsigned long long *__restrict__ best, int l,
                            uint8_t *__restrict__ mask, int32_t *__restrict__ core,
                            int32_t *__restrict__ level, unsigned long long *__restrict__ ncores) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const uint32_t h = chid[c];
  const unsigned long long b = best[h];
  if (!b) return;
  const int r = uf_find(parent, (int)c);
  const int pi = __float_as_int(cv[c].w);
  if (!core_ok(size[r], nmin, thr[h])) {
    mask[pi] = 0;
    return;
  }
  const int lab = minidx[r];
  if ((uint32_t)lab == ~(uint32_t)b) return;  // the primary core
  mask[pi] = 0;
  core[pi] = lab;
  level[pi] = l;
  if (r == (int)c) atomicAdd(ncores, 1ull);
}

__global__ void k_core_halos(int64_t H, const unsigned long long *__restrict__ best, int l,
                             int *__restrict__ active, int *__restrict__ last,
                             int *__restrict__ prim) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H || !active[h]) return;
  if (!best[h]) {
    active[h] = 0;
    return;
  }
  last[h] = l;
  prim[h] = (int)(~(uint32_t)best[h]);
}

// Loop l: the members of a searching halo's background were searched at l.
__global__ void k_core_searched(const uint32_t *__restrict__ hid, const float4 *__restrict__ v,
                                int64_t nhp, const uint8_t *__restrict__ mask,
                                const int *__restrict__ active, int l,
                                int32_t *__restrict__ searched) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int pi = __float_as_int(v[m].w);
  if (mask[pi] && active[hid[m]]) searched[pi] = l;
}

// The last primary core of every halo that found one.
__global__ void k_core_final(const uint32_t *__restrict__ hid, const float4 *__restrict__ v,
                             int64_t nhp, const uint8_t *__restrict__ mask,
                             const int *__restrict__ last, const int *__restrict__ prim,
                             int32_t *__restrict__ core, int32_t *__restrict__ level) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const uint32_t h = hid[m];
  const int pi = __float_as_int(v[m].w);
  if (mask[pi] && last[h] >= 0) {
    core[pi] = prim[h];
    level[pi] = last[h];
  }
}

}  // namespace

vr_status run_fof6d(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar,
                    const float *ell, const double *hp, int64_t nhalo, int32_t *label6,
                    cudaStream_t s, bool plain) {
  if (g.H == 0) return VR_OK;
  const int64_t H = g.H;
  Cands C;
  vr_status st = prep_cands(ctx, g, p->nmin, ar, ell, p->ell_th, nullptr, hp, nhalo, s, &C);
  if (st != VR_OK || C.nc == 0) return st;
  const int T = 256;
  const double vr2 = p->v_ratio * p->v_ratio;
  const double ct = cos(p->theta_op);
  const double cos2 = ct * ct;
  GrowArgs G{};
  if (plain) {  // one launch per halo
    std::vector<uint32_t> th(H + 1);
    VR_CUDA(ctx, cudaMemcpyAsync(th.data(), C.toff, (H + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t h = 0; h < H; ++h) {
      if (th[h + 1] == th[h]) continue;
      k_link6<kLink><<<grid_for(th[h + 1] - th[h], 4), 128, 0, s>>>(
          C.toff, C.coff, C.thalo, th[h], th[h + 1], C.cu, C.cv, C.tmin, C.tmax, hp, vr2, cos2,
          p->use_lv, p->use_vr_theta, C.parent, G);
      VR_LAUNCHED(ctx, "k_link6");
    }
  } else {
    // tiles per block from the tuning state; a linker still to be tuned is run once per
    // candidate shape from fresh sets (same labels each time) and keeps the fastest
    auto link = [&](int sh) {
      const int w = kLWarps[sh];
      k_link6<kLink><<<grid_for(C.ntiles, w), 32 * w, 0, s>>>(
          C.toff, C.coff, C.thalo, 0, C.ntiles, C.cu, C.cv, C.tmin, C.tmax, hp, vr2, cos2,
          p->use_lv, p->use_vr_theta, C.parent, G);
    };
    if (lmeasure(ctx)) {
      Tuning *tn = ctx->tune;
      cudaEvent_t e0, e1;
      VR_CUDA(ctx, cudaEventCreate(&e0));
      VR_CUDA(ctx, cudaEventCreate(&e1));
      int best = 0;
      for (int sh = 0; sh < kNLShapes; ++sh) {
        if (sh > 0) {
          k_cand_init<<<grid_for(C.nc, T), T, 0, s>>>(C.nc, C.parent, C.minidx, C.size);
          VR_LAUNCHED(ctx, "k_cand_init");
        }
        VR_CUDA(ctx, cudaEventRecord(e0, s));
        link(sh);
        VR_LAUNCHED(ctx, "k_link6");
        VR_CUDA(ctx, cudaEventRecord(e1, s));
        VR_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        VR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        tn->lms[sh] = ms;
        if (ms < tn->lms[best]) best = sh;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      tn->lshape = best;
      tn->ltuned = 1;
    } else {
      VR_TIMED(ctx, "link6", s, link(lshape_for(ctx)));
      VR_LAUNCHED(ctx, "k_link6");
    }
  }
  k_cand_roots<<<grid_for(C.nc, T), T, 0, s>>>(C.parent, C.cv, C.nc, C.minidx, C.size);
  VR_LAUNCHED(ctx, "k_cand_roots");
  k_cand_label<<<grid_for(C.nc, T), T, 0, s>>>(C.parent, C.cv, C.nc, C.minidx, C.size, p->nmin, label6);
  VR_LAUNCHED(ctx, "k_cand_label");
  return VR_OK;
}

vr_status run_grow(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, const vr_grow_params *gp,
                   Arena &ar, const float *ell, const double *hp, int64_t nhalo, int32_t *label6,
                   cudaStream_t s) {
  if (g.H == 0) return VR_OK;
  Cands C;
  vr_status st = prep_cands(ctx, g, p->nmin, ar, ell, p->ell_th / gp->gamma_ell, label6, hp,
                            nhalo, s, &C);
  if (st != VR_OK) return st;
  const int64_t n = g.n, tcap = grow_table_cap(n);
  int *tag = ar.take<int>(n);
  int *croot = ar.take<int>(n);
  int *grown = ar.take<int>(n);
  unsigned long long *best = ar.take<unsigned long long>(n);
  int *n0 = ar.take<int>(n);
  int *gpar = ar.take<int>(n);
  int *minidx = ar.take<int>(n);
  u64 *hkey = ar.take<u64>(tcap);
  uint32_t *hcnt = ar.take<uint32_t>(tcap);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int64_t nc = C.nc;
  if (nc == 0) return VR_OK;
  int64_t cap = 1024;  // table in use: a power of two >= 2 nc
  while (cap < 2 * nc && cap < tcap) cap <<= 1;
  const int T = 256;
  VR_CUDA(ctx, cudaMemsetAsync(n0, 0, n * sizeof(int), s));
  VR_CUDA(ctx, cudaMemsetAsync(best, 0, nc * sizeof(unsigned long long), s));
  k_grow_tags<<<grid_for(nc, T), T, 0, s>>>(C.cv, nc, label6, tag, n0);
  VR_LAUNCHED(ctx, "k_grow_tags");
  const double vr = p->v_ratio * gp->gamma_vr, ct = cos(p->theta_op * gp->gamma_theta);
  const double vr2 = vr * vr, cos2 = ct * ct;
  GrowArgs G{gp->gamma_x, tag, croot, grown, hkey, hcnt, (u64)(cap - 1), ctx->d_status};
  auto pass = [&](auto kernel) {
    kernel<<<grid_for(C.ntiles, 4), 128, 0, s>>>(C.toff, C.coff, C.thalo, 0, C.ntiles, C.cu, C.cv,
                                                 C.tmin, C.tmax, hp, vr2, cos2, p->use_lv,
                                                 p->use_vr_theta, C.parent, G);
  };
  // 1. components of the untagged candidates
  pass(k_link6<kUntagged>);
  VR_LAUNCHED(ctx, "k_link6<untagged>");
  k_grow_roots<<<grid_for(nc, T), T, 0, s>>>(C.parent, nc, croot);
  VR_LAUNCHED(ctx, "k_grow_roots");
  // 2. links from components to groups; each component joins its most linked group
  k_hash_clear<<<grid_for(cap, T), T, 0, s>>>(hkey, hcnt, cap);
  VR_LAUNCHED(ctx, "k_hash_clear");
  pass(k_link6<kToGroup>);
  VR_LAUNCHED(ctx, "k_link6<to_group>");
  k_grow_attach<<<grid_for(cap, T), T, 0, s>>>(hkey, hcnt, cap, best);
  VR_LAUNCHED(ctx, "k_grow_attach");
  k_grow_label<<<grid_for(nc, T), T, 0, s>>>(tag, croot, best, nc, grown);
  VR_LAUNCHED(ctx, "k_grow_label");
  // 3. links between grown groups; joins above the merge threshold
  k_hash_clear<<<grid_for(cap, T), T, 0, s>>>(hkey, hcnt, cap);
  VR_LAUNCHED(ctx, "k_hash_clear");
  pass(k_link6<kCross>);
  VR_LAUNCHED(ctx, "k_link6<cross>");
  k_iota<<<grid_for(n, T), T, 0, s>>>(gpar, n);
  VR_LAUNCHED(ctx, "k_iota");
  k_grow_merge<<<grid_for(cap, T), T, 0, s>>>(hkey, hcnt, cap, n0, gp->f_merge, gpar);
  VR_LAUNCHED(ctx, "k_grow_merge");
  // 4. labels: minimum particle index of each final group
  k_fill_i32<<<grid_for(n, T), T, 0, s>>>(minidx, n, 0x7fffffff);
  VR_LAUNCHED(ctx, "k_fill_i32");
  k_grow_min<<<grid_for(nc, T), T, 0, s>>>(gpar, grown, C.cv, nc, minidx);
  VR_LAUNCHED(ctx, "k_grow_min");
  k_grow_out<<<grid_for(nc, T), T, 0, s>>>(gpar, grown, C.cv, nc, minidx, label6);
  VR_LAUNCHED(ctx, "k_grow_out");
  return VR_OK;
}

size_t grow_bytes(int64_t n, int nmin) {
  Arena ar;
  ar.off = fof6d_bytes(n, nmin);
  ar.take<int>(n);                 // tag
  ar.take<int>(n);                 // croot
  ar.take<int>(n);                 // grown
  ar.take<unsigned long long>(n);  // best
  ar.take<int>(n);                 // n0
  ar.take<int>(n);                 // gpar
  ar.take<int>(n);                 // minidx
  ar.take<u64>(grow_table_cap(n));
  ar.take<uint32_t>(grow_table_cap(n));
  return ar.off;
}

vr_status run_cores(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, const vr_core_params *cp,
                    double lx, double alpha_v, Arena &ar, const int32_t *label6, double *hs,
                    int32_t *core, int32_t *level, int64_t *ncores, cudaStream_t s,
                    CoreExtra *ex) {
  if (ncores) *ncores = 0;
  const int64_t H = g.H, n = g.n;
  uint8_t *mask = ar.take<uint8_t>(n);
  int *active = ar.take<int>(H + 1);
  int *last = ar.take<int>(H + 1);
  int *prim = ar.take<int>(H + 1);
  double *lv = ar.take<double>(H + 1);
  double *thr = ar.take<double>(H + 1);
  unsigned long long *best = ar.take<unsigned long long>(H + 1);
  unsigned long long *cnt = ar.take<unsigned long long>(1);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int T = 256;
  vr_status st0 = fill_i32(ctx, core, n, -1, s);
  if (st0 == VR_OK) st0 = fill_i32(ctx, level, n, -1, s);
  if (st0 == VR_OK && ex && ex->searched) st0 = fill_i32(ctx, ex->searched, n, -1, s);
  if (ex) {
    ex->prim = prim;
    ex->last = last;
  }
  if (st0 != VR_OK || H == 0) return st0;
  VR_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_fill_i32<<<grid_for(H, T), T, 0, s>>>(last, H, -1);
  VR_LAUNCHED(ctx, "k_fill_i32");
  k_core_init<<<grid_for(g.NHP, T), T, 0, s>>>(g.hoff, g.hid, g.v, g.NHP, p->nsearch_min, label6, mask);
  VR_LAUNCHED(ctx, "k_core_init");
  const size_t mark = ar.off;
  double lxl = lx;
  for (int l = 0; l < cp->n_loop; ++l) {
    if (l > 0) lxl = lxl * cp->alpha_x;
    k_core_rows<<<grid_for(H, T), T, 0, s>>>(H, g.hoff, l, lxl * lxl, alpha_v, cp->alpha_v,
                                              cp->f_c, cp->alpha_n, p->nsearch_min, active, lv,
                                              thr, best, hs);
    VR_LAUNCHED(ctx, "k_core_rows");
    if (ex && ex->searched) {
      k_core_searched<<<grid_for(g.NHP, T), T, 0, s>>>(g.hid, g.v, g.NHP, mask, active, l,
                                                        ex->searched);
      VR_LAUNCHED(ctx, "k_core_searched");
    }
    ar.off = mark;
    Cands C;
    vr_status st = prep_cands(ctx, g, p->nmin, ar, nullptr, 0.0, nullptr, hs, H, s, &C, mask);
    if (st != VR_OK) return st;
    if (C.nc == 0) break;
    GrowArgs G{};
    VR_TIMED(ctx, "core_link", s, k_link6<kLink><<<grid_for(C.ntiles, 4), 128, 0, s>>>(
        C.toff, C.coff, C.thalo, 0, C.ntiles, C.cu, C.cv, C.tmin, C.tmax, hs, 0.0, 0.0, 1, 0,
        C.parent, G));
    VR_LAUNCHED(ctx, "k_link6");
    k_cand_roots<<<grid_for(C.nc, T), T, 0, s>>>(C.parent, C.cv, C.nc, C.minidx, C.size);
    VR_LAUNCHED(ctx, "k_cand_roots");
    k_core_best<<<grid_for(C.nc, T), T, 0, s>>>(C.parent, C.chid, C.nc, C.minidx, C.size, p->nmin,
                                                 thr, best);
    VR_LAUNCHED(ctx, "k_core_best");
    k_core_mark<<<grid_for(C.nc, T), T, 0, s>>>(C.parent, C.chid, C.cv, C.nc, C.minidx, C.size,
                                                 p->nmin, thr, best, l, mask, core, level, cnt);
    VR_LAUNCHED(ctx, "k_core_mark");
    k_core_halos<<<grid_for(H, T), T, 0, s>>>(H, best, l, active, last, prim);
    VR_LAUNCHED(ctx, "k_core_halos");
  }
  k_core_final<<<grid_for(g.NHP, T), T, 0, s>>>(g.hid, g.v, g.NHP, mask, last, prim, core, level);
  VR_LAUNCHED(ctx, "k_core_final");
  // cores = candidate cores + one primary core per halo that found a group
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 40, cnt, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
  std::vector<int> lh(H);
  VR_CUDA(ctx, cudaMemcpyAsync(lh.data(), last, H * sizeof(int), cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  int64_t np = 0;
  for (int64_t h = 0; h < H; ++h) np += lh[h] >= 0;
  if (ncores) *ncores = (int64_t)ctx->h_pinned[40] + np;
  return VR_OK;
}

size_t cores_bytes(int64_t n, int nmin) {
  Arena ar;
  const int64_t hmax = n / (nmin > 0 ? nmin : 1) + 2;
  ar.take<uint8_t>(n);
  for (int k = 0; k < 3; ++k) ar.take<int>(hmax + 1);
  ar.take<double>(hmax + 1);
  ar.take<double>(hmax + 1);
  ar.take<unsigned long long>(hmax + 1);
  ar.take<unsigned long long>(1);
  return ar.off + fof6d_bytes(n, nmin) + 4096;
}

}  // namespace vr
