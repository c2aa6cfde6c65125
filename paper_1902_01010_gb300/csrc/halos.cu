// Halo segmentation: 3D labels -> halos (groups of >= N_min members, Sec. 2.2) with their
// members contiguous, unwrapped into one periodic image and Morton-ordered within the
// halo. Everything stays on the device except one read-back of the halo count.
#include "halos.cuh"
#include "vr_workspace.h"

namespace vr {

namespace {

constexpr uint32_t kMaxHalo = 1u << 22;

__global__ void k_count(const int32_t *__restrict__ label, int64_t n, uint32_t *__restrict__ cnt,
                        DevStatus *st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int32_t l = -1;
  if (i < n) {
    l = label[i];
    if (l < 0 || l >= n) {
      raise_error(st, VR_ERR_INVALID_ARG, 4);
      l = -1;
    }
  }
  // lanes with the same label add their count once (members of a group are often
  // neighbours in index order)
  const int32_t key = l >= 0 ? l : -1 - lane;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (l >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[l], (uint32_t)__popc(peers));
}

// flag[l] = 1 if label l heads a halo; halos larger than 2^22 are rejected.
__global__ void k_halo_flags(const uint32_t *__restrict__ cnt, int64_t n, int nmin,
                             uint32_t *__restrict__ flag, DevStatus *st) {
  int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l > n) return;
  if (l == n) {
    flag[n] = 0;
    return;
  }
  uint32_t c = cnt[l];
  flag[l] = (c > 0 && c >= (uint32_t)nmin) ? 1u : 0u;
  if (c > kMaxHalo) raise_error(st, VR_ERR_UNSUPPORTED, 1);
}

__global__ void k_member_flags(const int32_t *__restrict__ label, const uint32_t *__restrict__ cnt,
                               int64_t n, int nmin, uint32_t *__restrict__ mflag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    mflag[n] = 0;
    return;
  }
  uint32_t c = cnt[label[i]];
  mflag[i] = (c >= (uint32_t)nmin) ? 1u : 0u;
}

// Compacts halo members in index order with key = halo id.
__global__ void k_member_keys(const int32_t *__restrict__ label, const uint32_t *__restrict__ cnt,
                              const uint32_t *__restrict__ hidx, const uint32_t *__restrict__ mpos,
                              int64_t n, int nmin, uint32_t *__restrict__ keys,
                              uint32_t *__restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t l = label[i];
  if (cnt[l] < (uint32_t)nmin) return;
  uint32_t m = mpos[i];
  keys[m] = hidx[l];
  vals[m] = (uint32_t)i;
}

// Slots sorted by (halo, index): halo starts and labels, unwrapped positions, local
// index (rank by particle index inside the halo) and the halo bounding box.
__global__ void k_halo_bounds(const uint32_t *__restrict__ hkey, const uint32_t *__restrict__ idx,
                              int64_t nhp, uint32_t *__restrict__ hoff, uint32_t *__restrict__ hlabel) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  uint32_t h = hkey[m];
  if (m == 0 || hkey[m - 1] != h) {
    hoff[h] = (uint32_t)m;
    hlabel[h] = idx[m];  // first member in index order = minimum index = label
  }
  if (m == nhp - 1) hoff[h + 1] = (uint32_t)nhp;
}

__device__ __forceinline__ void warp_minmax_atomic(int *mn, int *mx, uint32_t key, int vmin,
                                                   int vmax) {
  // warp-aggregated when the whole warp belongs to one halo
  const unsigned full = 0xffffffffu;
  unsigned act = __activemask();
  uint32_t k0 = __shfl_sync(act, key, __ffs(act) - 1);
  bool same = __all_sync(act, key == k0) && act == full;
  if (same) {
    for (int o = 16; o; o >>= 1) {
      vmin = min(vmin, __shfl_xor_sync(full, vmin, o));
      vmax = max(vmax, __shfl_xor_sync(full, vmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(mn, vmin);
      atomicMax(mx, vmax);
    }
  } else {
    atomicMin(mn, vmin);
    atomicMax(mx, vmax);
  }
}

__global__ void k_unwrap(const int32_t *__restrict__ pos, const uint32_t *__restrict__ hkey,
                         const uint32_t *__restrict__ idx, const uint32_t *__restrict__ hoff,
                         const uint32_t *__restrict__ hlabel, int64_t nhp, int4 *__restrict__ u,
                         int *__restrict__ bmin, int *__restrict__ bmax) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = m < nhp;
  uint32_t h = ok ? hkey[m] : 0xffffffffu;
  int4 r = make_int4(0, 0, 0, 0);
  if (ok) {
    uint32_t i = idx[m], a = hlabel[h];
    const uint32_t lm = (uint32_t)kLattice - 1u;
    int ax = (int)((uint32_t)pos[3 * (int64_t)a] & lm), ay = (int)((uint32_t)pos[3 * (int64_t)a + 1] & lm),
        az = (int)((uint32_t)pos[3 * (int64_t)a + 2] & lm);
    int px = (int)((uint32_t)pos[3 * (int64_t)i] & lm), py = (int)((uint32_t)pos[3 * (int64_t)i + 1] & lm),
        pz = (int)((uint32_t)pos[3 * (int64_t)i + 2] & lm);
    r = make_int4(ax + min_image(px - ax), ay + min_image(py - ay), az + min_image(pz - az),
                  (int)((uint32_t)m - hoff[h]));
    u[m] = r;
  }
  if (__any_sync(0xffffffffu, ok)) {
    if (ok) {
      warp_minmax_atomic(&bmin[3 * (int64_t)h], &bmax[3 * (int64_t)h], h, r.x, r.x);
      warp_minmax_atomic(&bmin[3 * (int64_t)h + 1], &bmax[3 * (int64_t)h + 1], h, r.y, r.y);
      warp_minmax_atomic(&bmin[3 * (int64_t)h + 2], &bmax[3 * (int64_t)h + 2], h, r.z, r.z);
    }
  }
}

// Every member is unwrapped to within 2^20 of the halo's first member, which gives one
// consistent periodic image only when the halo spans less than half the box along each
// axis; an unwrapped extent of 2^20 or more means it does not (error site 1).
__global__ void k_halo_span(const int *__restrict__ bmin, const int *__restrict__ bmax, int64_t H,
                            DevStatus *st) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  for (int a = 0; a < 3; ++a)
    if ((long long)bmax[3 * h + a] - bmin[3 * h + a] >= kHalf) {
      raise_error(st, VR_ERR_UNSUPPORTED, 1);
      return;
    }
}

// key = halo id << 30 | 30-bit Morton code of the position scaled into the halo's
// bounding cube (10 bits per axis); value = slot in (halo, index) order.
__global__ void k_morton_keys(const int4 *__restrict__ u, const uint32_t *__restrict__ hkey,
                              const int *__restrict__ bmin, const int *__restrict__ bmax,
                              int64_t nhp, u64 *__restrict__ keys, uint32_t *__restrict__ vals) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  uint32_t h = hkey[m];
  int4 r = u[m];
  int64_t lo0 = bmin[3 * (int64_t)h], lo1 = bmin[3 * (int64_t)h + 1], lo2 = bmin[3 * (int64_t)h + 2];
  int64_t e = max(bmax[3 * (int64_t)h] - lo0, max(bmax[3 * (int64_t)h + 1] - lo1, bmax[3 * (int64_t)h + 2] - lo2)) + 1;
  uint32_t qx = (uint32_t)(((r.x - lo0) << 10) / e), qy = (uint32_t)(((r.y - lo1) << 10) / e),
           qz = (uint32_t)(((r.z - lo2) << 10) / e);
  keys[m] = ((u64)h << 30) | morton3(qx, qy, qz);
  vals[m] = (uint32_t)m;
}

__global__ void k_gather_morton(const uint32_t *__restrict__ perm, const int4 *__restrict__ u_in,
                                const uint32_t *__restrict__ idx_in, const uint32_t *__restrict__ hkey_in,
                                const float *__restrict__ vel, int64_t nhp, int4 *__restrict__ u_out,
                                float4 *__restrict__ v_out, uint32_t *__restrict__ hid_out) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  uint32_t src = perm[m];
  u_out[m] = u_in[src];
  uint32_t i = idx_in[src];
  v_out[m] = make_float4(vel[3 * (int64_t)i], vel[3 * (int64_t)i + 1], vel[3 * (int64_t)i + 2],
                         __int_as_float((int)i));
  hid_out[m] = hkey_in[src];
}

// keys that sort halos by decreasing size
__global__ void k_size_keys(const uint32_t *__restrict__ hoff, int64_t H, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
  int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  keys[h] = 0xffffffffu - (hoff[h + 1] - hoff[h]);
  vals[h] = (uint32_t)h;
}

int bitlen(uint64_t x) {
  int b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

struct SegBufs {
  uint32_t *cnt, *flag, *mflag;
  uint32_t *k0, *k1, *v0, *v1;
  u64 *mk0, *mk1;
  uint32_t *mv0, *mv1;
  int4 *u_idx;
  int *bmin, *bmax;
  void *scr;
};

SegBufs seg_carve(Arena &ar, int64_t n, int nmin) {
  int64_t hmax = n / (nmin > 0 ? nmin : 1) + 2;
  SegBufs b;
  b.cnt = ar.take<uint32_t>(n + 1);
  b.flag = ar.take<uint32_t>(n + 1);
  b.mflag = ar.take<uint32_t>(n + 1);
  b.k0 = ar.take<uint32_t>(n);
  b.k1 = ar.take<uint32_t>(n);
  b.v0 = ar.take<uint32_t>(n);
  b.v1 = ar.take<uint32_t>(n);
  b.mk0 = ar.take<u64>(n);
  b.mk1 = ar.take<u64>(n);
  b.mv0 = ar.take<uint32_t>(n);
  b.mv1 = ar.take<uint32_t>(n);
  b.u_idx = ar.take<int4>(n);
  b.bmin = ar.take<int>(3 * hmax);
  b.bmax = ar.take<int>(3 * hmax);
  size_t a = radix_scratch_bytes<u64>(n), c = scan_scratch_bytes<uint32_t>(n + 1);
  b.scr = ar.take<char>(a > c ? a : c);
  return b;
}

}  // namespace

// The segmentation's outputs, kept for the later stages.
static void seg_keep(Arena &ar, int64_t n, int nmin, HaloSeg *g) {
  int64_t hmax = n / (nmin > 0 ? nmin : 1) + 2;
  uint32_t *hoff = ar.take<uint32_t>(hmax + 1);
  uint32_t *hlabel = ar.take<uint32_t>(hmax);
  uint32_t *horder = ar.take<uint32_t>(hmax);
  uint32_t *hid = ar.take<uint32_t>(n);
  int4 *u = ar.take<int4>(n);
  float4 *v = ar.take<float4>(n);
  uint32_t *scr = ar.take<uint32_t>(n + 1);
  if (g) {
    g->hoff = hoff;
    g->hlabel = hlabel;
    g->horder = horder;
    g->hid = hid;
    g->u = u;
    g->v = v;
    g->scratch_u32_a = scr;
  }
}

size_t halo_seg_bytes(int64_t n, int nmin) {
  Arena ar;
  seg_keep(ar, n, nmin, nullptr);
  return ar.off;
}

size_t halo_seg_temp_bytes(int64_t n, int nmin) {
  Arena ar;
  seg_carve(ar, n, nmin);
  return ar.off + 256;
}

vr_status build_halos(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                      const int32_t *label, int nmin, int nsmall, Arena &ar, cudaStream_t s,
                      HaloSeg *out) {
  HaloSeg &g = *out;
  g.n = n;
  seg_keep(ar, n, nmin, &g);
  // the build buffers below are released when this call returns (later stages reuse them)
  const size_t keep = ar.off;
  SegBufs B = seg_carve(ar, n, nmin);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  struct Release {
    Arena &a;
    size_t off;
    ~Release() { a.off = off; }
  } release{ar, keep};
  const int T = 256;
  VR_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, (n + 1) * sizeof(uint32_t), s));
  k_count<<<grid_for(n, T), T, 0, s>>>(label, n, B.cnt, ctx->d_status);
  VR_LAUNCHED(ctx, "k_count");
  k_halo_flags<<<grid_for(n + 1, T), T, 0, s>>>(B.cnt, n, nmin, B.flag, ctx->d_status);
  VR_LAUNCHED(ctx, "k_halo_flags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(B.flag, B.flag, n + 1, B.scr, s));
  k_member_flags<<<grid_for(n + 1, T), T, 0, s>>>(label, B.cnt, n, nmin, B.mflag);
  VR_LAUNCHED(ctx, "k_member_flags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(B.mflag, B.mflag, n + 1, B.scr, s));
  // read H, NHP and the error word
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 32, B.flag + n, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 33, B.mflag + n, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  vr_status st = read_status(ctx, s, nullptr);
  if (st != VR_OK) return st;
  uint32_t H = 0, NHP = 0;
  memcpy(&H, ctx->h_pinned + 32, 4);
  memcpy(&NHP, ctx->h_pinned + 33, 4);
  g.H = H;
  g.NHP = NHP;
  if (H == 0) return VR_OK;
  k_member_keys<<<grid_for(n, T), T, 0, s>>>(label, B.cnt, B.flag, B.mflag, n, nmin, B.k0, B.v0);
  VR_LAUNCHED(ctx, "k_member_keys");
  int which = 0;
  VR_CUDA(ctx, radix_sort_pairs<uint32_t>(B.k0, B.v0, B.k1, B.v1, NHP, 0, bitlen(H), B.scr, s, &which));
  uint32_t *hkey = which ? B.k1 : B.k0;
  uint32_t *idx = which ? B.v1 : B.v0;
  k_halo_bounds<<<grid_for(NHP, T), T, 0, s>>>(hkey, idx, NHP, g.hoff, g.hlabel);
  VR_LAUNCHED(ctx, "k_halo_bounds");
  // bounding boxes: min starts at INT_MAX, max at INT_MIN
  VR_CUDA(ctx, cudaMemsetAsync(B.bmin, 0x7f, 3 * H * sizeof(int), s));
  VR_CUDA(ctx, cudaMemsetAsync(B.bmax, 0x80, 3 * H * sizeof(int), s));
  k_unwrap<<<grid_for(NHP, T), T, 0, s>>>(pos, hkey, idx, g.hoff, g.hlabel, NHP, B.u_idx, B.bmin, B.bmax);
  VR_LAUNCHED(ctx, "k_unwrap");
  k_halo_span<<<grid_for(H, T), T, 0, s>>>(B.bmin, B.bmax, H, ctx->d_status);
  VR_LAUNCHED(ctx, "k_halo_span");
  k_morton_keys<<<grid_for(NHP, T), T, 0, s>>>(B.u_idx, hkey, B.bmin, B.bmax, NHP, B.mk0, B.mv0);
  VR_LAUNCHED(ctx, "k_morton_keys");
  VR_CUDA(ctx, radix_sort_pairs<u64>(B.mk0, B.mv0, B.mk1, B.mv1, NHP, 0, 30 + bitlen(H), B.scr, s,
                                     &which));
  uint32_t *perm = which ? B.mv1 : B.mv0;
  k_gather_morton<<<grid_for(NHP, T), T, 0, s>>>(perm, B.u_idx, idx, hkey, vel, NHP, g.u, g.v, g.hid);
  VR_LAUNCHED(ctx, "k_gather_morton");
  // halo work order: decreasing size (the sort is stable, so equal sizes keep label order)
  k_size_keys<<<grid_for(H, T), T, 0, s>>>(g.hoff, H, B.k0, B.v0);
  VR_LAUNCHED(ctx, "k_size_keys");
  VR_CUDA(ctx, radix_sort_pairs<uint32_t>(B.k0, B.v0, B.k1, B.v1, H, 0, 32, B.scr, s, &which));
  VR_CUDA(ctx, cudaMemcpyAsync(g.horder, which ? B.v1 : B.v0, H * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, s));
  (void)nsmall;
  return VR_OK;
}

}  // namespace vr
