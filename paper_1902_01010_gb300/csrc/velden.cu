// Local velocity density f_l (Sec. 2.2): Epanechnikov estimate from the N_v nearest in
// velocity among the N_se nearest in position, inside each halo.
//
// GB300 design (no neighbour list is ever materialised):
//  - halo members are Morton-ordered inside their halo (halos.cu); each run of 32
//    consecutive members is a "bucket" with an integer bounding box, and 32 consecutive
//    buckets of one halo form a "super-bucket";
//  - one warp handles one bucket: lane k is the query particle k. Each lane first bounds
//    its N_se-th neighbour distance by the N_se-th smallest distance among the 4 N_se
//    members around the bucket in Morton order (to within one of 32 histogram bins);
//    every later pass visits only the buckets whose boxes come within the largest
//    per-lane bound of the warp's own box (super-bucket boxes prune first);
//  - each visited bucket is staged once in shared memory and read back by every lane
//    with broadcast 16-byte loads; every lane keeps its own 32-bin histogram of the exact
//    key (d^2 << 22 | local index). Histogram passes narrow the key range until the bin
//    holding the N_se-th key has at most 16 keys; a last pass feeds every key below that
//    bin, plus the right number from the bin, into a per-lane list of the N_v smallest
//    |dv|^2 (shared memory);
//  - h^2 is the largest kept |dv|^2, and the kernel sum runs over the kept list only
//    (every neighbour with |dv| < h is in it).
// Position keys are exact integers, so the N_se set equals the oracle's; velocity
// differences and sums are FP32. Squared separations are 64-bit integers, or 32-bit ones
// wherever the two boxes involved (query bucket and candidate bucket or window) bound
// every separation by 32767 lattice units per axis, which makes them exact in uint32.
// Halos with at most N_se members use every member (one pass, no position search).
#include <math.h>

#include <vector>

#include "halos.cuh"
#include "tuning.cuh"
#include "vr_workspace.h"

namespace vr {

namespace {

constexpr int kNVMax = 64;
constexpr int kBinBits = 6;      // histogram levels resolve kBinBits bits of the key
constexpr int kBins = 1 << kBinBits;
constexpr int kBuf = 32;
constexpr int kWarps = 4;        // warps per block

// Optional instrumentation (compile with -DVR_VELDEN_STATS): warp-level counts of the
// buckets staged per pass, kept in the status block's info[] words. Off in normal builds.
constexpr int kStatPass0 = 1;    // info[1 + pass]: 0 window, 1.. histogram levels, 7 collect
#ifdef VR_VELDEN_STATS
#define VR_STAT(st, slot, val) \
  do { if ((threadIdx.x & 31) == 0) atomicAdd((unsigned long long *)&(st)->info[(slot)], (unsigned long long)(val)); } while (0)
#else
#define VR_STAT(st, slot, val) do { } while (0)
#endif
constexpr int kWindow = 4;       // window of kWindow * N_se members for the first bound

// Per-warp shared memory. The key histogram is used only by the bound and histogram
// passes and the final-bin buffer only by the collect pass, so the two share storage.
template <int NVM>
struct WarpSmem {
  int4 su[32];
  float4 sv[32];
  union {
    uint16_t hist[kBins][32];
    uint32_t bslot[kBuf][32];  // member slots of the keys in the final bin
  };
  float top[NVM][32];
};

template <int NVM>
struct SmallSmem {
  float4 sv[32];
  float top[NVM][32];
};

// Per-lane list of the nv smallest values, kept as a binary max-heap in the lane's
// shared-memory column (top[0] is the largest kept value), with its size and maximum.
struct TopV {
  int c, im;
  float m;
};

// Offers v to the list: while fewer than nv values are kept, v is added (sifted up);
// after that v replaces the largest when it is smaller (sifted down from the root), so
// a replacement costs log2(nv) steps instead of a scan of all nv values.
__device__ __forceinline__ void top_insert(float (*top)[32], int lane, TopV &t, int nv, float v) {
  if (t.c < nv) {
    int i = t.c++;
    while (i > 0) {
      const int p = (i - 1) >> 1;
      const float pv = top[p][lane];
      if (pv >= v) break;
      top[i][lane] = pv;
      i = p;
    }
    top[i][lane] = v;
    t.m = top[0][lane];
  } else if (v < t.m) {
    int i = 0;
    for (;;) {
      const int l = 2 * i + 1;
      if (l >= nv) break;
      int ch = l;
      float cv = top[l][lane];
      if (l + 1 < nv) {
        const float rv = top[l + 1][lane];
        if (rv > cv) {
          ch = l + 1;
          cv = rv;
        }
      }
      if (cv <= v) break;
      top[i][lane] = cv;
      i = ch;
    }
    top[i][lane] = v;
    t.m = top[0][lane];
  }
}

// f_l from the kept list: h^2 = largest kept |dv|^2 (the N_v-th smallest);
// f_l = 15/(8 pi h^3) * sum_{|dv| < h} (1 - |dv|^2/h^2) / N_se_eff.
__device__ __forceinline__ float top_density(float (*top)[32], int lane, const TopV &t,
                                             int nse_eff) {
  float h2 = t.m;
  if (!(h2 > 0.0f)) return INFINITY;
  float inv = 1.0f / h2;
  float sum = 0.0f;
  for (int q = 0; q < t.c; ++q) {
    float x = top[q][lane];
    if (x < h2) sum += 1.0f - x * inv;
  }
  float h = sqrtf(h2);
  const float c = 15.0f / (8.0f * 3.14159265358979f);
  return c / (h2 * h) * sum / (float)nse_eff;
}

__device__ __forceinline__ float dv2f(float4 a, float4 b) {
  float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ long long d2i(int4 a, int4 b) {
  long long dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz;
}
// The same squared separation in 32-bit arithmetic, exact when every component of a - b
// lies in [-32767, 32767]: then d^2 < 3 * 2^30 < 2^32.
__device__ __forceinline__ uint32_t d2u(int4 a, int4 b) {
  const int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return (uint32_t)(dx * dx) + (uint32_t)(dy * dy) + (uint32_t)(dz * dz);
}

// True when every separation between a point of box A and a point of box B has all
// components in [-32767, 32767] (d2u is then exact for every such pair).
__device__ __forceinline__ bool fits32(int4 alo, int4 ahi, int4 blo, int4 bhi) {
  const int ex = max(ahi.x - blo.x, bhi.x - alo.x), ey = max(ahi.y - blo.y, bhi.y - alo.y),
            ez = max(ahi.z - blo.z, bhi.z - alo.z);
  return max(ex, max(ey, ez)) <= 32767;
}

__device__ __forceinline__ uint32_t clamp32(u64 x) { return x > 0xffffffffull ? 0xffffffffu : (uint32_t)x; }

// ---------------------------------------------------------------- small halos
template <int NVM>
__global__ void __launch_bounds__(32 * kWarps) k_velden_small(
    const uint32_t *__restrict__ hoff, int64_t h0, int64_t h1, const float4 *__restrict__ v,
    int nse, int nv, float *__restrict__ f_l) {
  __shared__ SmallSmem<NVM> sm[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t h = h0 + (int64_t)blockIdx.x * kWarps + w;  // halos [h0, h1)
  if (h >= h1) return;
  const uint32_t hs = hoff[h], he = hoff[h + 1];
  const int nh = (int)(he - hs);
  if (nh > nse) return;
  const int nv_eff = nv < nh ? nv : nh;
  float(*top)[32] = sm[w].top;
  for (uint32_t qb = hs; qb < he; qb += 32) {
    const uint32_t k = qb + lane;
    const bool valid = k < he;
    const float4 vq = v[valid ? k : hs];
    TopV t = {0, 0, 0.0f};
    for (uint32_t jb = hs; jb < he; jb += 32) {
      const uint32_t j = jb + lane;
      __syncwarp();
      if (j < he) sm[w].sv[lane] = v[j];
      __syncwarp();
      const int cnt = (int)min(32u, he - jb);
      if (valid)
        for (int tt = 0; tt < cnt; ++tt) top_insert(top, lane, t, nv_eff, dv2f(sm[w].sv[tt], vq));
    }
    if (valid) f_l[__float_as_int(vq.w)] = top_density(top, lane, t, nh);
  }
}

// ------------------------------------------------------------- bucket boxes
// Super-buckets are laid out halo by halo in the size order (largest first), so that the
// buckets of each halo-size bin form one contiguous range. Halo h owns super-buckets
// [sbs[h], sbe[h]); its bucket b (0-based) holds slots [hoff[h] + 32 b,
// min(hoff[h+1], hoff[h] + 32 b + 32)) and has the global index 32 sbs[h] + b.
__global__ void k_sb_count(const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ horder,
                           int64_t H, int nse, uint32_t *__restrict__ sbr) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > H) return;
  if (r == H) {
    sbr[H] = 0;
    return;
  }
  const uint32_t h = horder[r];
  uint32_t nh = hoff[h + 1] - hoff[h];
  uint32_t nb = (nh + 31) / 32;
  sbr[r] = nh > (uint32_t)nse ? (nb + 31) / 32 : 0;
}

__global__ void k_sb_fill(const uint32_t *__restrict__ sbr, const uint32_t *__restrict__ horder,
                          int64_t H, uint32_t *__restrict__ sbs, uint32_t *__restrict__ sbe,
                          uint32_t *__restrict__ sbhalo) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= H) return;
  const uint32_t h = horder[r];
  sbs[h] = sbr[r];
  sbe[h] = sbr[r + 1];
  for (uint32_t s = sbr[r]; s < sbr[r + 1]; ++s) sbhalo[s] = h;
}

// First super-bucket of the halos of at most kVBinEdge0 and at most kVBinEdge1 members
// (sizes decrease along the order; the total when no halo is that small).
__global__ void k_bin_edges(const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ horder,
                            const uint32_t *__restrict__ sbr, int64_t H, uint32_t *__restrict__ edges) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= H) return;
  const uint32_t hr = horder[r];
  const uint32_t nr = hoff[hr + 1] - hoff[hr];
  uint32_t np = 0xffffffffu;
  if (r > 0) {
    const uint32_t hp = horder[r - 1];
    np = hoff[hp + 1] - hoff[hp];
  }
  const uint32_t e[2] = {kVBinEdge0, kVBinEdge1};
  for (int k = 0; k < 2; ++k) {
    if (np > e[k] && nr <= e[k]) edges[k] = sbr[r];
    if (r == H - 1 && nr > e[k]) edges[k] = sbr[H];
  }
}

__global__ void k_bucket_boxes(const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ sbs,
                               const uint32_t *__restrict__ sbhalo, int64_t nbpad,
                               const int4 *__restrict__ u, int4 *__restrict__ bmin,
                               int4 *__restrict__ bmax) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbpad) return;
  uint32_t h = sbhalo[b >> 5];
  uint32_t local = (uint32_t)b - 32u * sbs[h];
  uint32_t s0 = hoff[h] + 32u * local, s1 = min(s0 + 32u, hoff[h + 1]);
  int4 lo = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0);
  int4 hi = make_int4(-0x7fffffff, -0x7fffffff, -0x7fffffff, 0);
  for (uint32_t m = s0; m < s1; ++m) {
    int4 p = u[m];
    lo.x = min(lo.x, p.x); lo.y = min(lo.y, p.y); lo.z = min(lo.z, p.z);
    hi.x = max(hi.x, p.x); hi.y = max(hi.y, p.y); hi.z = max(hi.z, p.z);
  }
  bmin[b] = lo;  // empty (padding) buckets keep an inverted box
  bmax[b] = hi;
}

__global__ void k_superbucket_boxes(int64_t nsb, const int4 *__restrict__ bmin,
                                    const int4 *__restrict__ bmax, int4 *__restrict__ smin,
                                    int4 *__restrict__ smax) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsb) return;
  int4 lo = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0);
  int4 hi = make_int4(-0x7fffffff, -0x7fffffff, -0x7fffffff, 0);
  for (int k = 0; k < 32; ++k) {
    int4 a = bmin[32 * s + k], c = bmax[32 * s + k];
    lo.x = min(lo.x, a.x); lo.y = min(lo.y, a.y); lo.z = min(lo.z, a.z);
    hi.x = max(hi.x, c.x); hi.y = max(hi.y, c.y); hi.z = max(hi.z, c.z);
  }
  smin[s] = lo;
  smax[s] = hi;
}

__device__ __forceinline__ long long gap1(int alo, int ahi, int blo, int bhi) {
  long long g = 0;
  if (blo > ahi) g = (long long)blo - ahi;
  else if (alo > bhi) g = (long long)alo - bhi;
  return g;
}
__device__ __forceinline__ long long box_d2(int4 alo, int4 ahi, int4 blo, int4 bhi) {
  long long gx = gap1(alo.x, ahi.x, blo.x, bhi.x), gy = gap1(alo.y, ahi.y, blo.y, bhi.y),
            gz = gap1(alo.z, ahi.z, blo.z, bhi.z);
  return gx * gx + gy * gy + gz * gz;
}
__device__ __forceinline__ long long pt_box_d2(int4 p, int4 blo, int4 bhi) {
  return box_d2(p, p, blo, bhi);
}

__device__ __forceinline__ int bitlen64(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

// ---------------------------------------------------------------- big halos
// Launch shape (tuning.cuh): BATCH candidates computed side by side, at most MAXREG
// registers, any number of warps per block up to 8 (blockDim.x / 32).
template <int NVM, int BATCH, int MAXREG>
__global__ void __launch_bounds__(256) __maxnreg__(MAXREG) k_velden_big(
    const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ sbs,
    const uint32_t *__restrict__ sbe, const uint32_t *__restrict__ sbhalo, int64_t b0,
    int64_t b1, const int4 *__restrict__ u,
    const float4 *__restrict__ v, const int4 *__restrict__ bmin, const int4 *__restrict__ bmax,
    const int4 *__restrict__ smin, const int4 *__restrict__ smax, int nse, int nv,
    float *__restrict__ f_l, DevStatus *st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<NVM> &sm = reinterpret_cast<WarpSmem<NVM> *>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int64_t b = b0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // buckets [b0, b1)
  if (b >= b1) return;
  const uint32_t h = sbhalo[b >> 5];
  const uint32_t hs = hoff[h], he = hoff[h + 1];
  const uint32_t nh = he - hs;
  const uint32_t sb0 = sbs[h], sb1 = sbe[h];
  const uint32_t local = (uint32_t)b - 32u * sb0;
  const uint32_t nbh = (nh + 31) / 32;
  if (local >= nbh) return;  // padding bucket
  const uint32_t qs = hs + 32u * local, qe = min(qs + 32u, he);
  const uint32_t k = qs + lane;
  const bool valid = k < qe;
  const int4 q = u[valid ? k : qs];
  const float4 vq = v[valid ? k : qs];
  const int nse_eff = nse;  // nh > nse here
  const int nv_eff = nv;
  int pass_id = 0;  // instrumentation only
  auto warp_max = [&](long long x) {
    for (int o = 16; o; o >>= 1) {
      long long y = __shfl_xor_sync(FULL, x, o);
      x = y > x ? y : x;
    }
    return x;
  };
  // stages slots [s0, s0 + cnt) in shared memory (positions; velocities if asked); the
  // remaining entries get a sentinel position far outside any bound (d^2 > 2^58), so the
  // candidate loops always run 32 fixed iterations
  auto stage = [&](uint32_t s0, int cnt, bool with_v) {
    __syncwarp();
    if (lane < cnt) {
      sm.su[lane] = u[s0 + lane];
      if (with_v) sm.sv[lane] = v[s0 + lane];
    } else {
      sm.su[lane] = make_int4(0x3fffffff, 0x3fffffff, 0x3fffffff, 0);
    }
    __syncwarp();
    VR_STAT(st, kStatPass0 + pass_id, 1);
  };
  const int4 qlo = bmin[b], qhi = bmax[b];
  // 1. bound from the window of kWindow * N_se members around the bucket: the N_se-th
  //    smallest distance among them, rounded up to a histogram bin edge. When the window's
  //    box and the bucket's box bound every separation by 32767 per axis (a warp-uniform
  //    test), the distances are exact in 32-bit arithmetic.
  long long r2 = 0;
  {
    const int W = (int)min((uint32_t)(kWindow * nse), nh);
    int64_t w0 = (int64_t)qs + 16 - W / 2;
    if (w0 + W > (int64_t)he) w0 = (int64_t)he - W;
    if (w0 < (int64_t)hs) w0 = hs;
    int4 wlo = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0);
    int4 whi = make_int4(-0x7fffffff, -0x7fffffff, -0x7fffffff, 0);
    for (int c = lane; c < W; c += 32) {
      const int4 pw = u[w0 + c];
      wlo.x = min(wlo.x, pw.x); wlo.y = min(wlo.y, pw.y); wlo.z = min(wlo.z, pw.z);
      whi.x = max(whi.x, pw.x); whi.y = max(whi.y, pw.y); whi.z = max(whi.z, pw.z);
    }
    for (int o = 16; o; o >>= 1) {
      wlo.x = min(wlo.x, __shfl_xor_sync(FULL, wlo.x, o));
      wlo.y = min(wlo.y, __shfl_xor_sync(FULL, wlo.y, o));
      wlo.z = min(wlo.z, __shfl_xor_sync(FULL, wlo.z, o));
      whi.x = max(whi.x, __shfl_xor_sync(FULL, whi.x, o));
      whi.y = max(whi.y, __shfl_xor_sync(FULL, whi.y, o));
      whi.z = max(whi.z, __shfl_xor_sync(FULL, whi.z, o));
    }
    const bool wn = fits32(qlo, qhi, wlo, whi);  // warp-uniform
    long long wmax = 0;
    uint32_t wmax32 = 0;
    for (int c = 0; c < W; c += 32) {
      const int cnt = min(32, W - c);
      stage((uint32_t)(w0 + c), cnt, false);
      if (wn) {
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          uint32_t d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2u(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j) wmax32 = (t0 + j < cnt && d[j] > wmax32) ? d[j] : wmax32;
        }
      } else {
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          long long d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2i(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j) wmax = (t0 + j < cnt && d[j] > wmax) ? d[j] : wmax;
        }
      }
    }
    if (wn) wmax = (long long)wmax32;
    for (int cb = 0; cb < kBins; ++cb) sm.hist[cb][lane] = 0;
    int sh0 = bitlen64((unsigned long long)wmax) - kBinBits;  // kBins bins over [0, 2^bitlen)
    if (sh0 < 0) sh0 = 0;
    for (int c = 0; c < W; c += 32) {
      const int cnt = min(32, W - c);
      stage((uint32_t)(w0 + c), cnt, false);
      if (wn) {  // wmax < 2^32, so sh0 <= 26
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          uint32_t d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2u(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j)
            if (t0 + j < cnt) sm.hist[d[j] >> sh0][lane]++;
        }
      } else {
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          long long d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2i(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j)
            if (t0 + j < cnt) sm.hist[(unsigned)(d[j] >> sh0)][lane]++;
        }
      }
    }
    int cum = 0, bs = kBins - 1;
    for (int cb = 0; cb < kBins; ++cb) {
      cum += sm.hist[cb][lane];
      if (cum >= nse_eff) {
        bs = cb;
        break;
      }
    }
    r2 = (((long long)bs + 1) << sh0) - 1;  // every distance in bins <= bs is <= r2
    if (r2 > wmax) r2 = wmax;
  }
  if (r2 >= (1LL << 41)) {
    raise_error(st, VR_ERR_UNSUPPORTED, 1);
    return;
  }
  // Candidate buckets are enumerated on the fly in every pass: super-bucket boxes, then
  // bucket boxes, against the query bucket's box grown by the largest per-lane bound;
  // f(bucket index) is called warp-uniformly for every bucket that passes.
  auto for_each_bucket = [&](long long rmax2, auto &&f) {
    for (uint32_t sbase = sb0; sbase < sb1; sbase += 32) {
      uint32_t sx = sbase + lane;
      bool hit = sx < sb1 && box_d2(qlo, qhi, smin[sx], smax[sx]) <= rmax2;
      unsigned hm = __ballot_sync(FULL, hit);
      while (hm) {
        int t = __ffs(hm) - 1;
        hm &= hm - 1;
        uint32_t bb = 32u * (sbase + t) + lane;
        bool in = (bb - 32u * sb0) < nbh && box_d2(qlo, qhi, bmin[bb], bmax[bb]) <= rmax2;
        unsigned bm = __ballot_sync(FULL, in);
        while (bm) {
          int tb = __ffs(bm) - 1;
          bm &= bm - 1;
          f(32u * (sbase + t) + (uint32_t)tb);
        }
      }
    }
  };
  // 2. histogram passes over the exact keys (d^2 << 22 | local index). The first level
  //    spreads its bins over [r2/4, r2] only (the N_se-th key lies near the bound) and
  //    counts the keys below in one register; later levels split the chosen bin.
  u64 klo = (u64)(r2 >> 2) << 22;
  int sh = bitlen64((((u64)(r2 + 1)) << 22) - klo - 1) - kBinBits;
  if (sh < 0) sh = 0;
  int need = nse_eff;
  bool settled = !valid;
  u64 fin_lo = 0, fin_hi = 0;
  int need_in = 0;
  long long rcur = r2;  // per-lane bound on d^2 of keys still of interest
  bool focus = true;    // this lane's current level is the focused first level
  for (int level = 0; level < 16; ++level) {
    pass_id = level < 5 ? 1 + level : 5;
    int below = 0;
    if (!settled)
      for (int c = 0; c < kBins; ++c) sm.hist[c][lane] = 0;
    const long long rmax2 = warp_max(settled ? -1 : rcur);
    for_each_bucket(rmax2, [&](uint32_t bb) {
      bool want = !settled && pt_box_d2(q, bmin[bb], bmax[bb]) <= rcur;
      if (!__any_sync(FULL, want)) return;
      const uint32_t s0 = hs + 32u * (bb - 32u * sb0);
      const int cnt = (int)min(32u, he - s0);
      stage(s0, cnt, false);
      // 32-bit route: the boxes bound every separation by 32767 per axis and the bins
      // are at least one unit of d^2 wide, so a key's bin depends on d^2 alone (klo is a
      // multiple of 2^22): bin = (d^2 - (klo >> 22)) >> (sh - 22)
      const bool narrow = fits32(qlo, qhi, bmin[bb], bmax[bb]);
      if (want && narrow && sh >= 22 && (klo & 0x3fffffull) == 0) {
        const uint32_t r32 = clamp32((u64)rcur), dlo = clamp32(klo >> 22);
        const int shd = sh - 22;
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          uint32_t d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2u(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j) {
            if (t0 + j < cnt && d[j] <= r32) {
              if (d[j] >= dlo) {
                const uint32_t rel = shd >= 32 ? 0u : (d[j] - dlo) >> shd;
                if (rel < kBins) sm.hist[rel][lane]++;
              } else if (focus) {
                ++below;
              }
            }
          }
        }
      } else if (want) {
        for (int t0 = 0; t0 < 32; t0 += BATCH) {
          long long d[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) d[j] = d2i(q, sm.su[t0 + j]);
#pragma unroll
          for (int j = 0; j < BATCH; ++j) {
            if (d[j] <= rcur) {
              u64 key = ((u64)d[j] << 22) | (u64)sm.su[t0 + j].w;
              if (key >= klo) {
                u64 rel = (key - klo) >> sh;
                if (rel < kBins) sm.hist[rel][lane]++;
              } else if (focus) {
                ++below;
              }
            }
          }
        }
      }
    });
    if (!settled) {
      if (focus && below >= need) {
        // the N_se-th key lies below the focused range: bin [0, klo) next
        const u64 hi = klo;
        klo = 0;
        sh = bitlen64(hi - 1) - kBinBits;
        if (sh < 0) sh = 0;
        const long long top_d = (long long)((hi - 1) >> 22);
        rcur = top_d < rcur ? top_d : rcur;
        focus = false;
      } else {
        if (focus) need -= below;  // every key below the focused range is in
        focus = false;
        int cum = 0, bs = kBins - 1;
        for (int c = 0; c < kBins; ++c) {
          int hc = sm.hist[c][lane];
          if (cum + hc >= need) {
            bs = c;
            break;
          }
          cum += hc;
        }
        int hc = sm.hist[bs][lane];
        if (hc <= kBuf || sh == 0) {
          fin_lo = klo + ((u64)bs << sh);
          fin_hi = fin_lo + ((u64)1 << sh);
          need_in = need - cum;
          settled = true;
        } else {
          klo += (u64)bs << sh;
          need -= cum;
          const long long top_d = (long long)((klo + ((u64)1 << sh) - 1) >> 22);
          rcur = top_d < rcur ? top_d : rcur;
          sh = sh >= kBinBits ? sh - kBinBits : 0;
        }
      }
    }
    if (__all_sync(FULL, settled)) break;
  }
  // 3. collect: keys below the final bin are in; the final bin is buffered
  if (valid) {
    const long long top_d = (long long)((fin_hi - 1) >> 22);
    rcur = top_d < r2 ? top_d : r2;
  } else {
    rcur = -1;
  }
  float(*top)[32] = sm.top;
  TopV tv = {0, 0, 0.0f};
  int nbuf = 0;
  pass_id = 6;
  for_each_bucket(warp_max(rcur), [&](uint32_t bb) {
    bool want = valid && pt_box_d2(q, bmin[bb], bmax[bb]) <= rcur;
    if (!__any_sync(FULL, want)) return;
    const uint32_t s0 = hs + 32u * (bb - 32u * sb0);
    const int cnt = (int)min(32u, he - s0);
    stage(s0, cnt, true);
    // 32-bit route as in the histogram passes: with both final-bin edges multiples of
    // 2^22, key < edge iff d^2 < edge >> 22
    const bool narrow = fits32(qlo, qhi, bmin[bb], bmax[bb]);
    if (want && narrow && ((fin_lo | fin_hi) & 0x3fffffull) == 0) {
      const uint32_t r32 = clamp32((u64)rcur), flo = clamp32(fin_lo >> 22),
                     fhi = clamp32(fin_hi >> 22);
      for (int t0 = 0; t0 < 32; t0 += BATCH) {
        uint32_t d[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) d[j] = d2u(q, sm.su[t0 + j]);
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
          if (t0 + j < cnt && d[j] <= r32) {
            const int t = t0 + j;
            if (d[j] < flo) {
              top_insert(top, lane, tv, nv_eff, dv2f(sm.sv[t], vq));
            } else if (d[j] < fhi && nbuf < kBuf) {
              sm.bslot[nbuf][lane] = s0 + (uint32_t)t;
              ++nbuf;
            }
          }
        }
      }
    } else if (want) {
      for (int t0 = 0; t0 < 32; t0 += BATCH) {
        long long d[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) d[j] = d2i(q, sm.su[t0 + j]);
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
          if (d[j] <= rcur) {
            const int t = t0 + j;
            u64 key = ((u64)d[j] << 22) | (u64)sm.su[t].w;
            if (key < fin_lo) {
              top_insert(top, lane, tv, nv_eff, dv2f(sm.sv[t], vq));
            } else if (key < fin_hi && nbuf < kBuf) {
              sm.bslot[nbuf][lane] = s0 + (uint32_t)t;
              ++nbuf;
            }
          }
        }
      }
    }
  });
  if (!valid) return;
  // the need_in smallest keys of the final bin (keys recomputed from the buffered slots)
  u64 last = 0;
  for (int r = 0; r < need_in; ++r) {
    int best = -1;
    u64 bk = ~0ULL;
    for (int e = 0; e < nbuf; ++e) {
      const int4 pe = u[sm.bslot[e][lane]];
      const u64 x = ((u64)d2i(q, pe) << 22) | (u64)pe.w;
      if ((r == 0 || x > last) && x < bk) {
        bk = x;
        best = e;
      }
    }
    if (best < 0) break;
    last = bk;
    top_insert(top, lane, tv, nv_eff, dv2f(v[sm.bslot[best][lane]], vq));
  }
  f_l[__float_as_int(vq.w)] = top_density(top, lane, tv, nse_eff);
}

__global__ void k_fill_f32(float *__restrict__ a, int64_t n, float val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = val;
}

}  // namespace

// Buckets with their padding: a halo of more than N_se members pads its buckets to a
// multiple of 32, at most 31 per such halo.
inline int64_t bucket_bound(int64_t n, int nse) { return n / 32 + 32 * (n / (nse + 1) + 2) + 64; }

size_t velden_bytes(int64_t n, int nmin, int nse) {
  Arena ar;
  int64_t hmax = n / (nmin > 0 ? nmin : 1) + 2;
  int64_t nbmax = bucket_bound(n, nse);
  ar.take<uint32_t>(hmax + 1);  // sbr
  ar.take<uint32_t>(hmax);      // sbs
  ar.take<uint32_t>(hmax);      // sbe
  ar.take<uint32_t>(4);         // bin edges
  ar.take<uint32_t>(nbmax / 32 + 1);  // sbhalo
  ar.take<int4>(nbmax);   // bmin
  ar.take<int4>(nbmax);   // bmax
  ar.take<int4>(nbmax / 32 + 1);  // smin
  ar.take<int4>(nbmax / 32 + 1);  // smax
  ar.take<char>(scan_scratch_bytes<uint32_t>(hmax + 1));
  return ar.off;
}

namespace {

// The f_l kernel instance for launch shape `shape` (tuning.cuh); N_v above 32 always uses
// the default shape.
template <int NVM>
void *big_kernel(int shape) {
  if (NVM > 32) return (void *)k_velden_big<NVM, 4, 80>;
  switch (kVShapes[shape].batch) {
    case 2: return (void *)k_velden_big<NVM, 2, 80>;
    case 8: return (void *)k_velden_big<NVM, 8, 96>;
    default: return (void *)k_velden_big<NVM, 4, 80>;
  }
}

}  // namespace

// Runs the f_l stage on an existing segmentation; f_l must already hold NaN outside
// halos.
vr_status run_velden(vr_ctx *ctx, const HaloSeg &g, const vr_params *p, Arena &ar, float *f_l,
                     cudaStream_t s, const uint32_t *hoff_host, cudaEvent_t ev_big) {
  if (g.H == 0) {
    if (ev_big) VR_CUDA(ctx, cudaEventRecord(ev_big, s));
    return VR_OK;
  }
  const int64_t H = g.H;
  int64_t hmax = g.n / (p->nmin > 0 ? p->nmin : 1) + 2;
  int64_t nbmax = bucket_bound(g.n, p->nse);
  uint32_t *sbr = ar.take<uint32_t>(hmax + 1);
  uint32_t *sbs = ar.take<uint32_t>(hmax);
  uint32_t *sbe = ar.take<uint32_t>(hmax);
  uint32_t *edges = ar.take<uint32_t>(4);
  uint32_t *sbhalo = ar.take<uint32_t>(nbmax / 32 + 1);
  int4 *bmin = ar.take<int4>(nbmax);
  int4 *bmax = ar.take<int4>(nbmax);
  int4 *smin = ar.take<int4>(nbmax / 32 + 1);
  int4 *smax = ar.take<int4>(nbmax / 32 + 1);
  void *scr = ar.take<char>(scan_scratch_bytes<uint32_t>(hmax + 1));
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int T = 256;
  // small halos: all members are neighbours
  auto small = [&](int64_t a, int64_t z) {
    if (p->nv <= 32)
      k_velden_small<32><<<grid_for(z - a, kWarps), 32 * kWarps, 0, s>>>(g.hoff, a, z, g.v, p->nse, p->nv, f_l);
    else
      k_velden_small<kNVMax><<<grid_for(z - a, kWarps), 32 * kWarps, 0, s>>>(g.hoff, a, z, g.v, p->nse, p->nv, f_l);
  };
  if (hoff_host) {  // one launch per halo
    for (int64_t h = 0; h < H; ++h) {
      if (hoff_host[h + 1] - hoff_host[h] > (uint32_t)p->nse) continue;
      small(h, h + 1);
      VR_LAUNCHED(ctx, "k_velden_small");
    }
  } else {
    VR_TIMED(ctx, "velden_small", s, small(0, H));
    VR_LAUNCHED(ctx, "k_velden_small");
  }
  k_sb_count<<<grid_for(H + 1, T), T, 0, s>>>(g.hoff, g.horder, H, p->nse, sbr);
  VR_LAUNCHED(ctx, "k_sb_count");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(sbr, sbr, H + 1, scr, s));
  k_bin_edges<<<grid_for(H, T), T, 0, s>>>(g.hoff, g.horder, sbr, H, edges);
  VR_LAUNCHED(ctx, "k_bin_edges");
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 34, sbr + H, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 35, edges, 2 * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  uint32_t nsb = 0, eg[2] = {0, 0};
  memcpy(&nsb, ctx->h_pinned + 34, 4);
  memcpy(eg, ctx->h_pinned + 35, 8);
  if (nsb == 0) {
    if (ev_big) VR_CUDA(ctx, cudaEventRecord(ev_big, s));
    return VR_OK;
  }
  int64_t nbpad = 32LL * nsb;
  k_sb_fill<<<grid_for(H, T), T, 0, s>>>(sbr, g.horder, H, sbs, sbe, sbhalo);
  VR_LAUNCHED(ctx, "k_sb_fill");
  k_bucket_boxes<<<grid_for(nbpad, T), T, 0, s>>>(g.hoff, sbs, sbhalo, nbpad, g.u, bmin, bmax);
  VR_LAUNCHED(ctx, "k_bucket_boxes");
  k_superbucket_boxes<<<grid_for(nsb, T), T, 0, s>>>(nsb, bmin, bmax, smin, smax);
  VR_LAUNCHED(ctx, "k_superbucket_boxes");
  const size_t wsm = p->nv <= 32 ? sizeof(WarpSmem<32>) : sizeof(WarpSmem<kNVMax>);
  for (int sh = 0; sh < kNVShapes; ++sh) {
    void *kf = p->nv <= 32 ? big_kernel<32>(sh) : big_kernel<kNVMax>(sh);
    VR_CUDA(ctx, cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * wsm)));
  }
  // buckets [a, z) with launch shape `sh`
  auto big = [&](int sh, int64_t a, int64_t z) -> cudaError_t {
    const int w = p->nv <= 32 ? kVShapes[sh].warps : 4;
    void *kf = p->nv <= 32 ? big_kernel<32>(sh) : big_kernel<kNVMax>(sh);
    const int nse = p->nse, nv = p->nv;
    DevStatus *st = ctx->d_status;
    void *args[] = {(void *)&g.hoff, (void *)&sbs, (void *)&sbe, (void *)&sbhalo, (void *)&a,
                    (void *)&z, (void *)&g.u, (void *)&g.v, (void *)&bmin, (void *)&bmax,
                    (void *)&smin, (void *)&smax, (void *)&nse, (void *)&nv, (void *)&f_l,
                    (void *)&st};
    return cudaLaunchKernel(kf, dim3(grid_for(z - a, w)), dim3(32 * w), args, w * wsm, s);
  };
  if (hoff_host) {  // one launch per halo
    std::vector<uint32_t> s0(H), s1(H);
    VR_CUDA(ctx, cudaMemcpyAsync(s0.data(), sbs, H * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaMemcpyAsync(s1.data(), sbe, H * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t h = 0; h < H; ++h) {
      if (s1[h] == s0[h]) continue;
      VR_CUDA(ctx, big(0, 32LL * s0[h], 32LL * s1[h]));
      VR_LAUNCHED(ctx, "k_velden_big");
    }
    return VR_OK;
  }
  // one launch per halo-size bin, each with its own shape; a bin still to be tuned is
  // run once per candidate shape (same results each time) and keeps the fastest
  const int64_t lo[kVBins] = {0, 32LL * eg[0], 32LL * eg[1]};
  const int64_t hi[kVBins] = {32LL * eg[0], 32LL * eg[1], nbpad};
  timer_begin(ctx, "velden_big", s);
  for (int k = 0; k < kVBins; ++k) {
    if (hi[k] <= lo[k]) {
      if (k == 0 && ev_big) VR_CUDA(ctx, cudaEventRecord(ev_big, s));
      continue;
    }
    if (p->nv <= 32 && vmeasure(ctx, k)) {
      Tuning *tn = ctx->tune;
      cudaEvent_t e0, e1;
      VR_CUDA(ctx, cudaEventCreate(&e0));
      VR_CUDA(ctx, cudaEventCreate(&e1));
      int best = 0;
      for (int sh = 0; sh < kNVShapes; ++sh) {
        VR_CUDA(ctx, cudaEventRecord(e0, s));
        VR_CUDA(ctx, big(sh, lo[k], hi[k]));
        VR_LAUNCHED(ctx, "k_velden_big");
        VR_CUDA(ctx, cudaEventRecord(e1, s));
        VR_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        VR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        tn->vms[k][sh] = ms;
        if (ms < tn->vms[k][best]) best = sh;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      tn->vshape[k] = best;
      tn->vtuned[k] = 1;
    } else {
      VR_CUDA(ctx, big(p->nv <= 32 ? vshape_for(ctx, k) : 0, lo[k], hi[k]));
      VR_LAUNCHED(ctx, "k_velden_big");
    }
    if (k == 0 && ev_big) VR_CUDA(ctx, cudaEventRecord(ev_big, s));  // halos > kVBinEdge0 done
  }
  timer_end(ctx, "velden_big", s);
  return VR_OK;
}

vr_status fill_f32(vr_ctx *ctx, float *a, int64_t n, float val, cudaStream_t s) {
  k_fill_f32<<<grid_for(n, 256), 256, 0, s>>>(a, n, val);
  VR_LAUNCHED(ctx, "k_fill_f32");
  return VR_OK;
}

}  // namespace vr
