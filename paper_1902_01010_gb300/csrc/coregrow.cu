// Core cleaning and core growth (Sec. 2.3, "Cleaning the Catalogue" and "Core Growth &
// Mass Reconstruction"; Eqs. coremeanphase, coredispphase, coredist, coresig), after the
// core search of fof6d.cu.
//
// GB300 design:
//  - cores are enumerated by their root member (the member whose particle index is the
//    core label) in slot order, so each halo's cores form one contiguous id range found
//    by a prefix sum over the slots;
//  - one CTA per core sweeps its halo's slots twice (mean, then second moments about the
//    mean) and reduces in a fixed order (warp shuffles, then warp 0), so results are
//    deterministic; the same CTA factors the 6x6 tensor (Cholesky, FP64) and, on the
//    first pass, evaluates Eq. coresig against the mean of the primary group of the
//    core's loop;
//  - one thread per slot assigns untagged members of the current level to the nearest
//    active core of their halo (FP64 forward substitution), each thread writing only its
//    own slot, so a level needs no atomics; one host loop over the levels.
// Cholesky and D^2 use explicitly rounded FP64 operations in the order of the formulas.
#include <math.h>

#include "stages.h"
#include "vr_workspace.h"

namespace vr {

namespace {

constexpr int kCT = 256;  // threads per core CTA

// Packed lower triangle of a symmetric 6x6: (i, j), j <= i, at i (i + 1) / 2 + j.
__host__ __device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

struct CoreTab {
  int32_t *label;   // [K] core label (minimum particle index)
  int32_t *level;   // [K] loop at which the core was found
  int32_t *halo;    // [K]
  uint8_t *prim;    // [K] 1 for the halo's primary core
  uint8_t *alive;   // [K] kept by the cleaning
  uint8_t *pd;      // [K] tensor positive definite
  double *mean;     // [K][6]
  double *S;        // [K][21] tensor, packed lower triangle
  double *L;        // [K][21] Cholesky factor, packed lower triangle
};

__device__ __forceinline__ void load_x(const int4 *__restrict__ u, const float4 *__restrict__ v,
                                       int64_t m, double *X) {
  const int4 p = u[m];
  const float4 w = v[m];
  X[0] = (double)p.x; X[1] = (double)p.y; X[2] = (double)p.z;
  X[3] = (double)w.x; X[4] = (double)w.y; X[5] = (double)w.z;
}

// Cholesky of the packed 6x6 S into L (packed); false unless every pivot is > 0.
__device__ bool chol6(const double *S, double *L) {
  for (int j = 0; j < 6; ++j) {
    double d = S[tri(j, j)];
    for (int k = 0; k < j; ++k) d = __dsub_rn(d, __dmul_rn(L[tri(j, k)], L[tri(j, k)]));
    if (!(d > 0.0)) return false;
    const double ljj = __dsqrt_rn(d);
    L[tri(j, j)] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double t = S[tri(i, j)];
      for (int k = 0; k < j; ++k) t = __dsub_rn(t, __dmul_rn(L[tri(i, k)], L[tri(j, k)]));
      L[tri(i, j)] = __ddiv_rn(t, ljj);
    }
  }
  return true;
}

// Eq. coredist: D^2 = |y|^2 with L y = d (forward substitution).
__device__ __forceinline__ double dist6(const double *__restrict__ L, const double *d) {
  double y[6], D2 = 0.0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double t = d[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t = __dsub_rn(t, __dmul_rn(L[tri(i, k)], y[k]));
    y[i] = __ddiv_rn(t, L[tri(i, i)]);
    D2 = __dadd_rn(D2, __dmul_rn(y[i], y[i]));
  }
  return D2;
}

// Scalar form (growth mode 0): |dx|^2 / s_x^2 + |dv|^2 / s_v^2, s^2 the mean diagonal of
// the position / velocity block.
__device__ __forceinline__ double dist_scalar(const double *__restrict__ S, const double *d) {
  const double sx2 = __ddiv_rn(__dadd_rn(__dadd_rn(S[tri(0, 0)], S[tri(1, 1)]), S[tri(2, 2)]), 3.0);
  const double sv2 = __ddiv_rn(__dadd_rn(__dadd_rn(S[tri(3, 3)], S[tri(4, 4)]), S[tri(5, 5)]), 3.0);
  const double a = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  const double b = __dadd_rn(__dadd_rn(__dmul_rn(d[3], d[3]), __dmul_rn(d[4], d[4])), __dmul_rn(d[5], d[5]));
  return __dadd_rn(__ddiv_rn(a, sx2), __ddiv_rn(b, sv2));
}

// Block sum of NV doubles per thread, fixed order; the result is valid in thread 0.
template <int NV>
__device__ void block_sum(double *x, double (*red)[kCT / 32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o; o >>= 1) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][w] = x[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = red[k][0];
      for (int q = 1; q < kCT / 32; ++q) t += red[k][q];
      x[k] = t;
    }
}

__global__ void k_cg_roots(const float4 *__restrict__ v, int64_t nhp, const int32_t *__restrict__ core,
                           uint32_t *__restrict__ flag) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int pi = __float_as_int(v[m].w);
  flag[m] = core[pi] == pi ? 1u : 0u;
}

__global__ void k_cg_table(const uint32_t *__restrict__ hid, const float4 *__restrict__ v,
                           int64_t nhp, const int32_t *__restrict__ core,
                           const int32_t *__restrict__ level, const uint32_t *__restrict__ pre,
                           const int *__restrict__ prim, const int *__restrict__ last, CoreTab t,
                           int32_t *__restrict__ cid_of) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int pi = __float_as_int(v[m].w);
  if (core[pi] != pi) return;
  const uint32_t k = pre[m], h = hid[m];
  t.label[k] = pi;
  t.level[k] = level[pi];
  t.halo[k] = (int32_t)h;
  t.prim[k] = last[h] >= 0 && prim[h] == pi;
  t.alive[k] = 0;
  t.pd[k] = 0;
  cid_of[pi] = (int32_t)k;
}

// Current core of every slot (-1: untagged or not in a searched halo's background).
__global__ void k_cg_slots(const float4 *__restrict__ v, int64_t nhp, const int32_t *__restrict__ core,
                           const int32_t *__restrict__ cid_of, int32_t *__restrict__ gc) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int c = core[__float_as_int(v[m].w)];
  gc[m] = c >= 0 ? cid_of[c] : -1;
}

// One CTA per core: mean and tensor of the members whose current core is k (Eqs.
// coremeanphase, coredispphase), its Cholesky factor, and with `clean` set the cleaning
// of Eq. coresig. With l >= 0 only cores active at level l are recomputed.
__global__ void __launch_bounds__(kCT) k_cg_moments(
    const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ pre, const int4 *__restrict__ u,
    const float4 *__restrict__ v, const int32_t *__restrict__ gc, const int32_t *__restrict__ searched,
    CoreTab t, int l, int clean, double beta_c) {
  __shared__ double red[21][kCT / 32];
  __shared__ double smean[6];
  const int k = blockIdx.x;
  if (l >= 0 && !(t.alive[k] && (t.prim[k] || t.level[k] >= l))) return;
  const int h = t.halo[k];
  const uint32_t s0 = hoff[h], s1 = hoff[h + 1];
  const bool with_p = clean && !t.prim[k];
  // primary core id of the halo (for the primary group of the cleaning)
  int pk = -1;
  if (with_p)
    for (uint32_t q = pre[s0]; q < pre[s1]; ++q)
      if (t.prim[q]) pk = (int)q;
  const int lp = t.level[k] + 1;
  double acc[13];
#pragma unroll
  for (int a = 0; a < 13; ++a) acc[a] = 0.0;
  for (uint32_t m = s0 + threadIdx.x; m < s1; m += kCT) {
    const int c = gc[m];
    const bool in = c == k;
    const bool inp = with_p && (c == pk || searched[__float_as_int(v[m].w)] >= lp);
    if (!in && !inp) continue;
    double X[6];
    load_x(u, v, m, X);
    if (in) {
#pragma unroll
      for (int a = 0; a < 6; ++a) acc[a] += X[a];
      acc[12] += 1.0;
    }
    if (inp) {
#pragma unroll
      for (int a = 0; a < 6; ++a) acc[6 + a] += X[a];
    }
  }
  // the primary group's count rides in the reduction too
  double pc = 0.0;
  if (with_p)
    for (uint32_t m = s0 + threadIdx.x; m < s1; m += kCT) {
      const int c = gc[m];
      pc += (c == pk || searched[__float_as_int(v[m].w)] >= lp) ? 1.0 : 0.0;
    }
  double x14[14];
#pragma unroll
  for (int a = 0; a < 13; ++a) x14[a] = acc[a];
  x14[13] = pc;
  block_sum<14>(x14, red);
  const double M = x14[12];
  if (threadIdx.x == 0)
#pragma unroll
    for (int a = 0; a < 6; ++a) smean[a] = x14[a] / M;
  __syncthreads();
  double mean[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) mean[a] = smean[a];
  double c2[21];
#pragma unroll
  for (int a = 0; a < 21; ++a) c2[a] = 0.0;
  for (uint32_t m = s0 + threadIdx.x; m < s1; m += kCT) {
    if (gc[m] != k) continue;
    double X[6];
    load_x(u, v, m, X);
    double d[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) d[a] = X[a] - mean[a];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) c2[tri(i, j)] += d[i] * d[j];
  }
  block_sum<21>(c2, red);
  if (threadIdx.x != 0) return;
  double S[21], L[21];
#pragma unroll
  for (int a = 0; a < 21; ++a) S[a] = c2[a] / M;
  const bool pd = M > 0.0 && chol6(S, L);
#pragma unroll
  for (int a = 0; a < 6; ++a) t.mean[6 * (int64_t)k + a] = mean[a];
#pragma unroll
  for (int a = 0; a < 21; ++a) {
    t.S[21 * (int64_t)k + a] = S[a];
    t.L[21 * (int64_t)k + a] = L[a];
  }
  t.pd[k] = pd;
  if (clean) {
    if (t.prim[k]) {
      t.alive[k] = 1;
    } else {
      const double Mp = x14[13];
      double d[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) d[a] = x14[6 + a] / Mp - mean[a];
      t.alive[k] = pd && Mp > 0.0 && dist6(L, d) >= beta_c;
    }
  }
}

// Members of dropped cores return to the untagged background; halos that keep a
// candidate core grow.
__global__ void k_cg_drop(int64_t nhp, const uint32_t *__restrict__ hid, CoreTab t,
                          int32_t *__restrict__ gc, int *__restrict__ hgrow) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int c = gc[m];
  if (c < 0) return;
  if (!t.alive[c]) gc[m] = -1;
  else if (!t.prim[c]) hgrow[hid[m]] = 1;
}

// Level l: every untagged member last searched at l goes to the nearest active core.
__global__ void k_cg_assign(int64_t nhp, const uint32_t *__restrict__ hid,
                            const uint32_t *__restrict__ hoff, const uint32_t *__restrict__ pre,
                            const int4 *__restrict__ u, const float4 *__restrict__ v,
                            const int32_t *__restrict__ searched, const int *__restrict__ hgrow,
                            CoreTab t, int l, int mode, int32_t *__restrict__ gc) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  if (gc[m] >= 0) return;
  const uint32_t h = hid[m];
  if (!hgrow[h] || searched[__float_as_int(v[m].w)] != l) return;
  double X[6];
  load_x(u, v, m, X);
  double best = INFINITY;
  int bk = -1, blab = 0;
  for (uint32_t k = pre[hoff[h]]; k < pre[hoff[h + 1]]; ++k) {
    if (!t.alive[k] || !(t.prim[k] || t.level[k] >= l) || !t.pd[k]) continue;
    double d[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) d[a] = __dsub_rn(X[a], t.mean[6 * (int64_t)k + a]);
    const double D2 = mode == 0 ? dist_scalar(t.S + 21 * (int64_t)k, d) : dist6(t.L + 21 * (int64_t)k, d);
    if (!(D2 < INFINITY)) continue;
    const int lab = t.label[k];
    if (bk < 0 || D2 < best || (D2 == best && lab < blab)) {
      best = D2;
      bk = (int)k;
      blab = lab;
    }
  }
  if (bk >= 0) gc[m] = bk;
}

__global__ void k_cg_out(int64_t nhp, const float4 *__restrict__ v, const int32_t *__restrict__ gc,
                         CoreTab t, int32_t *__restrict__ grown) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const int c = gc[m];
  grown[__float_as_int(v[m].w)] = c >= 0 ? t.label[c] : -1;
}

__global__ void k_cg_count(int64_t K, CoreTab t, unsigned long long *cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K && t.alive[k]) atomicAdd(cnt, 1ull);
}

}  // namespace

size_t coregrow_bytes(int64_t n, int nmin) {
  Arena ar;
  const int64_t kmax = n / (nmin > 0 ? nmin : 1) + 2;
  ar.take<int32_t>(n);          // searched (taken by the caller before run_cores)
  ar.take<int32_t>(n);          // cid_of
  ar.take<int32_t>(n);          // gc
  ar.take<uint32_t>(n + 1);     // pre
  ar.take<int>(n / (nmin > 0 ? nmin : 1) + 2);  // hgrow
  for (int k = 0; k < 3; ++k) ar.take<int32_t>(kmax);
  for (int k = 0; k < 3; ++k) ar.take<uint8_t>(kmax);
  ar.take<double>(6 * kmax);
  ar.take<double>(21 * kmax);
  ar.take<double>(21 * kmax);
  ar.take<unsigned long long>(1);
  return ar.off + scan_scratch_bytes<uint32_t>(n + 1) + 4096;
}

vr_status run_core_grow(vr_ctx *ctx, const HaloSeg &g, const vr_core_params *cp,
                        const vr_core_grow_params *gp, Arena &ar, const int32_t *core,
                        const int32_t *level, const CoreExtra &ex, int32_t *grown,
                        int64_t *nkept, cudaStream_t s) {
  if (nkept) *nkept = 0;
  const int64_t n = g.n, NHP = g.NHP, H = g.H;
  vr_status st = fill_i32(ctx, grown, n, -1, s);
  if (st != VR_OK || NHP == 0 || H == 0) return st;
  const int T = 256;
  int32_t *cid_of = ar.take<int32_t>(n);
  int32_t *gc = ar.take<int32_t>(NHP);
  uint32_t *pre = ar.take<uint32_t>(NHP + 1);
  int *hgrow = ar.take<int>(H);
  unsigned long long *cnt = ar.take<unsigned long long>(1);
  void *scan_ws = ar.take<char>(scan_scratch_bytes<uint32_t>(NHP + 1));
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  k_cg_roots<<<grid_for(NHP, T), T, 0, s>>>(g.v, NHP, core, pre);
  VR_LAUNCHED(ctx, "k_cg_roots");
  VR_CUDA(ctx, cudaMemsetAsync(pre + NHP, 0, sizeof(uint32_t), s));
  VR_CUDA(ctx, exclusive_scan<uint32_t>(pre, pre, NHP + 1, scan_ws, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 41, pre + NHP, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  uint32_t k32;
  memcpy(&k32, ctx->h_pinned + 41, 4);
  const int64_t K = (int64_t)k32;
  if (K == 0) return VR_OK;
  CoreTab t;
  t.label = ar.take<int32_t>(K);
  t.level = ar.take<int32_t>(K);
  t.halo = ar.take<int32_t>(K);
  t.prim = ar.take<uint8_t>(K);
  t.alive = ar.take<uint8_t>(K);
  t.pd = ar.take<uint8_t>(K);
  t.mean = ar.take<double>(6 * K);
  t.S = ar.take<double>(21 * K);
  t.L = ar.take<double>(21 * K);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  k_cg_table<<<grid_for(NHP, T), T, 0, s>>>(g.hid, g.v, NHP, core, level, pre, ex.prim, ex.last, t,
                                            cid_of);
  VR_LAUNCHED(ctx, "k_cg_table");
  k_cg_slots<<<grid_for(NHP, T), T, 0, s>>>(g.v, NHP, core, cid_of, gc);
  VR_LAUNCHED(ctx, "k_cg_slots");
  // the cores as found, and the cleaning
  VR_TIMED(ctx, "core_grow", s, k_cg_moments<<<(unsigned)K, kCT, 0, s>>>(
      g.hoff, pre, g.u, g.v, gc, ex.searched, t, -1, 1, gp->beta_c));
  VR_LAUNCHED(ctx, "k_cg_moments");
  VR_CUDA(ctx, cudaMemsetAsync(hgrow, 0, H * sizeof(int), s));
  k_cg_drop<<<grid_for(NHP, T), T, 0, s>>>(NHP, g.hid, t, gc, hgrow);
  VR_LAUNCHED(ctx, "k_cg_drop");
  for (int l = cp->n_loop - 1; l >= 0; --l) {
    if (gp->mode == 2) {
      VR_TIMED(ctx, "core_grow", s, k_cg_moments<<<(unsigned)K, kCT, 0, s>>>(
          g.hoff, pre, g.u, g.v, gc, ex.searched, t, l, 0, 0.0));
      VR_LAUNCHED(ctx, "k_cg_moments");
    }
    VR_TIMED(ctx, "core_grow", s, k_cg_assign<<<grid_for(NHP, T), T, 0, s>>>(
        NHP, g.hid, g.hoff, pre, g.u, g.v, ex.searched, hgrow, t, l, gp->mode, gc));
    VR_LAUNCHED(ctx, "k_cg_assign");
  }
  k_cg_out<<<grid_for(NHP, T), T, 0, s>>>(NHP, g.v, gc, t, grown);
  VR_LAUNCHED(ctx, "k_cg_out");
  VR_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_cg_count<<<grid_for(K, T), T, 0, s>>>(K, t, cnt);
  VR_LAUNCHED(ctx, "k_cg_count");
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 42, cnt, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  if (nkept) *nkept = (int64_t)ctx->h_pinned[42];
  return VR_OK;
}

}  // namespace vr
