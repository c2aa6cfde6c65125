// Cleaning of outlier groups (Sec. 2.2, "Cleaning the catalogue", Eq. ellsig).
//
// A group of N particles is significant when <ell> >= ell_bar(ell_th) (1 + beta/sqrt(N)).
// A group that is not loses particles in order of smallest ell (ties: smaller particle
// index first) until it is, and is removed if fewer than N_min remain.
//
// GB300 design: the grouped particles are sorted once by (label, ell) with the stable
// radix sort (the particle index breaks ties, since the input is in index order); one
// warp then takes one group. It walks the sorted group from its end in 32-wide chunks,
// forming the sum of every suffix by a warp scan plus a carry, tests Eq. ellsig for every
// possible number of removed particles at once, and keeps the smallest that passes. The
// ell values are FP32, so every partial sum is exact in FP64 while the group's sum of ell
// stays below 2^53 ulp_FP32(smallest ell) (2^31 for ell >= 2): the sums, and with them
// the decisions, do not depend on the order of additions and equal a sequential FP64
// evaluation.
#include <math.h>

#include "vr_workspace.h"

namespace vr {

namespace {

constexpr int kClWarps = 4;

__device__ __forceinline__ uint32_t f2key(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_cl_flags(const int32_t *__restrict__ label6, int64_t n, uint32_t *__restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  flag[i] = (i < n && label6[i] >= 0) ? 1u : 0u;
}

__global__ void k_cl_keys(const int32_t *__restrict__ label6, const float *__restrict__ ell,
                          const uint32_t *__restrict__ flag, int64_t n, u64 *__restrict__ key,
                          uint32_t *__restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || flag[i + 1] == flag[i]) return;
  const uint32_t j = flag[i];
  key[j] = ((u64)(uint32_t)label6[i] << 32) | f2key(ell[i]);
  val[j] = (uint32_t)i;
}

// head[j] = 1 where a group starts in the sorted order (head[m] = 0).
__global__ void k_cl_heads(const u64 *__restrict__ key, int64_t m, uint32_t *__restrict__ head) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > m) return;
  head[j] = (j < m && (j == 0 || (key[j] >> 32) != (key[j - 1] >> 32))) ? 1u : 0u;
}

// goff[g] = first sorted position of group g; goff[G] = m (G = hscan[m]).
__global__ void k_cl_goff(const uint32_t *__restrict__ hscan, int64_t m, uint32_t *__restrict__ goff) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > m) return;
  if (j == m) goff[hscan[m]] = (uint32_t)m;
  else if (hscan[j + 1] != hscan[j]) goff[hscan[j]] = (uint32_t)j;
}

// One warp per group (grid-stride over groups).
__global__ void __launch_bounds__(32 * kClWarps) k_cl_group(
    const u64 *__restrict__ key, const uint32_t *__restrict__ val,
    const uint32_t *__restrict__ goff, const uint32_t *__restrict__ ngroups, double lbar,
    double beta, int nmin, int32_t *__restrict__ label6, unsigned long long *__restrict__ nkept) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const uint32_t G = *ngroups;
  const uint32_t nw = gridDim.x * kClWarps;
  for (uint32_t g = blockIdx.x * kClWarps + (threadIdx.x >> 5); g < G; g += nw) {
    const uint32_t b = goff[g];
    const int64_t N = (int64_t)goff[g + 1] - b;
    // smallest number of removed particles k after which Eq. ellsig holds (-1: none)
    int64_t cut = -1;
    double carry = 0.0;  // sum of ell after the current chunk
    for (int64_t cb = ((N - 1) / 32) * 32; cb >= 0; cb -= 32) {
      const int64_t k = cb + lane;
      const double x = k < N ? (double)key2f((uint32_t)key[b + k]) : 0.0;
      double sfx = x;  // sum over the chunk's positions >= k
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_down_sync(FULL, sfx, o);
        if (lane + o < 32) sfx = __dadd_rn(sfx, y);
      }
      const double S = __dadd_rn(sfx, carry);  // sum over positions >= k
      bool ok = false;
      if (k < N) {
        const double m = (double)(N - k);
        const double mean = __ddiv_rn(S, m);
        const double thr = __dmul_rn(lbar, __dadd_rn(1.0, __ddiv_rn(beta, __dsqrt_rn(m))));
        ok = mean >= thr;
      }
      const unsigned bm = __ballot_sync(FULL, ok);
      if (bm) cut = cb + (__ffs(bm) - 1);
      carry = __shfl_sync(FULL, S, 0);
    }
    const bool keep = cut >= 0 && N - cut >= nmin;
    uint32_t lab = 0xffffffffu;
    if (keep)
      for (int64_t k = cut + lane; k < N; k += 32) lab = min(lab, val[b + k]);
#pragma unroll
    for (int o = 16; o; o >>= 1) lab = min(lab, __shfl_xor_sync(FULL, lab, o));
    for (int64_t k = lane; k < N; k += 32)
      label6[val[b + k]] = (keep && k >= cut) ? (int32_t)lab : -1;
    if (keep && lane == 0) atomicAdd(nkept, 1ull);
  }
}

}  // namespace

size_t clean_bytes(int64_t n) {
  Arena ar;
  ar.take<uint32_t>(n + 1);  // flags / scan
  ar.take<u64>(n);           // keys
  ar.take<u64>(n);
  ar.take<uint32_t>(n);      // values
  ar.take<uint32_t>(n);
  ar.take<uint32_t>(n + 1);  // heads / scan
  ar.take<uint32_t>(n + 1);  // group offsets
  ar.take<unsigned long long>(1);
  const size_t a = scan_scratch_bytes<uint32_t>(n + 1), r = radix_scratch_bytes<u64>(n);
  ar.take<char>(a > r ? a : r);
  return ar.off;
}

// Tail mean of a unit Gaussian above ell_th (Eq. ellsig), in the operation order
// sqrt(2/pi) * exp((-0.5 ell_th) ell_th) / erfc(ell_th / sqrt 2).
double ell_bar_host(double ell_th) {
  const double a = -0.5 * ell_th;
  const double e = exp(a * ell_th);
  const double c = sqrt(2.0 / 3.14159265358979323846);
  return c * e / erfc(ell_th / sqrt(2.0));
}

vr_status run_clean(vr_ctx *ctx, const float *ell, int64_t n, const vr_params *p, double beta,
                    int32_t *label6, int64_t *ngroups, Arena &ar, cudaStream_t s) {
  uint32_t *flag = ar.take<uint32_t>(n + 1);
  u64 *k0 = ar.take<u64>(n);
  u64 *k1 = ar.take<u64>(n);
  uint32_t *v0 = ar.take<uint32_t>(n);
  uint32_t *v1 = ar.take<uint32_t>(n);
  uint32_t *head = ar.take<uint32_t>(n + 1);
  uint32_t *goff = ar.take<uint32_t>(n + 1);
  unsigned long long *nkept = ar.take<unsigned long long>(1);
  const size_t a = scan_scratch_bytes<uint32_t>(n + 1), r = radix_scratch_bytes<u64>(n);
  void *scr = ar.take<char>(a > r ? a : r);
  if (!ar.ok()) return set_error(ctx, VR_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
  const int T = 256;
  VR_CUDA(ctx, cudaMemsetAsync(nkept, 0, sizeof(unsigned long long), s));
  k_cl_flags<<<grid_for(n + 1, T), T, 0, s>>>(label6, n, flag);
  VR_LAUNCHED(ctx, "k_cl_flags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(flag, flag, n + 1, scr, s));
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 38, flag + n, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
  VR_CUDA(ctx, cudaStreamSynchronize(s));
  uint32_t m = 0;
  memcpy(&m, ctx->h_pinned + 38, 4);
  if (m > 0) {
    k_cl_keys<<<grid_for(n, T), T, 0, s>>>(label6, ell, flag, n, k0, v0);
    VR_LAUNCHED(ctx, "k_cl_keys");
    int which = 0;
    int lbits = 1;
    while (lbits < 31 && ((int64_t)1 << lbits) < n) ++lbits;  // labels are < n
    VR_CUDA(ctx, radix_sort_pairs<u64>(k0, v0, k1, v1, m, 0, 32 + lbits, scr, s, &which));
    const u64 *key = which ? k1 : k0;
    const uint32_t *val = which ? v1 : v0;
    k_cl_heads<<<grid_for(m + 1, T), T, 0, s>>>(key, m, head);
    VR_LAUNCHED(ctx, "k_cl_heads");
    VR_CUDA(ctx, exclusive_scan<uint32_t>(head, head, m + 1, scr, s));
    k_cl_goff<<<grid_for(m + 1, T), T, 0, s>>>(head, m, goff);
    VR_LAUNCHED(ctx, "k_cl_goff");
    const int64_t sms = ctx->sm_count > 0 ? ctx->sm_count : 152;
    int64_t grid = (m + 32 * kClWarps - 1) / (32 * kClWarps);
    if (grid > 8 * sms) grid = 8 * sms;
    VR_TIMED(ctx, "clean", s, k_cl_group<<<(unsigned)grid, 32 * kClWarps, 0, s>>>(
        key, val, goff, head + m, ell_bar_host(p->ell_th), beta, p->nmin, label6, nkept));
    VR_LAUNCHED(ctx, "k_cl_group");
  }
  VR_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 39, nkept, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
  vr_status st = read_status(ctx, s, nullptr);
  if (st != VR_OK) return st;
  if (ngroups) *ngroups = (int64_t)ctx->h_pinned[39];
  return VR_OK;
}

}  // namespace vr
