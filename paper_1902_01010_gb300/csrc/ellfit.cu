// Skew-Gaussian fit of each searched halo's R distribution (Eq. skewgaus) and the
// normalised ratio ell = (R - Rbar) / sigma_R (Eq. ell).
//
// One CTA per searched halo:
//  - median and MAD of the finite R values by exact radix selection (float keys, then
//    FP64 keys of |R - median|), MAD' = 1.4826 MAD;
//  - nbins = clamp(ceil(sqrt(N)), min, max) equal bins on [median - 6 MAD', median +
//    6 MAD'], bin = floor((R - lo) / width) evaluated without fused multiply-add, so the
//    counts equal those of an FP64 reference fed the same R values;
//  - Levenberg-Marquardt on the counts (unweighted least squares; start A = max count,
//    Rbar = centre of the first fullest bin, sigma = MAD', s = 1; lambda 1e-3, /10 on an
//    accepted step, x10 on a rejected one; stop on a relative cost change below 1e-15),
//    with warp 0 spreading the bins over its lanes.
#include <math.h>

#include <vector>

#include "halos.cuh"
#include "vr_workspace.h"
#include "background.cuh"

namespace vr {

namespace {

constexpr int kFT = 256;
#ifndef VR_FIT_MINB
#define VR_FIT_MINB 4  // resident CTAs per SM the register budget is set for
#endif
constexpr int kMaxFitBins = 1024;

__device__ __forceinline__ uint32_t fkey(float x) {
  uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// k-th smallest (0-based) 64-bit key among the CTA's keys produced by get(i) for i in
// [0, n) where valid(i); 8-bit radix selection with a 256-bin shared histogram.
template <class Get>
__device__ unsigned long long block_select(int n, int k, int nbits, Get get, uint32_t *s_dig,
                                           uint32_t *s_scan, unsigned long long *s_pre,
                                           int *s_rank) {
  const int t = threadIdx.x;
  if (t == 0) {
    *s_pre = 0ULL;
    *s_rank = k;
  }
  __syncthreads();
  for (int d = (nbits + 7) / 8 - 1; d >= 0; --d) {
    s_dig[t] = 0;
    __syncthreads();
    const int sh = 8 * d;
    const unsigned long long pre = *s_pre;
    for (int i = t; i < n; i += kFT) {
      unsigned long long key;
      if (!get(i, key)) continue;
      unsigned long long hk = (sh + 8 >= 64) ? 0ULL : key >> (sh + 8);
      unsigned long long hp = (sh + 8 >= 64) ? 0ULL : pre >> (sh + 8);
      if (hk == hp) atomicAdd(&s_dig[(key >> sh) & 0xffu], 1u);
    }
    __syncthreads();
    // inclusive scan of the 256 digit counts: warp scans, then the 8 warp totals
    const uint32_t c = s_dig[t];
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
      if ((t & 31) >= o) incl += x;
    }
    if ((t & 31) == 31) s_scan[t >> 5] = incl;
    __syncthreads();
    for (int w = 0; w < (t >> 5); ++w) incl += s_scan[w];
    const uint32_t excl = incl - c;
    const int rk = *s_rank;
    __syncthreads();
    if ((int)excl <= rk && rk < (int)incl) {
      *s_pre = pre | ((unsigned long long)t << sh);
      *s_rank = rk - (int)excl;
    }
    __syncthreads();
  }
  return *s_pre;
}

// Eq. skewgaus and its gradient with respect to (A, Rbar, sigma, s).
__device__ __forceinline__ double sg_eval(double x, const double *p, double *g) {
  const double A = p[0], mu = p[1], sg = p[2], s = p[3];
  const double d = x - mu;
  if (d < 0.0) {
    const double w = s * sg;
    const double e = exp(-d * d / (2.0 * w * w));
    if (g) {
      g[0] = e;
      g[1] = A * e * d / (w * w);
      g[2] = A * e * d * d / (w * w * sg);
      g[3] = A * e * d * d / (w * w * s);
    }
    return A * e;
  }
  const double e = exp(-d * d / (2.0 * sg * sg));
  if (g) {
    g[0] = e;
    g[1] = A * e * d / (sg * sg);
    g[2] = A * e * d * d / (sg * sg * sg);
    g[3] = 0.0;
  }
  return A * e;
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Solves (JtJ + lambda diag(JtJ)) x = b by Gaussian elimination with partial pivoting;
// jj holds the upper triangle of JtJ row by row.
__device__ bool solve4(const double *jj, double lambda, const double *b, double *x) {
  double a[4][5];
  int q = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = i; j < 4; ++j) {
      a[i][j] = a[j][i] = jj[q++];
    }
  for (int i = 0; i < 4; ++i) {
    a[i][i] = a[i][i] + lambda * a[i][i];
    a[i][4] = b[i];
  }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < 5; ++j) {
        double tt = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = tt;
      }
    for (int r = c + 1; r < 4; ++r) {
      double f = a[r][c] / a[c][c];
      for (int j = c; j < 5; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int r = 3; r >= 0; --r) {
    double s = a[r][4];
    for (int j = r + 1; j < 4; ++j) s -= a[r][j] * x[j];
    x[r] = s / a[r][r];
  }
  return true;
}

// R of every slot of the halos with szlo < N_H <= szhi, in slot order (the selections
// below read it many times).
__global__ void k_gather_r(const float4 *__restrict__ v, const float *__restrict__ R, int64_t nhp,
                           const uint32_t *__restrict__ hid, const uint32_t *__restrict__ hoff,
                           uint32_t szlo, uint32_t szhi, float *__restrict__ Rs) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nhp) return;
  const uint32_t h = hid[m], nh = hoff[h + 1] - hoff[h];
  if (nh > szlo && nh <= szhi) Rs[m] = R[__float_as_int(v[m].w)];
}

// The key of rank k - 1 given the key `a` of rank k (0-based, k >= 1) among the valid
// keys: `a` itself if fewer than k keys lie below it (a run of equal keys), else the
// largest key below `a`. One pass instead of a second selection.
template <class Get>
__device__ unsigned long long block_prev_rank(int n, int k, unsigned long long a, Get get,
                                              unsigned long long *s_max, int *s_cnt) {
  const int t = threadIdx.x;
  if (t == 0) {
    *s_max = 0ULL;
    *s_cnt = 0;
  }
  __syncthreads();
  unsigned long long mx = 0ULL;
  int c = 0;
  for (int i = t; i < n; i += kFT) {
    unsigned long long key;
    if (!get(i, key) || key >= a) continue;
    ++c;
    mx = key > mx ? key : mx;
  }
  atomicAdd(s_cnt, c);
  atomicMax(s_max, mx);
  __syncthreads();
  const unsigned long long r = *s_cnt < k ? a : *s_max;
  __syncthreads();
  return r;
}

}  // namespace

__global__ void __launch_bounds__(kFT, VR_FIT_MINB) k_ell_fit(const uint32_t *__restrict__ hoff,
                                                 const uint32_t *__restrict__ horder,
                                                 const uint32_t *__restrict__ nodeoff,
                                                 int64_t first, int64_t last,
                                                 const float4 *__restrict__ v,
                                                 const float *__restrict__ Rs, int nb_min,
                                                 int nb_max, int iters, double *__restrict__ hs,
                                                 float *__restrict__ ell, uint32_t szlo,
                                                 uint32_t szhi) {
  __shared__ uint32_t s_dig[256];
  __shared__ uint32_t s_scan[256];
  __shared__ unsigned long long s_pre;
  __shared__ int s_rank;
  __shared__ int s_cnt[kMaxFitBins];
  __shared__ int s_n;
  __shared__ double s_par[8];
  __shared__ unsigned long long s_max;
  __shared__ int s_lt;
  if (first + (int64_t)blockIdx.x >= last) return;
  const int64_t h = horder[first + blockIdx.x];  // largest halos first
  if (nodeoff[h + 1] == nodeoff[h]) return;  // not searched
  const uint32_t hb = hoff[h], he = hoff[h + 1];
  const int nh = (int)(he - hb);
  if (he - hb <= szlo || he - hb > szhi) return;  // another launch's halo
  const int t = threadIdx.x;
  auto rval = [&](int i) { return Rs[hb + i]; };
  // number of finite values
  if (t == 0) s_n = 0;
  __syncthreads();
  int c = 0;
  for (int i = t; i < nh; i += kFT) c += isfinite(rval(i)) ? 1 : 0;
  atomicAdd(&s_n, c);
  __syncthreads();
  const int n = s_n;
  double *row = hs + h * VR_HALO_COLS;
  if (n < 2) {
    if (t == 0) {
      row[VR_H_RBAR] = NAN;
      row[VR_H_SIGR] = NAN;
    }
    for (int i = t; i < nh; i += kFT) ell[__float_as_int(v[hb + i].w)] = NAN;
    return;
  }
  auto getf = [&](int i, unsigned long long &key) {
    float x = rval(i);
    if (!isfinite(x)) return false;
    key = fkey(x);
    return true;
  };
  double med;
  {
    const unsigned long long ka = block_select(nh, n / 2, 32, getf, s_dig, s_scan, &s_pre, &s_rank);
    float a = fkey_inv((uint32_t)ka);
    if (n & 1) {
      med = (double)a;
    } else {
      float b = fkey_inv((uint32_t)block_prev_rank(nh, n / 2, ka, getf, &s_max, &s_lt));
      med = 0.5 * ((double)b + (double)a);
    }
  }
  auto getd = [&](int i, unsigned long long &key) {
    float x = rval(i);
    if (!isfinite(x)) return false;
    key = (unsigned long long)__double_as_longlong(fabs(__dsub_rn((double)x, med)));
    return true;
  };
  double mad;
  {
    const unsigned long long ka = block_select(nh, n / 2, 64, getd, s_dig, s_scan, &s_pre, &s_rank);
    double a = __longlong_as_double((long long)ka);
    if (n & 1) {
      mad = a;
    } else {
      double b = __longlong_as_double((long long)block_prev_rank(nh, n / 2, ka, getd, &s_max, &s_lt));
      mad = 0.5 * (b + a);
    }
    mad = __dmul_rn(1.4826, mad);
  }
  if (!(mad > 0.0)) {
    if (t == 0) {
      row[VR_H_RBAR] = med;
      row[VR_H_SIGR] = NAN;
    }
    for (int i = t; i < nh; i += kFT) ell[__float_as_int(v[hb + i].w)] = NAN;
    return;
  }
  int nb = 0;
  while ((long long)nb * nb < n) ++nb;  // ceil(sqrt(n))
  if (nb < nb_min) nb = nb_min;
  if (nb > nb_max) nb = nb_max;
  const double lo = __dsub_rn(med, __dmul_rn(6.0, mad));
  const double width = __ddiv_rn(__dmul_rn(12.0, mad), (double)nb);
  for (int b = t; b < nb; b += kFT) s_cnt[b] = 0;
  __syncthreads();
  for (int i = t; i < nh; i += kFT) {
    float x = rval(i);
    if (!isfinite(x)) continue;
    double f = floor(__ddiv_rn(__dsub_rn((double)x, lo), width));
    if (f >= 0.0 && f < (double)nb) atomicAdd(&s_cnt[(int)f], 1);
  }
  __syncthreads();
  if (t < 32) {
    const int lane = t;
    int mode = 0;
    for (int b = 1; b < nb; ++b)
      if (s_cnt[b] > s_cnt[mode]) mode = b;
    double p[4] = {(double)s_cnt[mode], __dadd_rn(lo, __dmul_rn((double)mode + 0.5, width)), mad, 1.0};
    auto center = [&](int b) { return __dadd_rn(lo, __dmul_rn((double)b + 0.5, width)); };
    double cost = 0.0;
    for (int b = lane; b < nb; b += 32) {
      double r = (double)s_cnt[b] - sg_eval(center(b), p, nullptr);
      cost += r * r;
    }
    cost = warp_sum(cost);
    double lambda = 1e-3;
    // J^T J and J^T r depend on p alone: after a rejected step (p unchanged) the sums of
    // the previous iteration are reused as they are
    double jj[10], jr[4];
    bool fresh = true;
    for (int it = 0; it < iters; ++it) {
      if (fresh) {
        for (int q = 0; q < 10; ++q) jj[q] = 0.0;
        for (int i = 0; i < 4; ++i) jr[i] = 0.0;
        for (int b = lane; b < nb; b += 32) {
          double g[4];
          double r = (double)s_cnt[b] - sg_eval(center(b), p, g);
          int q = 0;
          for (int i = 0; i < 4; ++i) {
            jr[i] += g[i] * r;
            for (int j = i; j < 4; ++j) jj[q++] += g[i] * g[j];
          }
        }
        for (int q = 0; q < 10; ++q) jj[q] = warp_sum(jj[q]);
        for (int i = 0; i < 4; ++i) jr[i] = warp_sum(jr[i]);
        fresh = false;
      }
      double delta[4] = {0, 0, 0, 0};
      bool ok = solve4(jj, lambda, jr, delta);
      double qp[4];
      for (int i = 0; i < 4; ++i) qp[i] = p[i] + (ok ? delta[i] : 0.0);
      double ncost = INFINITY;
      if (ok && qp[2] > 0.0 && qp[3] > 0.0) {
        bool same = true;  // a step lost to rounding: the cost at qp is the cost at p
        for (int i = 0; i < 4; ++i) same &= __double_as_longlong(qp[i]) == __double_as_longlong(p[i]);
        if (same) {
          ncost = cost;
        } else {
          ncost = 0.0;
          for (int b = lane; b < nb; b += 32) {
            double r = (double)s_cnt[b] - sg_eval(center(b), qp, nullptr);
            ncost += r * r;
          }
          ncost = warp_sum(ncost);
        }
      }
      if (ncost < cost) {
        double rel = (cost - ncost) / cost;
        for (int i = 0; i < 4; ++i) p[i] = qp[i];
        cost = ncost;
        fresh = true;
        lambda /= 10.0;
        if (rel < 1e-15) break;
      } else {
        lambda *= 10.0;
        if (lambda > 1e30) break;
      }
    }
    if (lane == 0) {
      s_par[0] = p[1];
      s_par[1] = p[2];
      row[VR_H_RBAR] = p[1];
      row[VR_H_SIGR] = p[2];
    }
  }
  __syncthreads();
  const double rbar = s_par[0], sigr = s_par[1];
  for (int i = t; i < nh; i += kFT) {
    const int pi = __float_as_int(v[hb + i].w);
    ell[pi] = (float)(((double)Rs[hb + i] - rbar) / sigr);
  }
}

vr_status run_fit(vr_ctx *ctx, const HaloSeg &g, const Background &bg, const vr_params *p,
                  const float *R, double *halo_stats, float *ell, cudaStream_t s, const uint32_t *hoff_host,
                  uint32_t szlo, uint32_t szhi) {
  if (g.H == 0) return VR_OK;
  if (p->fit_nbins_max > kMaxFitBins)
    return set_error(ctx, VR_ERR_INVALID_ARG, "fit_nbins_max above %d", kMaxFitBins);
  float *Rs = reinterpret_cast<float *>(g.scratch_u32_a);  // [n + 1] words, unused here
  if (hoff_host) szlo = 0, szhi = 0xffffffffu;
  k_gather_r<<<grid_for(g.NHP, 256), 256, 0, s>>>(g.v, R, g.NHP, g.hid, g.hoff, szlo, szhi, Rs);
  VR_LAUNCHED(ctx, "k_gather_r");
  if (hoff_host) {  // one launch per searched halo, in the size order
    std::vector<uint32_t> ord(g.H);
    VR_CUDA(ctx, cudaMemcpyAsync(ord.data(), g.horder, g.H * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VR_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < g.H; ++i) {
      if (hoff_host[ord[i] + 1] - hoff_host[ord[i]] < (uint32_t)p->nsearch_min) continue;
      k_ell_fit<<<1, kFT, 0, s>>>(g.hoff, g.horder, bg.nodeoff, i, i + 1, g.v, Rs, p->fit_nbins_min,
                                  p->fit_nbins_max, p->fit_iters, halo_stats, ell, 0u, 0xffffffffu);
      VR_LAUNCHED(ctx, "k_ell_fit");
    }
    return VR_OK;
  }
  VR_TIMED(ctx, "ell_fit", s, k_ell_fit<<<(unsigned)g.H, kFT, 0, s>>>(g.hoff, g.horder, bg.nodeoff, 0, g.H, g.v, Rs,
                                                                       p->fit_nbins_min, p->fit_nbins_max,
                                                                       p->fit_iters, halo_stats, ell, szlo,
                                                                       szhi));
  VR_LAUNCHED(ctx, "k_ell_fit");
  return VR_OK;
}

}  // namespace vr
