// Device-wide primitives: exclusive prefix sum and a stable LSD radix sort of
// (key, value) pairs. Written for sm_103a: 256-thread blocks, warp-shuffle scans,
// __match_any_sync for stable in-tile ranking, coalesced round-major tile loads.
#include "vr_internal.cuh"

namespace vr {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T *total, T *s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = lane < (kScanThreads / 32) ? s_warp[lane] : T(0);
    T xi = warp_incl_scan(x);
    if (lane < (kScanThreads / 32)) s_warp[lane] = xi - x;
    if (lane == (kScanThreads / 32) - 1) s_warp[kScanThreads / 32] = xi;
  }
  __syncthreads();
  T r = inc - v + s_warp[w];
  *total = s_warp[kScanThreads / 32];
  __syncthreads();
  return r;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T *in, int64_t n, T *sums) {
  __shared__ T s_warp[kScanThreads / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  T acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = base + r * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  T tot;
  block_excl_scan(acc, &tot, s_warp);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const T *in, T *out, int64_t n,
                                                              const T *offs) {
  __shared__ T s_warp[kScanThreads / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  T run = offs ? offs[blockIdx.x] : T(0);
#pragma unroll 1
  for (int r = 0; r < kScanItems; ++r) {
    int64_t i = base + r * kScanThreads + threadIdx.x;
    T v = i < n ? in[i] : T(0);
    T tot;
    T ex = block_excl_scan(v, &tot, s_warp);
    if (i < n) out[i] = run + ex;
    run += tot;
  }
}

}  // namespace

template <class T>
size_t scan_scratch_bytes(int64_t n) {
  size_t b = 0;
  while (n > kScanTile) {
    n = ceil_div(n, kScanTile);
    b += ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
  }
  return b + 256;
}

template <class T>
cudaError_t exclusive_scan(const T *in, T *out, int64_t n, void *scratch, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n <= kScanTile) {
    k_scan_apply<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    count_launch();
    return cudaGetLastError();
  }
  int64_t nb = ceil_div(n, kScanTile);
  T *sums = (T *)scratch;
  char *rest = (char *)scratch + (((size_t)nb * sizeof(T) + 255) & ~(size_t)255);
  k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = exclusive_scan<T>(sums, sums, nb, rest, s);
  if (e != cudaSuccess) return e;
  k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  count_launch();
  return cudaGetLastError();
}

template size_t scan_scratch_bytes<uint32_t>(int64_t);
template size_t scan_scratch_bytes<unsigned long long>(int64_t);
template cudaError_t exclusive_scan<uint32_t>(const uint32_t *, uint32_t *, int64_t, void *,
                                              cudaStream_t);
template cudaError_t exclusive_scan<unsigned long long>(const unsigned long long *,
                                                        unsigned long long *, int64_t, void *,
                                                        cudaStream_t);

// ------------------------------------------------------------------ radix sort
namespace {

constexpr int kRadThreads = 256;
constexpr int kRadItems = 16;
constexpr int kRadTile = kRadThreads * kRadItems;  // 4096 keys per tile
constexpr int kRadWarps = kRadThreads / 32;

template <class K>
__global__ void __launch_bounds__(kRadThreads) k_radix_hist(const K *keys, int64_t n, int shift,
                                                             int64_t ntiles, uint32_t *counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRadTile;
#pragma unroll 4
  for (int r = 0; r < kRadItems; ++r) {
    int64_t i = base + r * kRadThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: every key's rank inside the tile (by digit, then tile order)
// is found round by round (kRadThreads keys per round: per-warp peer matching, then a
// prefix over the warps), the tile is reordered by digit in shared memory, and each
// digit's run is written out with consecutive threads on consecutive addresses.
template <class K>
__global__ void __launch_bounds__(kRadThreads) k_radix_scatter(const K *kin, const uint32_t *vin,
                                                                K *kout, uint32_t *vout, int64_t n,
                                                                int shift, int64_t ntiles,
                                                                const uint32_t *offs) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  K *s_key = reinterpret_cast<K *>(s_dyn);                                  // [kRadTile]
  uint32_t *s_val = reinterpret_cast<uint32_t *>(s_dyn + kRadTile * sizeof(K));  // [kRadTile]
  __shared__ uint32_t s_base[256];  // global offset of each digit's run of this tile
  __shared__ uint32_t s_loc[256];   // start of each digit's run inside the tile
  __shared__ uint32_t s_run[256];   // keys of each digit placed so far
  __shared__ uint32_t s_wcnt[kRadWarps][256];
  __shared__ uint32_t s_tot[kRadWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRadTile;
  const int tn = (int)min((int64_t)kRadTile, n - base);
  // this tile's count of digit t: the next entry of the digit-major, tile-minor scan
  const int64_t ix = (int64_t)t * ntiles + blockIdx.x;
  const uint32_t off = offs[ix];
  const uint32_t cnt = (ix + 1 < 256 * ntiles ? offs[ix + 1] : (uint32_t)n) - off;
  s_base[t] = off;
  s_run[t] = 0;
  // exclusive prefix of the counts over the 256 digits
  uint32_t incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) s_tot[w] = incl;
  __syncthreads();
  uint32_t pre = 0;
  for (int q = 0; q < w; ++q) pre += s_tot[q];
  s_loc[t] = pre + incl - cnt;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 1
  for (int r = 0; r < kRadItems; ++r) {
    for (int q = 0; q < kRadWarps; ++q) s_wcnt[q][t] = 0;
    __syncthreads();
    const int li = r * kRadThreads + t;
    const bool valid = li < tn;
    const K key = valid ? kin[base + li] : K(0);
    const uint32_t val = valid ? vin[base + li] : 0u;
    const uint32_t d = valid ? (uint32_t)(key >> shift) & 0xffu : 256u + lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lt);
    if (valid && rank == 0) s_wcnt[w][d] = __popc(peers);
    __syncthreads();
    uint32_t run = 0;  // thread t owns digit t: exclusive prefix over the warps
    for (int q = 0; q < kRadWarps; ++q) {
      const uint32_t c = s_wcnt[q][t];
      s_wcnt[q][t] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const uint32_t lp = s_loc[d] + s_run[d] + s_wcnt[w][d] + rank;
      s_key[lp] = key;
      s_val[lp] = val;
    }
    __syncthreads();
    s_run[t] += run;
  }
  __syncthreads();
  for (int li = t; li < tn; li += kRadThreads) {
    const K key = s_key[li];
    const uint32_t d = (uint32_t)(key >> shift) & 0xffu;
    const uint32_t pos = s_base[d] + (uint32_t)li - s_loc[d];
    kout[pos] = key;
    vout[pos] = s_val[li];
  }
}

}  // namespace

template <class K>
size_t radix_scratch_bytes(int64_t n) {
  int64_t ntiles = ceil_div(n > 0 ? n : 1, kRadTile);
  size_t c = (((size_t)ntiles * 256 * sizeof(uint32_t)) + 255) & ~(size_t)255;
  return c + scan_scratch_bytes<uint32_t>(ntiles * 256);
}

template <class K>
cudaError_t radix_sort_pairs(K *k0, uint32_t *v0, K *k1, uint32_t *v1, int64_t n, int begin_bit,
                             int end_bit, void *scratch, cudaStream_t s, int *which) {
  *which = 0;
  if (n <= 1 || end_bit <= begin_bit) return cudaSuccess;
  int64_t ntiles = ceil_div(n, kRadTile);
  {  // the tile buffers exceed the default 48 KB of shared memory for 64-bit keys
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kRadTile * (sizeof(K) + 4)));
    if (e != cudaSuccess) return e;
  }
  uint32_t *counts = (uint32_t *)scratch;
  char *scan_scr = (char *)scratch + ((((size_t)ntiles * 256 * sizeof(uint32_t)) + 255) & ~(size_t)255);
  K *kin = k0, *kout = k1;
  uint32_t *vin = v0, *vout = v1;
  int cur = 0;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    k_radix_hist<K><<<(unsigned)ntiles, kRadThreads, 0, s>>>(kin, n, shift, ntiles, counts);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan<uint32_t>(counts, counts, ntiles * 256, scan_scr, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<K><<<(unsigned)ntiles, kRadThreads, kRadTile * (sizeof(K) + 4), s>>>(
        kin, vin, kout, vout, n, shift, ntiles, counts);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    K *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
    cur ^= 1;
  }
  *which = cur;
  return cudaSuccess;
}

template size_t radix_scratch_bytes<uint32_t>(int64_t);
template size_t radix_scratch_bytes<unsigned long long>(int64_t);
template cudaError_t radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *,
                                                int64_t, int, int, void *, cudaStream_t, int *);
template cudaError_t radix_sort_pairs<unsigned long long>(unsigned long long *, uint32_t *,
                                                          unsigned long long *, uint32_t *, int64_t,
                                                          int, int, void *, cudaStream_t, int *);

}  // namespace vr
