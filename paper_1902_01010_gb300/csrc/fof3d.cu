// 3D friends-of-friends over a periodic lattice box (Sec. 2.1, Eq. fof3d).
//
// GB300 design:
//  1. sub-cells of side S = floor(sqrt((link_d2 - 1) / 3)) + 1, the largest side whose
//     diagonal is shorter than the linking length: all members of a sub-cell are linked
//     to each other, so each member is hooked straight below the sub-cell's first
//     particle without any distance test;
//  2. link cells of 2 sub-cells per axis (side 2S >= linking length; the last link cell
//     of each axis takes the 3 or 4 leftover sub-cells, so no link cell is thinner than
//     the linking length across the periodic edge): every linked pair lies in the same or
//     an adjacent link cell. Particles are ordered by (Morton code of the link cell,
//     position of the sub-cell inside it) with the library's radix sort, which makes
//     every sub-cell, link cell and coarse cell (2^q link cells per axis) one contiguous
//     run;
//  3. a dense table over coarse cells gives each link-cell lookup in one load plus a
//     short binary search; before it, one bit per link cell (the grid folded to 2^m
//     cells per axis, 8 n bits or more, 4x4x4 cells per 64-bit word) tells most empty
//     neighbours apart in one cached load: a clear bit means an empty link cell, a set
//     bit (the cell, or one folded onto it, holds particles) goes on to the lookup;
//  4. link cells are listed as runs of sub-cells; a warp takes 32 consecutive link cells,
//     each lane screening one against the bitmap of its 13 forward neighbours. A lane
//     whose link cell is one sub-cell links it on its own (a lookup and the sub-cell
//     pairs per occupied neighbour); a link cell of several sub-cells is taken by the
//     whole warp: lanes 0-12 find the 13 neighbours at once, the neighbour sub-cells are
//     gathered in shared memory, and the (own, neighbour) and (own, own) sub-cell pairs
//     are spread over the lanes. A pair of sub-cells with at most 4 member pairs is
//     tested particle by particle; otherwise box distances settle most pairs (none
//     linked / all linked), the rest are skipped when A and B are already in one
//     component, else particles are tested until a linked pair is found. Linked
//     sub-cells are merged by a lock-free union-find (atomicCAS hooks the larger root
//     under the smaller; finds halve paths);
//  5. labels are the minimum original index of each component (atomicMin per root).
// The grid is not a power of two per axis: the last sub-cell of each axis may be
// partial, and box tests use each cell's true extent across the periodic edge.
// Positions are gathered once into a 16-byte int4 stream in sorted order.
#include "vr_internal.cuh"
#include "vr_workspace.h"
#include "unionfind.cuh"

namespace vr {

namespace {

constexpr uint32_t kEmpty = 0xffffffffu;

struct FofGeom {
  int S;        // sub-cell side (lattice units)
  int G;        // sub-cells per axis (last one partial)
  int GL;       // link cells per axis: 2 sub-cells each, the last one 3 or 4
  int bl;       // bits per axis of link-cell coordinates
  int q;        // coarse cell = 2^q link cells per axis
  int64_t ncoarse;
  int om;       // occupancy bitmap: link cells folded to 2^om per axis
};

// Coarse table size: at most 8^m entries with 8^m <= max(n, 4096), m <= 9 (2^27).
int coarse_bits_per_axis(int64_t n) {
  int m = 4;
  while (m < 9 && (1LL << (3 * (m + 1))) <= n) ++m;
  return m;
}

// Occupancy bitmap: 2^(3m) bits, the smallest m >= 4 with 2^(3m) >= 8 n, m <= 11.
int occ_bits_per_axis(int64_t n) {
  int m = 4;
  while (m < 11 && (1LL << (3 * m)) < 8 * n) ++m;
  return m;
}

int64_t occ_words(int om) { return 1LL << (3 * om - 6); }

int64_t isqrt64(int64_t x) {
  int64_t r = (int64_t)sqrt((double)x);
  while (r * r > x) --r;
  while ((r + 1) * (r + 1) <= x) ++r;
  return r;
}

FofGeom fof_geom(int64_t link_d2, int64_t n) {
  FofGeom g;
  g.S = (int)isqrt64((link_d2 - 1) / 3) + 1;  // 3 (S-1)^2 <= link_d2 - 1 < link_d2
  g.G = (int)((kLattice + g.S - 1) / g.S);
  g.GL = (g.G - 1) / 2;
  g.bl = 0;
  while ((1 << g.bl) < g.GL) ++g.bl;
  if (g.bl == 0) g.bl = 1;
  int m = coarse_bits_per_axis(n);
  g.q = g.bl - m > 0 ? g.bl - m : 0;
  g.ncoarse = 1LL << (3 * (g.bl - g.q));
  g.om = occ_bits_per_axis(n);
  return g;
}

struct FofBufs {
  u64 *k0, *k1;
  uint32_t *v0, *v1;
  int4 *posS;
  int *parent;
  int *minidx;
  uint32_t *head;     // 1 at the first particle of each sub-cell, then its exclusive scan
  uint32_t *sc_start; // first sorted index of each sub-cell
  uint32_t *cstart, *cend;
  unsigned long long *occ;  // occupancy bitmap of the link cells
  void *scratch;      // radix sort / scan scratch
};

FofBufs fof_carve(Arena &ar, int64_t n, int64_t ncoarse, int om) {
  FofBufs b;
  b.k0 = ar.take<u64>(n + 1);  // n + 1: the spare one holds 2 n + 2 link-cell words
  b.k1 = ar.take<u64>(n + 1);
  b.v0 = ar.take<uint32_t>(n);
  b.v1 = ar.take<uint32_t>(n);
  b.posS = ar.take<int4>(n);
  b.parent = ar.take<int>(n);
  b.minidx = ar.take<int>(n);
  b.head = ar.take<uint32_t>(n + 1);
  b.sc_start = ar.take<uint32_t>(n + 1);
  b.cstart = ar.take<uint32_t>(ncoarse);
  b.cend = ar.take<uint32_t>(ncoarse);
  b.occ = ar.take<unsigned long long>(occ_words(om));
  size_t a = radix_scratch_bytes<u64>(n), c = scan_scratch_bytes<uint32_t>(n + 1);
  b.scratch = ar.take<char>(a > c ? a : c);
  return b;
}

// Sub-cell c of an axis lies in link cell min(c / 2, GL - 1) at position c - 2 * that.
__device__ __forceinline__ uint32_t link_of(uint32_t c, int GL) {
  uint32_t l = c >> 1;
  return l < (uint32_t)GL ? l : (uint32_t)GL - 1u;
}

// Word and bit of link cell (x, y, z) in the occupancy bitmap: coordinates taken modulo
// 2^om, then 4x4x4 cells per 64-bit word, words in x-fastest order.
__device__ __forceinline__ void occ_pos(uint32_t x, uint32_t y, uint32_t z, int om, u64 &word,
                                        uint32_t &bit) {
  const uint32_t M = (1u << om) - 1u;
  x &= M;
  y &= M;
  z &= M;
  const int b = om - 2;
  word = (u64)(x >> 2) | ((u64)(y >> 2) << b) | ((u64)(z >> 2) << (2 * b));
  bit = (x & 3u) | ((y & 3u) << 2) | ((z & 3u) << 4);
}

__device__ __forceinline__ uint32_t compact3(u64 x);

// Sort key: Morton code of the link cell << 6 | 2-bit sub-cell position per axis. Link
// cells (key >> 6) and coarse cells are its prefixes.
__global__ void k_fof_keys(const int32_t *__restrict__ pos, int64_t n, int S, int GL,
                           u64 *__restrict__ keys, uint32_t *__restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // masking keeps every cell index in range even for positions outside [0, 2^21)
  const uint32_t m = (uint32_t)kLattice - 1u;
  uint32_t x = ((uint32_t)pos[3 * i] & m) / (uint32_t)S,
           y = ((uint32_t)pos[3 * i + 1] & m) / (uint32_t)S,
           z = ((uint32_t)pos[3 * i + 2] & m) / (uint32_t)S;
  uint32_t lx = link_of(x, GL), ly = link_of(y, GL), lz = link_of(z, GL);
  keys[i] = (morton3(lx, ly, lz) << 6) | ((u64)(x - 2 * lx) << 4) | ((u64)(y - 2 * ly) << 2) |
            (u64)(z - 2 * lz);
  vals[i] = (uint32_t)i;
}


__global__ void k_fof_prepare(const int32_t *__restrict__ pos, const u64 *__restrict__ keyS,
                              const uint32_t *__restrict__ orig, int64_t n, int cshift,
                              int4 *__restrict__ posS, int *__restrict__ minidx,
                              uint32_t *__restrict__ head, uint32_t *__restrict__ cstart,
                              uint32_t *__restrict__ cend, unsigned long long *__restrict__ occ,
                              int om) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  if (p == n) {
    head[n] = 0;
    return;
  }
  int64_t i = orig[p];
  const uint32_t m = (uint32_t)kLattice - 1u;
  posS[p] = make_int4((int)((uint32_t)pos[3 * i] & m), (int)((uint32_t)pos[3 * i + 1] & m),
                      (int)((uint32_t)pos[3 * i + 2] & m), (int)i);
  minidx[p] = 0x7fffffff;
  u64 k = keyS[p];
  head[p] = (p == 0 || keyS[p - 1] != k) ? 1u : 0u;
  if (p == 0 || (keyS[p - 1] >> 6) != (k >> 6)) {  // first particle of its link cell
    u64 w;
    uint32_t bit;
    occ_pos(compact3(k >> 6), compact3(k >> 7), compact3(k >> 8), om, w, bit);
    atomicOr(&occ[w], 1ull << bit);
  }
  u64 c = k >> cshift;
  if (p == 0 || (keyS[p - 1] >> cshift) != c) cstart[c] = (uint32_t)p;
  if (p == n - 1 || (keyS[p + 1] >> cshift) != c) cend[c] = (uint32_t)(p + 1);
}

// excl[p] = number of sub-cell starts before p (exclusive scan of the start flags).
// Writes the sub-cell id of every sorted particle and the start of every sub-cell
// (sc_start[nsc] = n).
__global__ void k_fof_subcells(const u64 *__restrict__ keyS, const uint32_t *__restrict__ excl,
                               int64_t n, uint32_t *__restrict__ sid,
                               uint32_t *__restrict__ sc_start) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  bool first = (p == 0 || keyS[p - 1] != keyS[p]);
  uint32_t id = excl[p] - (first ? 0u : 1u);
  sid[p] = id;
  if (first) sc_start[id] = (uint32_t)p;
  if (p == n - 1) sc_start[id + 1] = (uint32_t)n;
}

// Every member of a sub-cell is hooked directly below the sub-cell's first particle:
// all members are within the linking length of each other (3 (S-1)^2 < link_d2).
__global__ void k_fof_hook(const uint32_t *__restrict__ sid, const uint32_t *__restrict__ sc_start,
                           int64_t n, int *__restrict__ parent) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  parent[p] = (int)sc_start[sid[p]];
}

__device__ __forceinline__ long long d2_periodic(int4 a, int4 b) {
  long long dx = min_image(a.x - b.x), dy = min_image(a.y - b.y), dz = min_image(a.z - b.z);
  return dx * dx + dy * dy + dz * dz;
}

// Forward half of the 26-neighbourhood: (dz > 0) or (dz == 0 and dy > 0) or
// (dz == 0, dy == 0, dx > 0). With >= 3 link cells per axis each unordered pair of
// adjacent cells is visited from exactly one side.
__constant__ signed char c_fwd[13][3] = {
    {1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1},
    {-1, 0, 1}, {0, 0, 1},  {1, 0, 1},  {-1, 1, 1}, {0, 1, 1},   {1, 1, 1}};

// Sub-cell extent along one axis: [c S, min((c + 1) S, 2^21) - 1].
__device__ __forceinline__ void cell_span(int c, int S, int &lo, int &hi) {
  lo = c * S;
  hi = min(lo + S, (int)kLattice) - 1;
}

// Gap and farthest separation between interval A = [alo, ahi] and interval B = [blo, bhi]
// taken in B's periodic image nearest to A. Returns B's shift into A's frame.
__device__ __forceinline__ int axis_gap(int alo, int ahi, int blo, int bhi, long long &gap,
                                        long long &far) {
  int shift = min_image(blo - alo) - (blo - alo);
  int b0 = blo + shift, b1 = bhi + shift;
  long long g = 0;
  if (b0 > ahi) g = (long long)b0 - ahi;
  else if (alo > b1) g = (long long)alo - b1;
  long long f1 = (long long)b1 - alo, f2 = (long long)ahi - b0;
  gap = g;
  far = f1 > f2 ? f1 : f2;
  return shift;
}

__device__ __forceinline__ uint32_t compact3(u64 x) {  // every third bit of x, from bit 0
  x &= 0x1249249249249249ULL;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
  x = (x ^ (x >> 32)) & 0x1fffffULL;
  return (uint32_t)x;
}


// Pairs of sub-cells with at most this many member pairs are tested particle by particle,
// without the box tests.
constexpr uint32_t kDirectPairs = 4;

// Links sub-cell A = [a0, a1) with sub-cell B = [b0, b1) (sub-cell coordinates bc) if any
// pair of their members is within the linking length.
__device__ __forceinline__ void link_subcells(const int4 *__restrict__ posS, int *parent,
                                              uint32_t a0, uint32_t a1, const int *alo,
                                              const int *ahi, uint32_t b0, uint32_t b1,
                                              uint32_t bcx, uint32_t bcy, uint32_t bcz, int S,
                                              long long T) {
  const uint32_t bc[3] = {bcx, bcy, bcz};
  if ((a1 - a0) * (b1 - b0) <= kDirectPairs) {
    for (uint32_t a = a0; a < a1; ++a) {
      const int4 xa = posS[a];
      for (uint32_t b = b0; b < b1; ++b) {
        if (d2_periodic(xa, posS[b]) < T) {
          uf_unite(parent, (int)a0, (int)b0);
          return;
        }
      }
    }
    return;
  }
  long long mind = 0, maxd = 0;
  int bl[3], bh[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int lo, hi;
    cell_span((int)bc[k], S, lo, hi);
    long long gp, fr;
    int sh = axis_gap(alo[k], ahi[k], lo, hi, gp, fr);
    bl[k] = lo + sh;
    bh[k] = hi + sh;
    mind += gp * gp;
    maxd += fr * fr;
  }
  if (mind >= T) return;  // no pair can link
  if (maxd < T) {         // every pair links
    uf_unite(parent, (int)a0, (int)b0);
    return;
  }
  if (uf_find(parent, (int)a0) == uf_find(parent, (int)b0)) return;
  for (uint32_t a = a0; a < a1; ++a) {
    const int4 xa = posS[a];  // inside A's box, so no wrap in A's frame
    long long gx = xa.x < bl[0] ? bl[0] - xa.x : (xa.x > bh[0] ? xa.x - bh[0] : 0);
    long long gy = xa.y < bl[1] ? bl[1] - xa.y : (xa.y > bh[1] ? xa.y - bh[1] : 0);
    long long gz = xa.z < bl[2] ? bl[2] - xa.z : (xa.z > bh[2] ? xa.z - bh[2] : 0);
    if (gx * gx + gy * gy + gz * gz >= T) continue;
    for (uint32_t b = b0; b < b1; ++b) {
      if (d2_periodic(xa, posS[b]) < T) {
        uf_unite(parent, (int)a0, (int)b0);
        return;
      }
    }
  }
}

// Sub-cell coordinates of sort key bk in link cell (lx, ly, lz): 2 l + the key's 2-bit
// position along each axis (three comma-separated values).
#define VR_SUB_OF(bk, lx, ly, lz)                                       \
  2u * (uint32_t)(lx) + (uint32_t)(((bk) >> 4) & 3u),                   \
      2u * (uint32_t)(ly) + (uint32_t)(((bk) >> 2) & 3u),               \
      2u * (uint32_t)(lz) + (uint32_t)((bk) & 3u)

// Link cells as runs of sub-cells: flag[A] = 1 at the first sub-cell A of each link cell
// (entries [0, n]; zero from nsc on), scanned in place into link-cell ids.
__global__ void k_fof_lcflags(const u64 *__restrict__ keyS, const uint32_t *__restrict__ sc_start,
                              const uint32_t *__restrict__ nsc_ptr, int64_t n,
                              uint32_t *__restrict__ flag) {
  const int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (A > n) return;
  const int64_t nsc = *nsc_ptr;
  uint32_t f = 0;
  if (A < nsc)
    f = (A == 0 || (keyS[sc_start[A - 1]] >> 6) != (keyS[sc_start[A]] >> 6)) ? 1u : 0u;
  flag[A] = f;
}

// After the scan (lcf[A] = link cell of a first sub-cell A, lcf[n] = number of link
// cells): lcfirst[c] = first sub-cell of link cell c, lcfirst[nlc] = nsc.
__global__ void k_fof_lcfirst(const u64 *__restrict__ keyS, const uint32_t *__restrict__ sc_start,
                              const uint32_t *__restrict__ nsc_ptr, int64_t n,
                              const uint32_t *__restrict__ lcf, uint32_t *__restrict__ lcfirst) {
  const int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (A > n) return;
  const int64_t nsc = *nsc_ptr;
  if (A > nsc) return;
  if (A == nsc) {
    lcfirst[lcf[A]] = (uint32_t)nsc;
    return;
  }
  if (A == 0 || (keyS[sc_start[A - 1]] >> 6) != (keyS[sc_start[A]] >> 6))
    lcfirst[lcf[A]] = (uint32_t)A;
}

constexpr int kLW = 8;       // warps per block of the link-cell kernel
constexpr int kLCap = 128;   // neighbour sub-cells a warp holds per round
constexpr int kLMaxSub = 64; // sub-cells of one link cell (4 x 4 x 4 at most)

__device__ __forceinline__ u64 pack_sub(uint32_t x, uint32_t y, uint32_t z) {
  return (u64)x | ((u64)y << 21) | ((u64)z << 42);
}

// Sub-cell pair (A, B) from packed sub-cell coordinates.
__device__ __forceinline__ void link_pair(const int4 *__restrict__ posS, int *parent, uint32_t a0,
                                          uint32_t a1, u64 ac, uint32_t b0, uint32_t b1, u64 bc,
                                          int S, long long T) {
  const u64 M = (1ull << 21) - 1ull;
  int alo[3], ahi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) cell_span((int)((ac >> (21 * k)) & M), S, alo[k], ahi[k]);
  link_subcells(posS, parent, a0, a1, alo, ahi, b0, b1, (uint32_t)(bc & M),
                (uint32_t)((bc >> 21) & M), (uint32_t)(bc >> 42), S, T);
}

// Persistent grid; each warp takes 32 consecutive link cells (sort order) at a time. Lane l
// screens link cell c0 + l against the occupancy bitmap of its 13 forward neighbours; a
// single-sub-cell link cell with occupied neighbours is linked by its lane alone; a link
// cell of several sub-cells is linked by the whole warp: the pairs of its own sub-cells,
// then, with lanes 0-12 each finding one forward link cell, every (own sub-cell,
// neighbour sub-cell) pair, the pairs spread over the lanes. Neighbour sub-cells are
// gathered kLCap at a time.
__global__ void __launch_bounds__(32 * kLW, 5) k_fof_link_w(
    const int4 *__restrict__ posS, const u64 *__restrict__ keyS, const uint32_t *__restrict__ sid,
    const uint32_t *__restrict__ sc_start, const uint32_t *__restrict__ lcf,
    const uint32_t *__restrict__ lcfirst, const uint32_t *__restrict__ cstart,
    const uint32_t *__restrict__ cend, const unsigned long long *__restrict__ occ, int om,
    int *parent, int64_t n, int S, int GL, int qshift, long long T) {
  __shared__ uint32_t s_b0[kLW][kLCap], s_b1[kLW][kLCap];
  __shared__ u64 s_bc[kLW][kLCap];
  __shared__ uint32_t s_a0[kLW][kLMaxSub + 1];
  __shared__ u64 s_ac[kLW][kLMaxSub];
  __shared__ int s_cnt[kLW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned FULL = 0xffffffffu;
  const int64_t nlc = lcf[n];
  for (int64_t c0 = ((int64_t)blockIdx.x * kLW + w) * 32; c0 < nlc; c0 += (int64_t)gridDim.x * kLW * 32) {
    // lane l screens link cell c0 + l: one sub-cell and no forward neighbour in the
    // occupancy bitmap means nothing to link
    int my_m = 0, mfx = 0, mfy = 0, mfz = 0;
    uint32_t my_s0 = 0, my_bits = 0;
    if (c0 + lane < nlc) {
      my_s0 = lcfirst[c0 + lane];
      my_m = (int)(lcfirst[c0 + lane + 1] - my_s0);
      const u64 k = keyS[sc_start[my_s0]] >> 6;
      mfx = (int)compact3(k);
      mfy = (int)compact3(k >> 1);
      mfz = (int)compact3(k >> 2);
#pragma unroll 1
      for (int q = 0; q < 13; ++q) {
        int x = mfx + c_fwd[q][0], y = mfy + c_fwd[q][1], z = mfz + c_fwd[q][2];
        x = x < 0 ? x + GL : (x >= GL ? x - GL : x);
        y = y < 0 ? y + GL : (y >= GL ? y - GL : y);
        z = z < 0 ? z + GL : (z >= GL ? z - GL : z);
        u64 ow;
        uint32_t ob;
        occ_pos((uint32_t)x, (uint32_t)y, (uint32_t)z, om, ow, ob);
        if ((__ldg(&occ[ow]) >> ob) & 1ull) my_bits |= 1u << q;
      }
    }
    if (my_m == 1 && my_bits != 0) {  // a single sub-cell: this lane links it on its own
      const uint32_t a0 = sc_start[my_s0], a1 = sc_start[my_s0 + 1];
      const u64 ak = keyS[a0];
      int alo[3], ahi[3];
      cell_span((int)(2u * (uint32_t)mfx + (uint32_t)((ak >> 4) & 3u)), S, alo[0], ahi[0]);
      cell_span((int)(2u * (uint32_t)mfy + (uint32_t)((ak >> 2) & 3u)), S, alo[1], ahi[1]);
      cell_span((int)(2u * (uint32_t)mfz + (uint32_t)(ak & 3u)), S, alo[2], ahi[2]);
#pragma unroll 1
      for (int q = 0; q < 13; ++q) {
        if (!((my_bits >> q) & 1u)) continue;
        int x = mfx + c_fwd[q][0], y = mfy + c_fwd[q][1], z = mfz + c_fwd[q][2];
        x = x < 0 ? x + GL : (x >= GL ? x - GL : x);
        y = y < 0 ? y + GL : (y >= GL ? y - GL : y);
        z = z < 0 ? z + GL : (z >= GL ? z - GL : z);
        const u64 key = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
        const u64 c = key >> qshift;
        uint32_t lo = __ldg(&cstart[c]);
        if (lo == kEmpty) continue;
        uint32_t hi = __ldg(&cend[c]);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((keyS[mid] >> 6) < key) lo = mid + 1; else hi = mid;
        }
        for (uint32_t j = lo; j < (uint32_t)n;) {
          const u64 bk = keyS[j];
          if ((bk >> 6) != key) break;
          const uint32_t j1 = sc_start[sid[j] + 1];
          link_subcells(posS, parent, a0, a1, alo, ahi, j, j1, VR_SUB_OF(bk, x, y, z), S, T);
          j = j1;
        }
      }
      my_bits = 0;
    }
    unsigned todo = __ballot_sync(FULL, my_m > 1 || my_bits != 0);
    while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const uint32_t s0 = __shfl_sync(FULL, my_s0, src);
    const int m = __shfl_sync(FULL, my_m, src);
    const int fx = __shfl_sync(FULL, mfx, src), fy = __shfl_sync(FULL, mfy, src),
              fz = __shfl_sync(FULL, mfz, src);
    const uint32_t bits = __shfl_sync(FULL, my_bits, src);
    for (int i = lane; i <= m; i += 32) {  // sub-cell starts (and the end of the last)
      const uint32_t p0 = sc_start[s0 + i];
      s_a0[w][i] = p0;
      if (i < m) {
        const u64 k = keyS[p0];
        s_ac[w][i] = pack_sub(VR_SUB_OF(k, fx, fy, fz));
      }
    }
    __syncwarp();
    for (int t = lane; t < m * m; t += 32) {  // own sub-cells, i < j
      const int i = t / m, j = t - i * m;
      if (j <= i) continue;
      link_pair(posS, parent, s_a0[w][i], s_a0[w][i + 1], s_ac[w][i], s_a0[w][j], s_a0[w][j + 1],
                s_ac[w][j], S, T);
    }
    uint32_t cur = (uint32_t)n;  // lane k < 13: next particle of forward link cell k
    u64 nkey = 0;
    int nx = 0, ny = 0, nz = 0;
    if (lane < 13 && ((bits >> lane) & 1u)) {
      nx = fx + c_fwd[lane][0];
      ny = fy + c_fwd[lane][1];
      nz = fz + c_fwd[lane][2];
      nx = nx < 0 ? nx + GL : (nx >= GL ? nx - GL : nx);
      ny = ny < 0 ? ny + GL : (ny >= GL ? ny - GL : ny);
      nz = nz < 0 ? nz + GL : (nz >= GL ? nz - GL : nz);
      {
        nkey = morton3((uint32_t)nx, (uint32_t)ny, (uint32_t)nz);
        const u64 c = nkey >> qshift;
        uint32_t lo = __ldg(&cstart[c]);
        if (lo != kEmpty) {
          uint32_t hi = __ldg(&cend[c]);
          while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((keyS[mid] >> 6) < nkey) lo = mid + 1; else hi = mid;
          }
          cur = lo;
        }
      }
    }
    while (__any_sync(FULL, cur < (uint32_t)n)) {
      if (lane == 0) s_cnt[w] = 0;
      __syncwarp();
      while (cur < (uint32_t)n) {
        const u64 bk = keyS[cur];
        if ((bk >> 6) != nkey) {
          cur = (uint32_t)n;
          break;
        }
        const int slot = atomicAdd(&s_cnt[w], 1);
        if (slot >= kLCap) break;  // full: this sub-cell waits for the next round
        const uint32_t j1 = sc_start[sid[cur] + 1];
        s_b0[w][slot] = cur;
        s_b1[w][slot] = j1;
        s_bc[w][slot] = pack_sub(VR_SUB_OF(bk, nx, ny, nz));
        cur = j1;
      }
      __syncwarp();
      const int nb = min(s_cnt[w], kLCap);
      for (int t = lane; t < m * nb; t += 32) {
        const int i = t / nb, j = t - i * nb;
        link_pair(posS, parent, s_a0[w][i], s_a0[w][i + 1], s_ac[w][i], s_b0[w][j], s_b1[w][j],
                  s_bc[w][j], S, T);
      }
      __syncwarp();
    }
    __syncwarp();  // s_a0 / s_ac are rewritten for the next link cell
    }
  }
}

// Root of every particle and the minimum original index per root. Neighbours in sort
// order mostly share a root, so the lanes of a warp with the same root combine their
// minimum first and one of them updates the root (one atomic per root and warp).
__global__ void k_fof_roots(int *parent, const int4 *__restrict__ posS, int64_t n,
                            int *__restrict__ minidx) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = p < n;
  int r = -1 - lane, w = 0x7fffffff;
  if (valid) {
    r = uf_find(parent, (int)p);
    parent[p] = r;
    w = posS[p].w;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, r);
  const int m = __reduce_min_sync(peers, w);
  if (valid && lane == __ffs(peers) - 1) atomicMin(&minidx[r], m);
}

// A fresh find: parent[p] written by k_fof_roots may since have been overwritten by a
// concurrent path-halving store with an older ancestor, so it is not read directly.
__global__ void k_fof_label(int *parent, const int4 *__restrict__ posS,
                            const int *__restrict__ minidx, int64_t n, int32_t *__restrict__ label) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  label[posS[p].w] = minidx[uf_find(parent, (int)p)];
}

}  // namespace

size_t ws_fof3d(int64_t n) {
  Arena ar;
  fof_carve(ar, n, 1LL << (3 * coarse_bits_per_axis(n)), occ_bits_per_axis(n));
  return ar.off;
}

}  // namespace vr

using namespace vr;

extern "C" vr_status vr_fof3d(vr_ctx *ctx, const int32_t *pos, int64_t n, int64_t link_d2,
                              int32_t *label, void *ws, size_t ws_bytes, void *stream) {
  if (!ctx) return VR_ERR_INVALID_ARG;
  if (n < 0 || n >= (1LL << 31))
    return set_error(ctx, VR_ERR_INVALID_ARG, "n must be in [0, 2^31)");
  if (n == 0) return VR_OK;
  if (!pos || !label || !ws) return set_error(ctx, VR_ERR_INVALID_ARG, "NULL pointer");
  if (link_d2 < 1 || link_d2 > (1LL << 38))
    return set_error(ctx, VR_ERR_INVALID_ARG, "link_d2 must be in [1, 2^38]");
  cudaStream_t s = (cudaStream_t)stream;
  FofGeom g = fof_geom(link_d2, n);
  Arena ar(ws, ws_bytes);
  FofBufs B = fof_carve(ar, n, g.ncoarse, g.om);
  vr_status st = check_ws(ctx, ar, ws_bytes);
  if (st != VR_OK) return st;
  const int T = 256;
  k_fof_keys<<<grid_for(n, T), T, 0, s>>>(pos, n, g.S, g.GL, B.k0, B.v0);
  VR_LAUNCHED(ctx, "k_fof_keys");
  int which = 0;
  VR_CUDA(ctx, radix_sort_pairs<u64>(B.k0, B.v0, B.k1, B.v1, n, 0, 6 + 3 * g.bl, B.scratch, s,
                                     &which));
  u64 *keyS = which ? B.k1 : B.k0;
  uint32_t *orig = which ? B.v1 : B.v0;
  VR_CUDA(ctx, cudaMemsetAsync(B.cstart, 0xff, g.ncoarse * sizeof(uint32_t), s));
  VR_CUDA(ctx, cudaMemsetAsync(B.occ, 0, occ_words(g.om) * sizeof(unsigned long long), s));
  const int qshift = 3 * g.q;      // link-cell key -> coarse-cell key
  const int cshift = 6 + qshift;   // sort key -> coarse-cell key
  k_fof_prepare<<<grid_for(n + 1, T), T, 0, s>>>(pos, keyS, orig, n, cshift, B.posS, B.minidx,
                                                 B.head, B.cstart, B.cend, B.occ, g.om);
  VR_LAUNCHED(ctx, "k_fof_prepare");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(B.head, B.head, n + 1, B.scratch, s));
  uint32_t *sid = which ? B.v0 : B.v1;  // the sort's spare value buffer
  k_fof_subcells<<<grid_for(n, T), T, 0, s>>>(keyS, B.head, n, sid, B.sc_start);
  VR_LAUNCHED(ctx, "k_fof_subcells");
  k_fof_hook<<<grid_for(n, T), T, 0, s>>>(sid, B.sc_start, n, B.parent);
  VR_LAUNCHED(ctx, "k_fof_hook");
  // link cells as runs of sub-cells, in the sort's spare key buffer (2 n + 2 words):
  // lcf [0, n] the scanned first-sub-cell flags, lcfirst [n + 1, 2 n + 2) the first
  // sub-cell of each link cell; the number of sub-cells, head[n], stays on the device
  uint32_t *lcf = reinterpret_cast<uint32_t *>(which ? B.k0 : B.k1);
  uint32_t *lcfirst = lcf + (n + 1);
  k_fof_lcflags<<<grid_for(n + 1, T), T, 0, s>>>(keyS, B.sc_start, B.head + n, n, lcf);
  VR_LAUNCHED(ctx, "k_fof_lcflags");
  VR_CUDA(ctx, exclusive_scan<uint32_t>(lcf, lcf, n + 1, B.scratch, s));
  k_fof_lcfirst<<<grid_for(n + 1, T), T, 0, s>>>(keyS, B.sc_start, B.head + n, n, lcf, lcfirst);
  VR_LAUNCHED(ctx, "k_fof_lcfirst");
  int sms = ctx->sm_count;
  if (sms <= 0) VR_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  VR_TIMED(ctx, "fof_link", s, k_fof_link_w<<<5 * sms, 32 * kLW, 0, s>>>(B.posS, keyS, sid, B.sc_start, lcf, lcfirst, B.cstart,
                                          B.cend, B.occ, g.om, B.parent, n, g.S, g.GL, qshift,
                                          (long long)link_d2));
  VR_LAUNCHED(ctx, "k_fof_link_w");
  k_fof_roots<<<grid_for(n, T), T, 0, s>>>(B.parent, B.posS, n, B.minidx);
  VR_LAUNCHED(ctx, "k_fof_roots");
  k_fof_label<<<grid_for(n, T), T, 0, s>>>(B.parent, B.posS, B.minidx, n, label);
  VR_LAUNCHED(ctx, "k_fof_label");
  return log_call(ctx, "vr_fof3d", n, VR_OK);
}
