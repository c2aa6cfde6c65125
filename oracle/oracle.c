/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, single-threaded FP64 restatement of the VELOCIraptor substructure
 * hot path (Elahi et al. 2019, "Hunting for Galaxies and Halos in simulations with
 * VELOCIraptor", Sec. 2.1-2.2). It exists to check the CUDA library; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it. It shares no code
 * with the CUDA library: both read the same synthetic arrays, nothing else.
 *
 * Conventions (readings of points the paper leaves open; each repeated where used):
 *  - positions are int32 on a periodic 2^21 lattice; separations use the minimum image
 *    per axis and squared separations are exact int64;
 *  - links are strict ("< 1", Eqs. fof3d, fof6d, linkingcriteria b) and tested as
 *    d^2 < T with an integer T;
 *  - group labels are the minimum particle index of the group;
 *  - ties in distance orderings are broken by particle index.
 *
 * Every function follows the definition it cites step by step; nothing is blocked,
 * fused or reordered beyond what that definition states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_L 2097152LL
#define OR_HALF 1048576LL
#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------- utilities */

/* Minimum image of a lattice difference d in (-2^21, 2^21) (periodic box, Sec. 2.1). */
static int64_t or_min_image(int64_t d) {
  if (d >= OR_HALF) d -= OR_L;
  else if (d < -OR_HALF) d += OR_L;
  return d;
}

static int64_t or_d2_periodic(const int32_t *a, const int32_t *b) {
  int64_t s = 0;
  for (int k = 0; k < 3; ++k) {
    int64_t d = or_min_image((int64_t)a[k] - (int64_t)b[k]);
    s += d * d;
  }
  return s;
}

/* Sequential union-find; the root of every set is its minimum element because the
 * larger root is always hung below the smaller one. */
static int64_t or_find(int64_t *parent, int64_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}
static void or_union(int64_t *parent, int64_t a, int64_t b) {
  int64_t ra = or_find(parent, a), rb = or_find(parent, b);
  if (ra == rb) return;
  if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
}

/* ---------------------------------------------------------- 3D FOF (Eq. fof3d) */

/* Brute force over all pairs: i, j linked iff |x_i - x_j|^2 < link_d2 (Eq. fof3d with
 * the strict inequality); label = minimum index of the connected component. */
int or_fof3d_brute(const int32_t *pos, int64_t n, int64_t link_d2, int32_t *label) {
  if (n < 0 || (n > 0 && (!pos || !label))) return 1;
  int64_t *parent = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  if (!parent) return 2;
  for (int64_t i = 0; i < n; ++i) parent[i] = i;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      if (or_d2_periodic(pos + 3 * i, pos + 3 * j) < link_d2) or_union(parent, i, j);
  for (int64_t i = 0; i < n; ++i) label[i] = (int32_t)or_find(parent, i);
  free(parent);
  return 0;
}

typedef struct {
  int64_t cell;
  int64_t idx;
} or_cellkey;

static int or_cmp_cellkey(const void *pa, const void *pb) {
  const or_cellkey *a = (const or_cellkey *)pa, *b = (const or_cellkey *)pb;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Same definition as or_fof3d_brute, with candidate pairs drawn from a grid of cells of
 * side g >= the linking length, so every linked pair lies in the same or adjacent cells. */
int or_fof3d(const int32_t *pos, int64_t n, int64_t link_d2, int32_t *label) {
  if (n < 0 || (n > 0 && (!pos || !label)) || link_d2 < 0) return 1;
  if (n == 0) return 0;
  /* cell side: smallest power of two with side^2 >= link_d2 */
  int64_t side = 1;
  while (side * side < link_d2 && side < OR_L) side <<= 1;
  int64_t g = OR_L / side; /* cells per axis */
  if (g < 3) return or_fof3d_brute(pos, n, link_d2, label);
  or_cellkey *keys = (or_cellkey *)malloc((size_t)n * sizeof(or_cellkey));
  int64_t *parent = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!keys || !parent) { free(keys); free(parent); return 2; }
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = pos[3 * i] / side, cy = pos[3 * i + 1] / side, cz = pos[3 * i + 2] / side;
    keys[i].cell = (cx * g + cy) * g + cz;
    keys[i].idx = i;
    parent[i] = i;
  }
  qsort(keys, (size_t)n, sizeof(or_cellkey), or_cmp_cellkey);
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = pos[3 * i] / side, cy = pos[3 * i + 1] / side, cz = pos[3 * i + 2] / side;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int64_t nx = (cx + dx + g) % g, ny = (cy + dy + g) % g, nz = (cz + dz + g) % g;
          int64_t c = (nx * g + ny) * g + nz;
          /* first key with cell >= c */
          int64_t lo = 0, hi = n;
          while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (keys[mid].cell < c) lo = mid + 1; else hi = mid;
          }
          for (int64_t p = lo; p < n && keys[p].cell == c; ++p) {
            int64_t j = keys[p].idx;
            if (j <= i) continue;
            if (or_d2_periodic(pos + 3 * i, pos + 3 * j) < link_d2) or_union(parent, i, j);
          }
        }
  }
  for (int64_t i = 0; i < n; ++i) label[i] = (int32_t)or_find(parent, i);
  free(keys);
  free(parent);
  return 0;
}

/* ------------------------------------------------------ halos and unwrapping */

/* Halos are 3D FOF groups with at least nmin members (Sec. 2.2, "N >= N_min").
 * Halo h is the h-th such group in increasing label order. offsets[H+1] and members
 * (particle indices, increasing within each halo) are written when non-NULL.
 * Returns H, or -1 on bad input. */
int64_t or_halos(const int32_t *label, int64_t n, int32_t nmin, int64_t *offsets,
                 int32_t *members) {
  if (n < 0 || (n > 0 && !label)) return -1;
  int64_t *count = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
  int64_t *hid = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  if (!count || !hid) { free(count); free(hid); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    if (label[i] < 0 || label[i] >= n) { free(count); free(hid); return -1; }
    count[label[i]]++;
  }
  int64_t H = 0, tot = 0;
  for (int64_t l = 0; l < n; ++l) {
    if (count[l] >= nmin && count[l] > 0) {
      hid[l] = H;
      if (offsets) offsets[H] = tot;
      tot += count[l];
      H++;
    } else {
      hid[l] = -1;
    }
  }
  if (offsets) offsets[H] = tot;
  if (members && offsets) {
    int64_t *fill = (int64_t *)calloc((size_t)(H ? H : 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
      int64_t h = hid[label[i]];
      if (h >= 0) members[offsets[h] + fill[h]++] = (int32_t)i;
    }
    free(fill);
  }
  free(count);
  free(hid);
  return H;
}

/* Positions of a halo's members in one periodic image: the minimum image of each
 * member relative to the halo's first (minimum-index) member. Valid while the halo
 * spans less than half the box per axis. upos is int64 [nh][3]. */
void or_unwrap(const int32_t *pos, const int32_t *members, int64_t nh, int64_t *upos) {
  if (nh <= 0) return;
  const int32_t *a = pos + 3 * (int64_t)members[0];
  for (int64_t m = 0; m < nh; ++m) {
    const int32_t *p = pos + 3 * (int64_t)members[m];
    for (int k = 0; k < 3; ++k)
      upos[3 * m + k] = (int64_t)a[k] + or_min_image((int64_t)p[k] - (int64_t)a[k]);
  }
}

/* ----------------------------------- local velocity density f_l (Sec. 2.2) */

typedef struct {
  int64_t d2;
  int64_t idx;
} or_nb;

static int or_nb_less(const or_nb *a, const or_nb *b) {
  return a->d2 < b->d2 || (a->d2 == b->d2 && a->idx < b->idx);
}

/* Rearranges a[0..n) so that a[0..k) are the k smallest by (d2, idx). Quickselect. */
static void or_select_nb(or_nb *a, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi && k > lo && k <= hi) {
    or_nb piv = a[(lo + hi) / 2];
    int64_t i = lo, j = hi;
    while (i <= j) {
      while (or_nb_less(&a[i], &piv)) ++i;
      while (or_nb_less(&piv, &a[j])) --j;
      if (i <= j) { or_nb t = a[i]; a[i] = a[j]; a[j] = t; ++i; --j; }
    }
    if (k <= j) hi = j;
    else if (k >= i) lo = i;
    else break;
  }
}

/* k-th smallest (1-based) of n doubles; the array is permuted. */
static double or_kth_double(double *a, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n - 1, t = k - 1;
  while (lo < hi) {
    double piv = a[(lo + hi) / 2];
    int64_t i = lo, j = hi;
    while (i <= j) {
      while (a[i] < piv) ++i;
      while (piv < a[j]) --j;
      if (i <= j) { double s = a[i]; a[i] = a[j]; a[j] = s; ++i; --j; }
    }
    if (t <= j) hi = j;
    else if (t >= i) lo = i;
    else return a[t];
  }
  return a[t];
}

/* Local velocity density of member k of a halo (Sec. 2.2; defaults N_v = 32,
 * N_se = 256, Table 1). Steps:
 *  1. the N_se nearest members in position (squared separation, then index), k itself
 *     included, N_se_eff = min(N_se, N_H);
 *  2. h = distance in velocity to the N_v-th nearest of that set (k counts as one);
 *  3. Epanechnikov estimate over the set, f_l = (1/N_se_eff) sum_j
 *     15/(8 pi h^3) (1 - |v_j - v_k|^2 / h^2) for |v_j - v_k| < h.
 * The 1/N_se_eff normalisation makes f_l a density of the N_se velocity sample.
 * upos int64 [nh][3] (one periodic image), vel float [n][3] indexed by members[].
 * scratch_nb must hold nh entries, scratch_r nse entries. */
static double or_velden_member(const int64_t *upos, const float *vel, const int32_t *members,
                               int64_t nh, int64_t k, int nse, int nv, or_nb *scratch_nb,
                               double *scratch_r) {
  int64_t nse_eff = nse < nh ? nse : nh;
  int64_t nv_eff = nv < nse_eff ? nv : nse_eff;
  for (int64_t m = 0; m < nh; ++m) {
    int64_t s = 0;
    for (int c = 0; c < 3; ++c) {
      int64_t d = upos[3 * m + c] - upos[3 * k + c];
      s += d * d;
    }
    scratch_nb[m].d2 = s;
    scratch_nb[m].idx = members[m];
  }
  or_select_nb(scratch_nb, nh, nse_eff);
  const float *vk = vel + 3 * (int64_t)members[k];
  for (int64_t q = 0; q < nse_eff; ++q) {
    const float *vj = vel + 3 * scratch_nb[q].idx;
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d = (double)vj[c] - (double)vk[c];
      s += d * d;
    }
    scratch_r[q] = s; /* squared velocity separation */
  }
  double r2[1024];
  double *tmp = nse_eff <= 1024 ? r2 : (double *)malloc((size_t)nse_eff * sizeof(double));
  memcpy(tmp, scratch_r, (size_t)nse_eff * sizeof(double));
  double h2 = or_kth_double(tmp, nse_eff, nv_eff);
  if (tmp != r2) free(tmp);
  if (!(h2 > 0.0)) return INFINITY;
  double h = sqrt(h2);
  double norm = 15.0 / (8.0 * OR_PI * h * h * h);
  double sum = 0.0;
  for (int64_t q = 0; q < nse_eff; ++q) {
    if (scratch_r[q] < h2) sum += norm * (1.0 - scratch_r[q] / h2);
  }
  return sum / (double)nse_eff;
}

/* f_l for every member of one halo. Returns 0 on success. */
int or_velden_halo(const int64_t *upos, const float *vel, const int32_t *members, int64_t nh,
                   int nse, int nv, double *f_l) {
  if (nh <= 0) return 0;
  if (nse < 1 || nv < 1 || nv > nse) return 1;
  or_nb *nb = (or_nb *)malloc((size_t)nh * sizeof(or_nb));
  double *r = (double *)malloc((size_t)(nse < nh ? nse : nh) * sizeof(double));
  if (!nb || !r) { free(nb); free(r); return 2; }
  for (int64_t k = 0; k < nh; ++k) f_l[k] = or_velden_member(upos, vel, members, nh, k, nse, nv, nb, r);
  free(nb);
  free(r);
  return 0;
}

/* f_l of a single member k (for sampled checks on large halos). */
double or_velden_one(const int64_t *upos, const float *vel, const int32_t *members, int64_t nh,
                     int64_t k, int nse, int nv) {
  if (nh <= 0 || k < 0 || k >= nh || nse < 1 || nv < 1 || nv > nse) return NAN;
  or_nb *nb = (or_nb *)malloc((size_t)nh * sizeof(or_nb));
  double *r = (double *)malloc((size_t)(nse < nh ? nse : nh) * sizeof(double));
  double v = or_velden_member(upos, vel, members, nh, k, nse, nv, nb, r);
  free(nb);
  free(r);
  return v;
}

/* The N_se-nearest set of member k as particle indices, sorted by (d^2, index);
 * returns its size. Exposed for the k-NN pins. */
int64_t or_knn_one(const int64_t *upos, const int32_t *members, int64_t nh, int64_t k, int nse,
                   int32_t *out) {
  if (nh <= 0 || k < 0 || k >= nh) return -1;
  int64_t nse_eff = nse < nh ? nse : nh;
  or_nb *nb = (or_nb *)malloc((size_t)nh * sizeof(or_nb));
  for (int64_t m = 0; m < nh; ++m) {
    int64_t s = 0;
    for (int c = 0; c < 3; ++c) {
      int64_t d = upos[3 * m + c] - upos[3 * k + c];
      s += d * d;
    }
    nb[m].d2 = s;
    nb[m].idx = members[m];
  }
  or_select_nb(nb, nh, nse_eff);
  /* order the selected set for output (insertion sort; small) */
  for (int64_t a = 1; a < nse_eff; ++a) {
    or_nb t = nb[a];
    int64_t b = a - 1;
    while (b >= 0 && or_nb_less(&t, &nb[b])) { nb[b + 1] = nb[b]; --b; }
    nb[b + 1] = t;
  }
  for (int64_t q = 0; q < nse_eff; ++q) out[q] = (int32_t)nb[q].idx;
  free(nb);
  return nse_eff;
}

/* --------------------------------- background cells: entropy kd-tree (Sec. 2.2) */

/* Number of particles per background cell: N_cell = f_cell N_H, raised when below
 * ncell_min (100) to min(ncell_min, floor(N_H / 8)) (Sec. 2.2). */
int64_t or_ncell(int64_t nh, double f_cell, int32_t ncell_min) {
  int64_t nc = (int64_t)floor(f_cell * (double)nh);
  if (nc < ncell_min) {
    nc = ncell_min;
    if (nh / 8 < nc) nc = nh / 8;
  }
  if (nc < 1) nc = 1;
  return nc;
}

/* largest m with m^3 <= n */
static int64_t or_icbrt(int64_t n) {
  int64_t m = (int64_t)cbrt((double)n);
  while (m > 0 && m * m * m > n) --m;
  while ((m + 1) * (m + 1) * (m + 1) <= n) ++m;
  return m;
}

typedef struct {
  int64_t lo[3], hi[3]; /* half-open region */
  int axis;             /* -1 for a leaf */
  int64_t split;
  int64_t left, right;  /* child node ids */
  int64_t leaf;         /* leaf id (DFS order, left first) or -1 */
  int64_t beg, end;     /* range in the permutation */
} or_node;

typedef struct {
  or_node *nodes;
  int64_t nnodes, cap;
  int64_t nleaves;
  int64_t *perm;         /* local member indices, leaves contiguous */
  const int64_t *upos;
  int64_t ncell;
  int split_rule;
} or_tree;

static const int64_t *or_sort_upos;
static int or_sort_axis;
static int or_cmp_axis(const void *pa, const void *pb) {
  int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
  int64_t xa = or_sort_upos[3 * a + or_sort_axis], xb = or_sort_upos[3 * b + or_sort_axis];
  if (xa != xb) return xa < xb ? -1 : 1;
  return a < b ? -1 : (a > b);
}

static int64_t or_new_node(or_tree *t) {
  if (t->nnodes == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 64;
    t->nodes = (or_node *)realloc(t->nodes, (size_t)t->cap * sizeof(or_node));
  }
  memset(&t->nodes[t->nnodes], 0, sizeof(or_node));
  return t->nnodes++;
}

/* Shannon entropy of the node's coordinates along one axis (Eq. S): n_b equal integer
 * bins spanning [min, max], bin = floor((x - min) n_b / (max - min + 1)),
 * S = -sum_k (m_k/m) ln(m_k/m) / ln n_b with unit masses. */
static double or_entropy(const or_tree *t, int64_t beg, int64_t end, int axis, int64_t mn,
                         int64_t mx, int64_t nb) {
  int64_t *cnt = (int64_t *)calloc((size_t)nb, sizeof(int64_t));
  int64_t n = end - beg;
  for (int64_t p = beg; p < end; ++p) {
    int64_t x = t->upos[3 * t->perm[p] + axis];
    cnt[(x - mn) * nb / (mx - mn + 1)]++;
  }
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    if (cnt[b] > 0) {
      double f = (double)cnt[b] / (double)n;
      s -= f * log(f);
    }
  }
  free(cnt);
  return s / log((double)nb);
}

/* Splits node id while it holds more than N_cell particles (Sec. 2.2): along the axis
 * that maximises S (split_rule 0; 1 = minimises), ties within 1e-12 to the lower axis;
 * split value = coordinate of element floor(n/2) in (coordinate, index) order;
 * left = {x < x_s}, right = {x >= x_s}; an axis that leaves a side empty is skipped
 * in favour of the next-best one; with none left the node is a leaf. */
static void or_split(or_tree *t, int64_t id) {
  int64_t beg = t->nodes[id].beg, end = t->nodes[id].end, n = end - beg;
  t->nodes[id].axis = -1;
  t->nodes[id].leaf = -1;
  if (n > t->ncell) {
    int64_t mn[3], mx[3];
    for (int a = 0; a < 3; ++a) { mn[a] = INT64_MAX; mx[a] = INT64_MIN; }
    for (int64_t p = beg; p < end; ++p)
      for (int a = 0; a < 3; ++a) {
        int64_t x = t->upos[3 * t->perm[p] + a];
        if (x < mn[a]) mn[a] = x;
        if (x > mx[a]) mx[a] = x;
      }
    int64_t nb = or_icbrt(n);
    if (nb < 2) nb = 2;
    double S[3];
    int ok[3];
    for (int a = 0; a < 3; ++a) {
      ok[a] = mx[a] > mn[a];
      S[a] = ok[a] ? or_entropy(t, beg, end, a, mn[a], mx[a], nb) : 0.0;
    }
    /* preference order of the axes */
    int order[3], used[3] = {0, 0, 0}, norder = 0;
    for (int r = 0; r < 3; ++r) {
      int best = -1;
      for (int a = 0; a < 3; ++a) {
        if (!ok[a] || used[a]) continue;
        if (best < 0) { best = a; continue; }
        if (t->split_rule == 0 ? (S[a] > S[best] + 1e-12) : (S[a] < S[best] - 1e-12)) best = a;
      }
      if (best < 0) break;
      used[best] = 1;
      order[norder++] = best;
    }
    for (int r = 0; r < norder; ++r) {
      int a = order[r];
      or_sort_upos = t->upos;
      or_sort_axis = a;
      qsort(t->perm + beg, (size_t)n, sizeof(int64_t), or_cmp_axis);
      int64_t xs = t->upos[3 * t->perm[beg + n / 2] + a];
      int64_t nleft = 0;
      while (nleft < n && t->upos[3 * t->perm[beg + nleft] + a] < xs) ++nleft;
      if (nleft == 0) continue; /* left side empty: next axis */
      int64_t l = or_new_node(t), rgt = or_new_node(t);
      or_node *me = &t->nodes[id];
      me->axis = a;
      me->split = xs;
      me->left = l;
      me->right = rgt;
      or_node *L = &t->nodes[l], *R = &t->nodes[rgt];
      for (int c = 0; c < 3; ++c) {
        L->lo[c] = R->lo[c] = me->lo[c];
        L->hi[c] = R->hi[c] = me->hi[c];
      }
      L->hi[a] = xs;
      R->lo[a] = xs;
      L->beg = beg; L->end = beg + nleft;
      R->beg = beg + nleft; R->end = end;
      or_split(t, l);
      or_split(t, rgt);
      return;
    }
  }
  t->nodes[id].leaf = t->nleaves++;
}

/* Leaf containing point p (descend by the split rule), or -1 if p is outside the root
 * region. */
static int64_t or_locate(const or_tree *t, const int64_t *p) {
  const or_node *r = &t->nodes[0];
  for (int a = 0; a < 3; ++a)
    if (p[a] < r->lo[a] || p[a] >= r->hi[a]) return -1;
  int64_t id = 0;
  while (t->nodes[id].axis >= 0) {
    const or_node *nd = &t->nodes[id];
    id = p[nd->axis] < nd->split ? nd->left : nd->right;
  }
  return t->nodes[id].leaf;
}

/* Cholesky of a symmetric 3x3 given by its unique entries (xx, yy, zz, xy, xz, yz);
 * returns 0 if not positive definite. L is lower triangular (l00, l10, l11, l20, l21, l22). */
static int or_chol3(const double *s, double *L) {
  double a00 = s[0], a11 = s[1], a22 = s[2], a10 = s[3], a20 = s[4], a21 = s[5];
  if (!(a00 > 0.0)) return 0;
  double l00 = sqrt(a00);
  double l10 = a10 / l00, l20 = a20 / l00;
  double d1 = a11 - l10 * l10;
  if (!(d1 > 0.0)) return 0;
  double l11 = sqrt(d1);
  double l21 = (a21 - l20 * l10) / l11;
  double d2 = a22 - l20 * l20 - l21 * l21;
  if (!(d2 > 0.0)) return 0;
  double l22 = sqrt(d2);
  L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = l22;
  return 1;
}

/* ln f_bg (Eq. fvbg): multivariate Gaussian of mean vbar and dispersion tensor sig
 * (unique entries xx, yy, zz, xy, xz, yz) evaluated at v, via the Cholesky factor:
 * q = |L^-1 (v - vbar)|^2, ln|Sigma|^(1/2) = sum ln L_ii. NaN if sig is not PD. */
double or_ln_fbg(const double *v, const double *vbar, const double *sig) {
  double L[6];
  if (!or_chol3(sig, L)) return NAN;
  double d0 = v[0] - vbar[0], d1 = v[1] - vbar[1], d2 = v[2] - vbar[2];
  double y0 = d0 / L[0];
  double y1 = (d1 - L[1] * y0) / L[2];
  double y2 = (d2 - L[3] * y0 - L[4] * y1) / L[5];
  double q = y0 * y0 + y1 * y1 + y2 * y2;
  return -0.5 * q - 1.5 * log(2.0 * OR_PI) - (log(L[0]) + log(L[2]) + log(L[5]));
}

/* Background model and log ratio R for one halo (Sec. 2.2):
 *  - entropy kd-tree cells of at most N_cell members (or_split);
 *  - per cell: centre of mass (Eq. meanpos), mean velocity (Eq. meanvel) and the
 *    dispersion tensor about it divided by the cell mass (Eq. meandispvel);
 *  - at each member: inverse-distance interpolation (Eq. cellinterp) of vbar and the six
 *    unique tensor entries over its own cell and the face-neighbour cells, the latter
 *    being the leaves that contain the member's position moved just across each of
 *    its cell's six faces (skipped when outside the halo's region; a cell counted
 *    once); a zero distance gives that cell alone;
 *  - R = ln f_l - ln f_bg (Eq. fvbg), NaN when the interpolated tensor is not PD.
 * f_l [nh] in member order; outputs R [nh], leaf_of [nh] (may be NULL),
 * cell_stats [nleaves][13] (mass, xbar[3], vbar[3], sig[6]; may be NULL, sized by the
 * caller to at least nh entries), leaf_box [nleaves][6] (the half-open region lo[3],
 * hi[3] of each leaf; may be NULL, sized like cell_stats). Returns the number of leaves,
 * or -1. */
int64_t or_background_halo(const int64_t *upos, const float *vel, const int32_t *members,
                           int64_t nh, const double *f_l, double f_cell, int32_t ncell_min,
                           int split_rule, double *R, int32_t *leaf_of, double *cell_stats,
                           int64_t *leaf_box) {
  if (nh <= 0) return 0;
  or_tree t;
  memset(&t, 0, sizeof(t));
  t.upos = upos;
  t.ncell = or_ncell(nh, f_cell, ncell_min);
  t.split_rule = split_rule;
  t.perm = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t m = 0; m < nh; ++m) t.perm[m] = m;
  int64_t root = or_new_node(&t);
  for (int a = 0; a < 3; ++a) {
    int64_t mn = INT64_MAX, mx = INT64_MIN;
    for (int64_t m = 0; m < nh; ++m) {
      if (upos[3 * m + a] < mn) mn = upos[3 * m + a];
      if (upos[3 * m + a] > mx) mx = upos[3 * m + a];
    }
    t.nodes[root].lo[a] = mn;
    t.nodes[root].hi[a] = mx + 1;
  }
  t.nodes[root].beg = 0;
  t.nodes[root].end = nh;
  or_split(&t, root);

  int64_t nl = t.nleaves;
  int64_t *leaf = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  int64_t *leaf_node = (int64_t *)malloc((size_t)nl * sizeof(int64_t));
  for (int64_t id = 0; id < t.nnodes; ++id) {
    if (t.nodes[id].axis >= 0) continue;
    leaf_node[t.nodes[id].leaf] = id;
    for (int64_t p = t.nodes[id].beg; p < t.nodes[id].end; ++p) leaf[t.perm[p]] = t.nodes[id].leaf;
  }
  /* cell moments, FP64, members visited in increasing index order */
  double *cs = (double *)calloc((size_t)nl * 13, sizeof(double));
  for (int64_t m = 0; m < nh; ++m) {
    double *c = cs + 13 * leaf[m];
    const float *v = vel + 3 * (int64_t)members[m];
    c[0] += 1.0;
    for (int a = 0; a < 3; ++a) {
      c[1 + a] += (double)upos[3 * m + a];
      c[4 + a] += (double)v[a];
    }
  }
  for (int64_t l = 0; l < nl; ++l) {
    double *c = cs + 13 * l;
    for (int a = 0; a < 6; ++a) c[1 + a] /= c[0];
  }
  for (int64_t m = 0; m < nh; ++m) {
    double *c = cs + 13 * leaf[m];
    const float *v = vel + 3 * (int64_t)members[m];
    double d0 = (double)v[0] - c[4], d1 = (double)v[1] - c[5], d2 = (double)v[2] - c[6];
    c[7] += d0 * d0;
    c[8] += d1 * d1;
    c[9] += d2 * d2;
    c[10] += d0 * d1;
    c[11] += d0 * d2;
    c[12] += d1 * d2;
  }
  for (int64_t l = 0; l < nl; ++l) {
    double *c = cs + 13 * l;
    for (int a = 7; a < 13; ++a) c[a] /= c[0];
  }
  /* per member: interpolation and R */
  for (int64_t m = 0; m < nh; ++m) {
    int64_t own = leaf[m];
    const or_node *nd = &t.nodes[leaf_node[own]];
    int64_t cells[7];
    int nc = 0;
    cells[nc++] = own;
    for (int a = 0; a < 3; ++a) {
      for (int side = 0; side < 2; ++side) {
        int64_t p[3] = {upos[3 * m], upos[3 * m + 1], upos[3 * m + 2]};
        p[a] = side == 0 ? nd->lo[a] - 1 : nd->hi[a];
        int64_t q = or_locate(&t, p);
        if (q < 0) continue;
        int dup = 0;
        for (int u = 0; u < nc; ++u) dup |= cells[u] == q;
        if (!dup) cells[nc++] = q;
      }
    }
    double w[7];
    int zero = -1;
    for (int u = 0; u < nc; ++u) {
      const double *c = cs + 13 * cells[u];
      double dx = (double)upos[3 * m] - c[1], dy = (double)upos[3 * m + 1] - c[2],
             dz = (double)upos[3 * m + 2] - c[3];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r == 0.0) { zero = u; break; }
      w[u] = 1.0 / r;
    }
    double vbar[3] = {0, 0, 0}, sig[6] = {0, 0, 0, 0, 0, 0};
    if (zero >= 0) {
      const double *c = cs + 13 * cells[zero];
      for (int a = 0; a < 3; ++a) vbar[a] = c[4 + a];
      for (int a = 0; a < 6; ++a) sig[a] = c[7 + a];
    } else {
      double wsum = 0.0;
      for (int u = 0; u < nc; ++u) wsum += w[u];
      for (int u = 0; u < nc; ++u) {
        const double *c = cs + 13 * cells[u];
        double f = w[u] / wsum;
        for (int a = 0; a < 3; ++a) vbar[a] += f * c[4 + a];
        for (int a = 0; a < 6; ++a) sig[a] += f * c[7 + a];
      }
    }
    const float *vf = vel + 3 * (int64_t)members[m];
    double v[3] = {(double)vf[0], (double)vf[1], (double)vf[2]};
    double lnfbg = or_ln_fbg(v, vbar, sig);
    R[m] = log(f_l[m]) - lnfbg;
    if (leaf_of) leaf_of[m] = (int32_t)own;
  }
  if (cell_stats) memcpy(cell_stats, cs, (size_t)nl * 13 * sizeof(double));
  if (leaf_box)
    for (int64_t l = 0; l < nl; ++l)
      for (int a = 0; a < 3; ++a) {
        leaf_box[6 * l + a] = t.nodes[leaf_node[l]].lo[a];
        leaf_box[6 * l + 3 + a] = t.nodes[leaf_node[l]].hi[a];
      }
  free(cs);
  free(leaf);
  free(leaf_node);
  free(t.perm);
  free(t.nodes);
  return nl;
}

/* ------------------------------- skew-Gaussian fit of the R distribution (Eq. skewgaus) */

static int or_cmp_double(const void *pa, const void *pb) {
  double a = *(const double *)pa, b = *(const double *)pb;
  return a < b ? -1 : (a > b);
}

static double or_median_sorted(const double *a, int64_t n) {
  return (n & 1) ? a[n / 2] : 0.5 * (a[n / 2 - 1] + a[n / 2]);
}

/* f_SG and its partial derivatives w.r.t. (A, Rbar, sigma, s) at x (Eq. skewgaus):
 * left of the mode the width is s*sigma, right of it sigma. */
static double or_sg(double x, const double *p, double *g) {
  double A = p[0], mu = p[1], sg = p[2], s = p[3];
  double d = x - mu;
  if (d < 0.0) {
    double w = s * sg;
    double e = exp(-d * d / (2.0 * w * w));
    if (g) {
      g[0] = e;
      g[1] = A * e * d / (w * w);
      g[2] = A * e * d * d / (w * w * sg);
      g[3] = A * e * d * d / (w * w * s);
    }
    return A * e;
  } else {
    double e = exp(-d * d / (2.0 * sg * sg));
    if (g) {
      g[0] = e;
      g[1] = A * e * d / (sg * sg);
      g[2] = A * e * d * d / (sg * sg * sg);
      g[3] = 0.0;
    }
    return A * e;
  }
}

/* Solves the 4x4 system M x = b by Gaussian elimination with partial pivoting.
 * Returns 0 if singular. */
static int or_solve4(double M[4][4], double *b, double *x) {
  double a[4][5];
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) a[i][j] = M[i][j];
    a[i][4] = b[i];
  }
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (!(fabs(a[piv][c]) > 0.0)) return 0;
    if (piv != c)
      for (int j = 0; j < 5; ++j) { double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
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
  return 1;
}

/* Binning of one halo's R values for the fit of Eq. skewgaus (Sec. 2.2):
 *  - finite R values only; median and MAD' = 1.4826 * median |R - median|;
 *  - nbins = clamp(ceil(sqrt(N)), nbins_min, nbins_max) equal bins on
 *    [median - 6 MAD', median + 6 MAD'], bin = floor((R - lo) / width), values outside
 *    dropped.
 * counts [nbins_max] out (may be NULL); meta = (median, MAD', lo, width, nbins) out.
 * Returns 0, or 1 when degenerate (fewer than 2 finite values or MAD' = 0; meta[0] is
 * the median when there are at least 2 values, NaN otherwise, and nbins is 0). */
int or_ell_bins(const double *R, int64_t nh, int nbins_min, int nbins_max, double *counts,
                double *meta) {
  double *a = (double *)malloc((size_t)(nh ? nh : 1) * sizeof(double));
  int64_t n = 0;
  for (int64_t i = 0; i < nh; ++i)
    if (isfinite(R[i])) a[n++] = R[i];
  for (int k = 0; k < 5; ++k) meta[k] = NAN;
  meta[4] = 0.0;
  if (n < 2) { free(a); return 1; }
  qsort(a, (size_t)n, sizeof(double), or_cmp_double);
  double med = or_median_sorted(a, n);
  double *dev = (double *)malloc((size_t)n * sizeof(double));
  for (int64_t i = 0; i < n; ++i) dev[i] = fabs(a[i] - med);
  qsort(dev, (size_t)n, sizeof(double), or_cmp_double);
  double mad = 1.4826 * or_median_sorted(dev, n);
  free(dev);
  meta[0] = med;
  meta[1] = mad;
  if (!(mad > 0.0)) { free(a); return 1; }
  int64_t nb = 0;
  while (nb * nb < n) ++nb; /* ceil(sqrt(n)) */
  if (nb < nbins_min) nb = nbins_min;
  if (nb > nbins_max) nb = nbins_max;
  double lo = med - 6.0 * mad, width = 12.0 * mad / (double)nb;
  double *cnt = (double *)calloc((size_t)nb, sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    double f = floor((a[i] - lo) / width);
    if (f >= 0.0 && f < (double)nb) cnt[(int64_t)f] += 1.0;
  }
  free(a);
  meta[2] = lo;
  meta[3] = width;
  meta[4] = (double)nb;
  if (counts) memcpy(counts, cnt, (size_t)nb * sizeof(double));
  free(cnt);
  return 0;
}

/* Least-squares fit of Eq. skewgaus, A f_SG(x; Rbar, sigma, s), to nb binned counts
 * whose bin b is centred at x_b = lo + (b + 1/2) width (Sec. 2.2): Levenberg-Marquardt,
 * unweighted, started from A = max count, Rbar = centre of the first fullest bin,
 * sigma = sigma0, s = 1; lambda = 1e-3, divided by 10 on an accepted step and multiplied
 * by 10 on a rejected one; at most `iters` iterations, stopping early when an accepted
 * step changes the cost by less than 1e-15 relative. out = (Rbar, sigma_R, s, A). */
void or_sg_fit(const double *cnt, int64_t nb, double lo, double width, double sigma0,
               int iters, double *out) {
  int64_t mode = 0;
  for (int64_t b = 1; b < nb; ++b)
    if (cnt[b] > cnt[mode]) mode = b;
  double p[4] = {cnt[mode], lo + ((double)mode + 0.5) * width, sigma0, 1.0};
  double lambda = 1e-3;
  double cost = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    double x = lo + ((double)b + 0.5) * width;
    double r = cnt[b] - or_sg(x, p, NULL);
    cost += r * r;
  }
  for (int it = 0; it < iters; ++it) {
    double JtJ[4][4] = {{0}}, Jtr[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < nb; ++b) {
      double x = lo + ((double)b + 0.5) * width, g[4];
      double r = cnt[b] - or_sg(x, p, g);
      for (int i = 0; i < 4; ++i) {
        Jtr[i] += g[i] * r;
        for (int j = 0; j < 4; ++j) JtJ[i][j] += g[i] * g[j];
      }
    }
    double M[4][4], delta[4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) M[i][j] = JtJ[i][j] + (i == j ? lambda * JtJ[i][i] : 0.0);
    int ok = or_solve4(M, Jtr, delta);
    double q[4];
    for (int i = 0; i < 4; ++i) q[i] = p[i] + (ok ? delta[i] : 0.0);
    double ncost = INFINITY;
    if (ok && q[2] > 0.0 && q[3] > 0.0) {
      ncost = 0.0;
      for (int64_t b = 0; b < nb; ++b) {
        double x = lo + ((double)b + 0.5) * width;
        double r = cnt[b] - or_sg(x, q, NULL);
        ncost += r * r;
      }
    }
    if (ncost < cost) {
      double rel = (cost - ncost) / cost;
      for (int i = 0; i < 4; ++i) p[i] = q[i];
      cost = ncost;
      lambda /= 10.0;
      if (rel < 1e-15) break;
    } else {
      lambda *= 10.0;
      if (lambda > 1e30) break;
    }
  }
  out[0] = p[1];
  out[1] = p[2];
  out[2] = p[3];
  out[3] = p[0];
}

/* Fit of Eq. skewgaus to the binned R distribution of one halo (Sec. 2.2): the binning
 * of or_ell_bins, then or_sg_fit started from sigma = MAD'.
 * out = (Rbar, sigma_R, s, A, lo, width, nbins, MAD'). Returns 0, or 1 when degenerate
 * (fewer than 2 finite values or MAD' = 0: out[0] = median, out[1] = NaN). */
int or_ell_fit(const double *R, int64_t nh, int nbins_min, int nbins_max, int iters, double *out) {
  for (int k = 0; k < 8; ++k) out[k] = NAN;
  double meta[5];
  double *cnt = (double *)calloc((size_t)(nbins_max > 0 ? nbins_max : 1), sizeof(double));
  int deg = or_ell_bins(R, nh, nbins_min, nbins_max, cnt, meta);
  out[0] = meta[0];
  out[7] = meta[1];
  if (deg) { free(cnt); return 1; }
  double fit[4];
  or_sg_fit(cnt, (int64_t)meta[4], meta[2], meta[3], meta[1], iters, fit);
  free(cnt);
  out[0] = fit[0];
  out[1] = fit[1];
  out[2] = fit[2];
  out[3] = fit[3];
  out[4] = meta[2];
  out[5] = meta[3];
  out[6] = meta[4];
  return 0;
}

/* --------------------------- phase-space linking of outliers (Eq. linkingcriteria) */

/* Link predicate for outliers i, j of one halo (Eqs. linkingcriteria b-d, with the 6D
 * velocity term of Eq. fof6d when use_lv is set). Evaluation order is fixed and uses
 * no fused multiply-add:
 *   dv_c = v_i,c - v_j,c (FP64), dv2 = (dv_x^2 + dv_y^2) + dv_z^2,
 *   q = dx2 / lx2 (+ dv2 / lv2), link needs q < 1;
 *   u = v - v_frame, s = (u_x^2 + u_y^2) + u_z^2:
 *   speed ratio: s_i, s_j > 0, s_i <= V_r^2 s_j and s_j <= V_r^2 s_i;
 *   opening angle: dot = (u_i,x u_j,x + u_i,y u_j,y) + u_i,z u_j,z, dot >= 0 and
 *   dot^2 >= (cos^2 Theta_op s_i) s_j (valid for Theta_op < pi/2). */
static int or_link6(int64_t dx2, const float *vi, const float *vj, const double *prm,
                    double vr2, double cos2, int use_lv, int use_vt) {
  double lx2 = prm[0], lv2 = prm[1];
  double q = (double)dx2 / lx2;
  if (use_lv) {
    double d0 = (double)vi[0] - (double)vj[0], d1 = (double)vi[1] - (double)vj[1],
           d2 = (double)vi[2] - (double)vj[2];
    double dv2 = (d0 * d0 + d1 * d1) + d2 * d2;
    q = q + dv2 / lv2;
  }
  if (!(q < 1.0)) return 0;
  if (use_vt) {
    double ui[3], uj[3];
    for (int c = 0; c < 3; ++c) {
      ui[c] = (double)vi[c] - prm[2 + c];
      uj[c] = (double)vj[c] - prm[2 + c];
    }
    double si = (ui[0] * ui[0] + ui[1] * ui[1]) + ui[2] * ui[2];
    double sj = (uj[0] * uj[0] + uj[1] * uj[1]) + uj[2] * uj[2];
    if (!(si > 0.0 && sj > 0.0)) return 0;
    if (!(si <= vr2 * sj && sj <= vr2 * si)) return 0;
    double dot = (ui[0] * uj[0] + ui[1] * uj[1]) + ui[2] * uj[2];
    if (!(dot >= 0.0)) return 0;
    if (!(dot * dot >= (cos2 * si) * sj)) return 0;
  }
  return 1;
}

/* 6D linking inside one halo (Sec. 2.2, "Linking particles"): candidates are the
 * members flagged in `cand` (ell >= ell_th, or all members for a plain 6DFOF); every
 * candidate pair is tested (brute force) and linked pairs are merged; groups with fewer
 * than nmin members get -1, others the minimum particle index of the group.
 * prm = (lx2, lv2, vframe_x, vframe_y, vframe_z). label6 [nh] in member order. */
int or_fof6d_halo(const int64_t *upos, const float *vel, const int32_t *members, int64_t nh,
                  const uint8_t *cand, const double *prm, double v_ratio, double theta_op,
                  int use_lv, int use_vt, int32_t nmin, int32_t *label6) {
  if (nh <= 0) return 0;
  int64_t *parent = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t m = 0; m < nh; ++m) parent[m] = m;
  double vr2 = v_ratio * v_ratio;
  double ct = cos(theta_op);
  double cos2 = ct * ct;
  for (int64_t i = 0; i < nh; ++i) {
    if (!cand[i]) continue;
    for (int64_t j = i + 1; j < nh; ++j) {
      if (!cand[j]) continue;
      int64_t s = 0;
      for (int c = 0; c < 3; ++c) {
        int64_t d = upos[3 * i + c] - upos[3 * j + c];
        s += d * d;
      }
      if (or_link6(s, vel + 3 * (int64_t)members[i], vel + 3 * (int64_t)members[j], prm, vr2,
                   cos2, use_lv, use_vt))
        or_union(parent, i, j);
    }
  }
  int64_t *size = (int64_t *)calloc((size_t)nh, sizeof(int64_t));
  for (int64_t m = 0; m < nh; ++m)
    if (cand[m]) size[or_find(parent, m)]++;
  for (int64_t m = 0; m < nh; ++m) {
    if (!cand[m]) { label6[m] = -1; continue; }
    int64_t r = or_find(parent, m); /* minimum member slot = minimum particle index */
    label6[m] = size[r] >= nmin ? members[r] : -1;
  }
  free(size);
  free(parent);
  return 0;
}

/* --------------------------------------------------------------- halo frame */

/* Mean velocity and sigma_host = |Sigma|^(1/6) of a halo (Table A2's sigma_v), with
 * the dispersion tensor about the mean divided by N_H. out = (vbar[3], sigma_host). */
void or_halo_frame(const float *vel, const int32_t *members, int64_t nh, double *out) {
  double m[3] = {0, 0, 0};
  for (int64_t i = 0; i < nh; ++i)
    for (int c = 0; c < 3; ++c) m[c] += (double)vel[3 * (int64_t)members[i] + c];
  for (int c = 0; c < 3; ++c) m[c] /= (double)nh;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < nh; ++i) {
    const float *v = vel + 3 * (int64_t)members[i];
    double d0 = (double)v[0] - m[0], d1 = (double)v[1] - m[1], d2 = (double)v[2] - m[2];
    s[0] += d0 * d0; s[1] += d1 * d1; s[2] += d2 * d2;
    s[3] += d0 * d1; s[4] += d0 * d2; s[5] += d1 * d2;
  }
  for (int c = 0; c < 6; ++c) s[c] /= (double)nh;
  /* det of [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]] */
  double det = s[0] * (s[1] * s[2] - s[5] * s[5]) - s[3] * (s[3] * s[2] - s[5] * s[4]) +
               s[4] * (s[3] * s[5] - s[1] * s[4]);
  out[0] = m[0]; out[1] = m[1]; out[2] = m[2];
  out[3] = det > 0.0 ? pow(det, 1.0 / 6.0) : 0.0;
}

/* ------------------------------------------- significance cleaning (Sec. 2.2) */

double or_ell_bar(double ell_th);

typedef struct {
  double ell;
  int64_t idx;
} or_ev;

static int or_cmp_ev(const void *pa, const void *pb) {
  const or_ev *a = (const or_ev *)pa, *b = (const or_ev *)pb;
  if (a->ell != b->ell) return a->ell < b->ell ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Cleaning the catalogue (Sec. 2.2, Eq. ellsig). A group of N particles is significant
 * when its mean ell satisfies <ell> >= ell_bar(ell_th) (1 + beta/sqrt(N)), ell_bar the
 * tail mean of Eq. ellsig (or_ell_bar). A group that is not loses its particles in order
 * of smallest ell (ties: smaller particle index first) until it is; a group left with
 * fewer than nmin particles is removed. Removed particles get -1; the particles kept get
 * the minimum particle index among them. The mean is (sum of the kept ell) / N in FP64,
 * the threshold ell_bar * (1 + beta / sqrt(N)).
 * label6 [n] in/out (groups: equal labels >= 0), ell [n]. Returns the groups kept. */
int64_t or_clean_groups(const double *ell, int32_t *label6, int64_t n, double ell_th,
                        double beta, int32_t nmin) {
  const double lbar = or_ell_bar(ell_th);
  /* group the particles by label (counting sort on the label value) */
  int64_t *count = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    if (label6[i] >= 0) count[label6[i] + 1]++;
  for (int64_t l = 0; l < n; ++l) count[l + 1] += count[l];
  or_ev *ev = (or_ev *)malloc((size_t)(count[n] ? count[n] : 1) * sizeof(or_ev));
  int64_t *fill = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    if (label6[i] < 0) continue;
    int64_t l = label6[i];
    ev[count[l] + fill[l]].ell = ell[i];
    ev[count[l] + fill[l]].idx = i;
    fill[l]++;
  }
  int64_t kept = 0;
  for (int64_t l = 0; l < n; ++l) {
    const int64_t b = count[l], N = count[l + 1] - count[l];
    if (N == 0) continue;
    or_ev *g = ev + b;
    qsort(g, (size_t)N, sizeof(or_ev), or_cmp_ev);
    double sum = 0.0;
    for (int64_t k = 0; k < N; ++k) sum += g[k].ell;
    int64_t cut = -1; /* particles removed */
    for (int64_t k = 0; k < N; ++k) {
      const int64_t m = N - k;
      const double mean = sum / (double)m;
      const double thr = lbar * (1.0 + beta / sqrt((double)m));
      if (mean >= thr) { cut = k; break; }
      sum -= g[k].ell;
    }
    const int keep = cut >= 0 && N - cut >= nmin;
    int64_t newlab = n;
    if (keep)
      for (int64_t k = cut; k < N; ++k) newlab = g[k].idx < newlab ? g[k].idx : newlab;
    for (int64_t k = 0; k < N; ++k)
      label6[g[k].idx] = (keep && k >= cut) ? (int32_t)newlab : -1;
    kept += keep;
  }
  free(fill);
  free(ev);
  free(count);
  return kept;
}

/* ------------------------------------------------- two-stage linking (Sec. 2.2) */

typedef struct {
  int64_t a, b;
} or_pair;

/* Slot of particle index x among ascending members, -1 if absent. */
static int64_t or_slot(const int32_t *members, int64_t nh, int64_t x) {
  int64_t lo = 0, hi = nh;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (members[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < nh && members[lo] == x ? lo : -1;
}

static int or_cmp_pair(const void *pa, const void *pb) {
  const or_pair *x = (const or_pair *)pa, *y = (const or_pair *)pb;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  return x->b < y->b ? -1 : (x->b > y->b);
}

/* Two-stage linking inside one halo (Sec. 2.2, "Linking particles": conservative
 * criteria find the candidate substructures, relaxed criteria then link previously
 * untagged particles to them; substructures are joined only when the new connections
 * exceed f_merge times the original size of either).
 *   lab1  [nh] stage-1 labels of the members (minimum particle index of the group, -1
 *         for untagged members); ell [nh] their ell
 *   prm   (lx2, lv2, vframe_x, vframe_y, vframe_z) of the conservative pass
 *   gam   (gamma_ell, gamma_x, gamma_vr, gamma_theta): the relaxed pass takes
 *         candidates with ell >= ell_th / gamma_ell (and every tagged member), and links
 *         with lx2 gamma_x^2, V_r gamma_vr, Theta_op gamma_theta (lv2, frame unchanged)
 * Steps, in this order:
 *  1. the untagged candidates form connected components under the relaxed links among
 *     themselves;
 *  2. a component joins the stage-1 group with the most relaxed links between its
 *     members and the group's members (ties: the smaller label); with no such link it
 *     stays untagged;
 *  3. two grown groups A, B are joined iff the number of relaxed links between their
 *     members exceeds f_merge N_o(A) or f_merge N_o(B), N_o the stage-1 size; joins are
 *     transitive;
 *  4. every final group is labelled with its minimum particle index; untagged members
 *     get -1.
 * members ascending (as or_halos gives them). out [nh]: final labels. Returns 0. */
int or_grow_halo(const int64_t *upos, const float *vel, const int32_t *members, int64_t nh,
                 const double *ell, const int32_t *lab1, const double *prm, double ell_th,
                 double v_ratio, double theta_op, int use_lv, int use_vt, const double *gam,
                 double f_merge, int32_t *out) {
  for (int64_t i = 0; i < nh; ++i) out[i] = -1;
  if (nh <= 0) return 0;
  const double thr = ell_th / gam[0];
  const double prm2[5] = {prm[0] * gam[1] * gam[1], prm[1], prm[2], prm[3], prm[4]};
  const double vr = v_ratio * gam[2], ct = cos(theta_op * gam[3]);
  const double vr2 = vr * vr, cos2 = ct * ct;
  uint8_t *cand = (uint8_t *)malloc((size_t)nh);
  for (int64_t i = 0; i < nh; ++i) cand[i] = lab1[i] >= 0 || ell[i] >= thr;
  /* the relaxed links, once (over the candidates, in member order) */
  int64_t nc = 0;
  int64_t *ci = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i)
    if (cand[i]) ci[nc++] = i;
  int64_t ne = 0, cap = 1024;
  or_pair *e = (or_pair *)malloc((size_t)cap * sizeof(or_pair));
  for (int64_t x = 0; x < nc; ++x) {
    const int64_t i = ci[x];
    for (int64_t y = x + 1; y < nc; ++y) {
      const int64_t j = ci[y];
      int64_t d2 = 0;
      for (int c = 0; c < 3; ++c) {
        int64_t d = upos[3 * i + c] - upos[3 * j + c];
        d2 += d * d;
      }
      if (!or_link6(d2, vel + 3 * (int64_t)members[i], vel + 3 * (int64_t)members[j], prm2,
                    vr2, cos2, use_lv, use_vt))
        continue;
      if (ne == cap) {
        cap *= 2;
        e = (or_pair *)realloc(e, (size_t)cap * sizeof(or_pair));
      }
      e[ne].a = i;
      e[ne].b = j;
      ne++;
    }
  }
  /* 1. components of the untagged candidates */
  int64_t *parent = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) parent[i] = i;
  for (int64_t k = 0; k < ne; ++k)
    if (lab1[e[k].a] < 0 && lab1[e[k].b] < 0) or_union(parent, e[k].a, e[k].b);
  /* 2. links between components and groups: (component root, group label) pairs */
  or_pair *cg = (or_pair *)malloc((size_t)(ne ? ne : 1) * sizeof(or_pair));
  int64_t ncg = 0;
  for (int64_t k = 0; k < ne; ++k) {
    int64_t a = e[k].a, b = e[k].b;
    if ((lab1[a] < 0) == (lab1[b] < 0)) continue;
    int64_t u = lab1[a] < 0 ? a : b, t = lab1[a] < 0 ? b : a;
    cg[ncg].a = or_find(parent, u);
    cg[ncg].b = lab1[t];
    ncg++;
  }
  qsort(cg, (size_t)ncg, sizeof(or_pair), or_cmp_pair);
  int64_t *best = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  int64_t *bestn = (int64_t *)calloc((size_t)nh, sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) best[i] = -1;
  for (int64_t k = 0; k < ncg;) {
    int64_t k2 = k;
    while (k2 < ncg && cg[k2].a == cg[k].a && cg[k2].b == cg[k].b) k2++;
    int64_t c = cg[k].a, cnt = k2 - k;
    if (cnt > bestn[c]) { /* groups ascend within a component: ties keep the smaller */
      bestn[c] = cnt;
      best[c] = cg[k].b;
    }
    k = k2;
  }
  int64_t *grown = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) {
    if (lab1[i] >= 0) grown[i] = lab1[i];
    else if (cand[i]) grown[i] = best[or_find(parent, i)];
    else grown[i] = -1;
  }
  /* 3. joins between grown groups; group labels are particle indices of members, mapped
   *    to the member slot of that particle for a union-find over slots */
  int64_t *n0 = (int64_t *)calloc((size_t)nh, sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i)
    if (lab1[i] >= 0) n0[or_slot(members, nh, lab1[i])]++;
  or_pair *ab = (or_pair *)malloc((size_t)(ne ? ne : 1) * sizeof(or_pair));
  int64_t nab = 0;
  for (int64_t k = 0; k < ne; ++k) {
    int64_t ga = grown[e[k].a], gb = grown[e[k].b];
    if (ga < 0 || gb < 0 || ga == gb) continue;
    ab[nab].a = ga < gb ? ga : gb;
    ab[nab].b = ga < gb ? gb : ga;
    nab++;
  }
  qsort(ab, (size_t)nab, sizeof(or_pair), or_cmp_pair);
  int64_t *gpar = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) gpar[i] = i;
  for (int64_t k = 0; k < nab;) {
    int64_t k2 = k;
    while (k2 < nab && ab[k2].a == ab[k].a && ab[k2].b == ab[k].b) k2++;
    const int64_t sa = or_slot(members, nh, ab[k].a), sb = or_slot(members, nh, ab[k].b);
    double cnt = (double)(k2 - k);
    if (cnt > f_merge * (double)n0[sa] || cnt > f_merge * (double)n0[sb]) or_union(gpar, sa, sb);
    k = k2;
  }
  /* 4. labels */
  int64_t *minidx = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) minidx[i] = INT64_MAX;
  int64_t *gslot = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) {
    gslot[i] = -1;
    if (grown[i] < 0) continue;
    gslot[i] = or_find(gpar, or_slot(members, nh, grown[i]));
    if (members[i] < minidx[gslot[i]]) minidx[gslot[i]] = members[i];
  }
  for (int64_t i = 0; i < nh; ++i) out[i] = gslot[i] >= 0 ? (int32_t)minidx[gslot[i]] : -1;
  free(gslot); free(minidx); free(gpar); free(ab); free(n0); free(grown);
  free(bestn); free(best); free(cg); free(parent); free(e); free(ci); free(cand);
  return 0;
}

/* --------------------------------------------------------- core search (Sec. 2.3) */

/* Core search inside one halo (Sec. 2.3, "Core Identification", Eq. coreloop). The
 * "background" starts as the members outside substructure (lab6 < 0). Loop l = 0, 1,
 * ..., n_loop - 1: a 6DFOF (Eq. fof6d, all background members candidates) with
 * lx_l = alpha_x,C^l lx and lv_l = alpha_v,C^l lv, each length obtained by repeated
 * multiplication from lx and lv; groups count if they hold >= nmin and >= N_min,C =
 * f_C N_H alpha_N,C^l members (also by repeated multiplication, compared as reals).
 * With no such group the loop stops. Otherwise the largest group (ties: the smaller
 * label) becomes the next background, the "primary core", and every other group is a
 * candidate core of level l. After the loop the last primary core is labelled too.
 * Labels are the minimum particle index of each core.
 *   out_core [nh]: core label of each member, -1 if none; out_level [nh]: its level.
 * Returns the number of cores (candidate cores + the primary core). */
/* The loop itself. Besides the outputs above it gives, per member, the last loop at which
 * it was in the searched background (searched[i], -1 if never), and the primary core's
 * label and level (-1 if the halo found no group). */
static int64_t or_core_loop(const int64_t *upos, const float *vel, const int32_t *members,
                            int64_t nh, const int32_t *lab6, double lx, double lv, double ax,
                            double av, int n_loop, double f_c, double an, int32_t nmin,
                            int32_t *out_core, int32_t *out_level, int32_t *searched,
                            int32_t *prim_label, int32_t *prim_lev) {
  for (int64_t i = 0; i < nh; ++i) { out_core[i] = -1; out_level[i] = -1; searched[i] = -1; }
  *prim_label = -1;
  *prim_lev = -1;
  if (nh <= 0) return 0;
  uint8_t *bg = (uint8_t *)malloc((size_t)nh);
  int32_t *l6 = (int32_t *)malloc((size_t)nh * sizeof(int32_t));
  int64_t *size = (int64_t *)calloc((size_t)nh, sizeof(int64_t));
  for (int64_t i = 0; i < nh; ++i) bg[i] = lab6 ? lab6[i] < 0 : 1;
  double lxl = lx, lvl = lv, thr = f_c * (double)nh;
  int64_t ncore = 0, prim = -1;
  int prim_level = -1;
  for (int l = 0; l < n_loop; ++l) {
    if (l > 0) { lxl = lxl * ax; lvl = lvl * av; thr = thr * an; }
    double prm[5] = {lxl * lxl, lvl * lvl, 0.0, 0.0, 0.0};
    for (int64_t i = 0; i < nh; ++i)
      if (bg[i]) searched[i] = l;
    or_fof6d_halo(upos, vel, members, nh, bg, prm, 0.0, 0.0, 1, 0, 1, l6);
    /* group sizes by label slot (labels are member indices: the slot of a label) */
    for (int64_t i = 0; i < nh; ++i) size[i] = 0;
    for (int64_t i = 0; i < nh; ++i)
      if (l6[i] >= 0) size[or_slot(members, nh, l6[i])]++;
    int64_t big = -1;
    for (int64_t i = 0; i < nh; ++i) {
      if (size[i] < nmin || (double)size[i] < thr) continue;
      if (big < 0 || size[i] > size[big]) big = i; /* ascending slots: ties keep the smaller */
    }
    if (big < 0) break;
    for (int64_t i = 0; i < nh; ++i) {
      if (l6[i] < 0) { bg[i] = 0; continue; }
      const int64_t g = or_slot(members, nh, l6[i]);
      if (size[g] < nmin || (double)size[g] < thr) { bg[i] = 0; continue; }
      if (g == big) continue; /* stays in the background */
      bg[i] = 0;
      out_core[i] = l6[i];
      out_level[i] = l;
    }
    for (int64_t i = 0; i < nh; ++i)
      if (i != big && size[i] >= nmin && (double)size[i] >= thr) ncore++;
    prim = big;
    prim_level = l;
  }
  if (prim >= 0) {
    for (int64_t i = 0; i < nh; ++i)
      if (bg[i]) { out_core[i] = members[prim]; out_level[i] = prim_level; }
    ncore++;
    *prim_label = members[prim];
    *prim_lev = prim_level;
  }
  free(size);
  free(l6);
  free(bg);
  return ncore;
}

int64_t or_core_search(const int64_t *upos, const float *vel, const int32_t *members,
                       int64_t nh, const int32_t *lab6, double lx, double lv, double ax,
                       double av, int n_loop, double f_c, double an, int32_t nmin,
                       int32_t *out_core, int32_t *out_level) {
  int32_t *searched = (int32_t *)malloc((size_t)(nh > 0 ? nh : 1) * sizeof(int32_t));
  int32_t pl, pv;
  int64_t nc = or_core_loop(upos, vel, members, nh, lab6, lx, lv, ax, av, n_loop, f_c, an, nmin,
                            out_core, out_level, searched, &pl, &pv);
  free(searched);
  return nc;
}

/* ------------------------------------------- core growth (Sec. 2.3, growth) */

/* Phase-space mean and dispersion tensor (Eqs. coremeanphase, coredispphase) of the
 * rows i of X [n][6] with sel[i] != 0, unit masses (M = their count): mean = sum X / M,
 * then S_ab = sum (X_a - mean_a)(X_b - mean_b) / M, both summed in row order. S is a
 * full row-major 6x6. Returns M (mean and S untouched when M = 0). */
static int64_t or_phase_moments(const double *X, int64_t n, const uint8_t *sel, double *mean,
                                double *S) {
  int64_t m = 0;
  double sum[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    if (!sel[i]) continue;
    for (int a = 0; a < 6; ++a) sum[a] += X[6 * i + a];
    m++;
  }
  if (m == 0) return 0;
  for (int a = 0; a < 6; ++a) mean[a] = sum[a] / (double)m;
  double c[36];
  for (int a = 0; a < 36; ++a) c[a] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!sel[i]) continue;
    double d[6];
    for (int a = 0; a < 6; ++a) d[a] = X[6 * i + a] - mean[a];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) c[6 * a + b] += d[a] * d[b];
  }
  for (int a = 0; a < 36; ++a) S[a] = c[a] / (double)m;
  return m;
}

/* Cholesky L L^T = S of a symmetric 6x6 (row-major; the lower triangle is read), L
 * row-major lower triangular. Returns 0 when a pivot is not > 0 (S not positive
 * definite, or NaN). */
static int or_chol6(const double *S, double *L) {
  for (int a = 0; a < 36; ++a) L[a] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double d = S[6 * j + j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0)) return 0;
    const double ljj = sqrt(d);
    L[6 * j + j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double t = S[6 * i + j];
      for (int k = 0; k < j; ++k) t -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = t / ljj;
    }
  }
  return 1;
}

/* Eq. coredist: D^2 = d^T S^-1 d with S = L L^T, by forward substitution L y = d and
 * D^2 = y . y. */
static double or_dist6(const double *L, const double *d) {
  double y[6], D2 = 0.0;
  for (int i = 0; i < 6; ++i) {
    double t = d[i];
    for (int k = 0; k < i; ++k) t -= L[6 * i + k] * y[k];
    y[i] = t / L[6 * i + i];
    D2 += y[i] * y[i];
  }
  return D2;
}

/* Distance of X to a core (mean, S, L) under growth mode `mode`: modes 1 and 2 use
 * Eq. coredist; mode 0 uses the scalar form D^2 = |x - xbar|^2 / s_x^2 + |v - vbar|^2 / s_v^2
 * with s_x^2 = (S_xx + S_yy + S_zz) / 3 and s_v^2 = (S_vxvx + S_vyvy + S_vzvz) / 3. +inf
 * for a core whose tensor is not positive definite. */
static double or_core_d2(int mode, const double *mean, const double *S, const double *L, int pd,
                         const double *X) {
  double d[6];
  for (int a = 0; a < 6; ++a) d[a] = X[a] - mean[a];
  if (!pd) return INFINITY;
  if (mode != 0) return or_dist6(L, d);
  const double sx2 = (S[0] + S[7] + S[14]) / 3.0, sv2 = (S[21] + S[28] + S[35]) / 3.0;
  return (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / sx2 +
         (d[3] * d[3] + d[4] * d[4] + d[5] * d[5]) / sv2;
}

/* One assignment step of core growth on given points (Sec. 2.3, Eqs. coremeanphase,
 * coredispphase, coredist; the paper's Gaussian-mixture comparison): X [n][6] phase-space
 * points, init[i] the core (0 .. ncore - 1) that point i seeds or -1. Every core's mean
 * and tensor come from its seed points; every unseeded point goes to the core of
 * smallest D^2 under `mode` (or_core_d2; ties: the smaller core; -1 if no core is
 * finite); seeds keep their core. Returns the number of cores whose tensor is positive
 * definite. */
int or_core_assign(const double *X, int64_t n, const int32_t *init, int ncore, int mode,
                   int32_t *out) {
  double *mean = (double *)malloc((size_t)(ncore > 0 ? ncore : 1) * 6 * sizeof(double));
  double *S = (double *)malloc((size_t)(ncore > 0 ? ncore : 1) * 36 * sizeof(double));
  double *L = (double *)malloc((size_t)(ncore > 0 ? ncore : 1) * 36 * sizeof(double));
  int *pd = (int *)malloc((size_t)(ncore > 0 ? ncore : 1) * sizeof(int));
  uint8_t *sel = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
  int npd = 0;
  for (int c = 0; c < ncore; ++c) {
    for (int64_t i = 0; i < n; ++i) sel[i] = init[i] == c;
    pd[c] = or_phase_moments(X, n, sel, mean + 6 * c, S + 36 * c) > 0 &&
            or_chol6(S + 36 * c, L + 36 * c);
    npd += pd[c];
  }
  for (int64_t i = 0; i < n; ++i) {
    out[i] = init[i];
    if (init[i] >= 0) continue;
    double best = INFINITY;
    for (int c = 0; c < ncore; ++c) {
      const double D2 = or_core_d2(mode, mean + 6 * c, S + 36 * c, L + 36 * c, pd[c], X + 6 * i);
      if (D2 < best) { best = D2; out[i] = c; }
    }
  }
  free(sel); free(pd); free(L); free(S); free(mean);
  return npd;
}

/* Core search followed by core cleaning and core growth inside one halo (Sec. 2.3,
 * "Core Growth & Mass Reconstruction" and "Cleaning the Catalogue"; Eqs. coremeanphase,
 * coredispphase, coredist, coresig). The search is or_core_search's. Then:
 *  - cores: the candidate cores of every level and the primary core, each with its
 *    members at the end of the search;
 *  - cleaning (Eq. coresig): candidate core n of level l_n is kept iff
 *    D^2(mean_p -> core n) >= beta_c, with core n's own tensor and mean_p the mean of the
 *    primary group of level l_n (the largest group of that loop: the members searched
 *    at loop l_n + 1, plus the final primary core). A core whose tensor is not positive
 *    definite is dropped. A dropped core's members return to the untagged background;
 *  - growth, only when at least one candidate core is kept: for l = n_loop - 1 down to 0,
 *    the active cores are the primary core and the kept candidate cores of level >= l;
 *    every untagged member that was last searched at loop l is assigned to the active
 *    core of smallest D^2 (ties: the smaller label; cores whose tensor is not positive
 *    definite are skipped), all members of one level against the tensors held at the
 *    start of that level. Mode 2 (Table A1 default) recomputes every active core's
 *    mean and tensor from its current members at the start of each level, mode 1 keeps
 *    the tensors of the cores as found, mode 0 uses the scalar form of or_core_d2.
 *   out_core, out_level: as or_core_search; out_grown [nh]: the core label of each
 *   member after cleaning and growth, -1 for none; out_gap [nh] (may be NULL): for a
 *   member assigned by distance, the second smallest D^2 minus the smallest (+inf if
 *   one core was finite), else NaN.
 * Returns the number of cores kept (kept candidate cores + the primary core). */
int64_t or_core_grow(const int64_t *upos, const float *vel, const int32_t *members, int64_t nh,
                     const int32_t *lab6, double lx, double lv, double ax, double av, int n_loop,
                     double f_c, double an, int32_t nmin, double beta_c, int mode,
                     int32_t *out_core, int32_t *out_level, int32_t *out_grown, double *out_gap) {
  const size_t nb = (size_t)(nh > 0 ? nh : 1);
  int32_t *searched = (int32_t *)malloc(nb * sizeof(int32_t));
  int32_t prim_label, prim_lev;
  or_core_loop(upos, vel, members, nh, lab6, lx, lv, ax, av, n_loop, f_c, an, nmin, out_core,
               out_level, searched, &prim_label, &prim_lev);
  for (int64_t i = 0; i < nh; ++i) {
    out_grown[i] = out_core[i];
    if (out_gap) out_gap[i] = NAN;
  }
  if (prim_label < 0) { free(searched); return 0; }
  double *X = (double *)malloc(nb * 6 * sizeof(double));  /* (x, y, z, vx, vy, vz) rows */
  for (int64_t i = 0; i < nh; ++i) {
    const float *v = vel + 3 * (int64_t)members[i];
    for (int a = 0; a < 3; ++a) {
      X[6 * i + a] = (double)upos[3 * i + a];
      X[6 * i + 3 + a] = (double)v[a];
    }
  }
  /* cores, in increasing label order: a core's label is its minimum member index, so
   * its root is the member whose own index is the label */
  int64_t nc = 0;
  for (int64_t i = 0; i < nh; ++i)
    if (out_core[i] == members[i]) nc++;
  int32_t *clab = (int32_t *)malloc((size_t)nc * sizeof(int32_t));
  int32_t *clev = (int32_t *)malloc((size_t)nc * sizeof(int32_t));
  uint8_t *alive = (uint8_t *)malloc((size_t)nc);
  double *cmean = (double *)malloc((size_t)nc * 6 * sizeof(double));
  double *cS = (double *)malloc((size_t)nc * 36 * sizeof(double));
  double *cL = (double *)malloc((size_t)nc * 36 * sizeof(double));
  int *cpd = (int *)malloc((size_t)nc * sizeof(int));
  int32_t *cur = (int32_t *)malloc(nb * sizeof(int32_t));  /* core index of each member */
  int32_t *nxt = (int32_t *)malloc(nb * sizeof(int32_t));
  uint8_t *sel = (uint8_t *)malloc(nb);
  int64_t k = 0, pc = -1;
  for (int64_t i = 0; i < nh; ++i)
    if (out_core[i] == members[i]) {
      clab[k] = out_core[i];
      clev[k] = out_level[i];
      alive[k] = 1;
      if (out_core[i] == prim_label) pc = k;
      k++;
    }
  for (int64_t i = 0; i < nh; ++i) {
    cur[i] = -1;
    if (out_core[i] < 0) continue;
    int64_t lo = 0, hi = nc;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (clab[mid] < out_core[i]) lo = mid + 1; else hi = mid;
    }
    cur[i] = (int32_t)lo;
  }
  /* the cores as found (Eqs. coremeanphase, coredispphase) */
  for (int64_t c = 0; c < nc; ++c) {
    for (int64_t i = 0; i < nh; ++i) sel[i] = cur[i] == c;
    or_phase_moments(X, nh, sel, cmean + 6 * c, cS + 36 * c);
    cpd[c] = or_chol6(cS + 36 * c, cL + 36 * c);
  }
  /* cleaning (Eq. coresig) */
  int64_t kept = 0;
  for (int64_t c = 0; c < nc; ++c) {
    if (c == pc) continue;
    for (int64_t i = 0; i < nh; ++i) sel[i] = searched[i] >= clev[c] + 1 || out_core[i] == prim_label;
    double mp[6], Sp[36];
    or_phase_moments(X, nh, sel, mp, Sp);
    double d[6];
    for (int a = 0; a < 6; ++a) d[a] = mp[a] - cmean[6 * c + a];
    const int keep = cpd[c] && or_dist6(cL + 36 * c, d) >= beta_c;
    alive[c] = (uint8_t)keep;
    kept += keep;
  }
  for (int64_t i = 0; i < nh; ++i)
    if (cur[i] >= 0 && !alive[cur[i]]) cur[i] = -1;
  if (kept > 0) {
    for (int l = n_loop - 1; l >= 0; --l) {
      if (mode == 2)
        for (int64_t c = 0; c < nc; ++c) {
          if (!alive[c] || (c != pc && clev[c] < l)) continue;
          for (int64_t i = 0; i < nh; ++i) sel[i] = cur[i] == c;
          or_phase_moments(X, nh, sel, cmean + 6 * c, cS + 36 * c);
          cpd[c] = or_chol6(cS + 36 * c, cL + 36 * c);
        }
      for (int64_t i = 0; i < nh; ++i) {
        nxt[i] = cur[i];
        if (cur[i] >= 0 || searched[i] != l) continue;
        double b1 = INFINITY, b2 = INFINITY;
        int64_t bc = -1;
        for (int64_t c = 0; c < nc; ++c) {  /* increasing labels: ties keep the smaller */
          if (!alive[c] || (c != pc && clev[c] < l)) continue;
          const double D2 =
              or_core_d2(mode, cmean + 6 * c, cS + 36 * c, cL + 36 * c, cpd[c], X + 6 * i);
          if (!(D2 < INFINITY)) continue;
          if (bc < 0 || D2 < b1) { b2 = b1; b1 = D2; bc = c; }
          else if (D2 < b2) b2 = D2;
        }
        if (bc >= 0) {
          nxt[i] = (int32_t)bc;
          if (out_gap) out_gap[i] = b2 - b1;
        }
      }
      for (int64_t i = 0; i < nh; ++i) cur[i] = nxt[i];
    }
  }
  for (int64_t i = 0; i < nh; ++i) out_grown[i] = cur[i] >= 0 ? clab[cur[i]] : -1;
  free(sel); free(nxt); free(cur); free(cpd); free(cL); free(cS); free(cmean); free(alive);
  free(clev); free(clab); free(X); free(searched);
  return kept + 1;
}

/* ------------------------------------------------------- field 6DFOF (Sec. 2.1) */

/* Field halos (Sec. 2.1, Eq. fof6d): every 3DFOF group of >= nmin members is split by a
 * 6DFOF inside it. For group k, sigma_v,k = |Sigma_k|^(1/6) of its velocity dispersion
 * tensor (Table A2, sigV; or_halo_frame) and lv = alpha_v sigma_v,k (Table 1, alpha_v);
 * members i, j are linked iff dx^2/lx^2 + dv^2/lv^2 < 1, dx the separation of the
 * unwrapped positions. Groups of these links with >= nmin members keep the minimum
 * particle index as label; every other particle gets -1. A group with sigma_v,k = 0
 * has lv = 0, so dv^2/lv^2 is +inf or NaN and no pair links (IEEE arithmetic, the
 * paper being silent). rows (may be NULL): per 3D group, in label order,
 * {label3, N_H, sigma_v, lx^2, lv^2}. Returns the number of 3D groups, -1 on error. */
int64_t or_field6d(const int32_t *pos, const float *vel, int64_t n, const int32_t *label3,
                   double lx, double alpha_v, int32_t nmin, int32_t *label6, double *rows) {
  for (int64_t i = 0; i < n; ++i) label6[i] = -1;
  int64_t H = or_halos(label3, n, nmin, NULL, NULL);
  if (H < 0) return -1;
  int64_t *off = (int64_t *)malloc((size_t)(H + 1) * sizeof(int64_t));
  int32_t *mem = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  or_halos(label3, n, nmin, off, mem);
  for (int64_t h = 0; h < H; ++h) {
    const int32_t *m = mem + off[h];
    const int64_t nh = off[h + 1] - off[h];
    int64_t *up = (int64_t *)malloc((size_t)nh * 3 * sizeof(int64_t));
    uint8_t *cand = (uint8_t *)malloc((size_t)nh);
    int32_t *l6 = (int32_t *)malloc((size_t)nh * sizeof(int32_t));
    or_unwrap(pos, m, nh, up);
    double frame[4];
    or_halo_frame(vel, m, nh, frame);
    const double lv = alpha_v * frame[3];
    double prm[5] = {lx * lx, lv * lv, frame[0], frame[1], frame[2]};
    for (int64_t k = 0; k < nh; ++k) cand[k] = 1;
    or_fof6d_halo(up, vel, m, nh, cand, prm, 0.0, 0.0, 1, 0, nmin, l6);
    for (int64_t k = 0; k < nh; ++k) label6[m[k]] = l6[k];
    if (rows) {
      double *r = rows + 5 * h;
      r[0] = (double)m[0];
      r[1] = (double)nh;
      r[2] = frame[3];
      r[3] = prm[0];
      r[4] = prm[1];
    }
    free(up);
    free(cand);
    free(l6);
  }
  free(off);
  free(mem);
  return H;
}

/* ------------------------------------------------------------ full pipeline */

typedef struct {
  int32_t nse, nv;
  double f_cell;
  int32_t ncell_min, nmin, nsearch_min;
  double ell_th, v_ratio, theta_op;
  int32_t use_lv, use_vr_theta, split_rule;
  int32_t fit_nbins_min, fit_nbins_max, fit_iters;
} or_params;

/* Per-halo output row (or_pipeline): */
#define OR_HS 12 /* label, N_H, searched, Rbar, sigma_R, vframe[3], sigma_host, lx2, lv2, ncells */

/* The whole hot path on one box (Sec. 2.1-2.2, Fig. 2 first pass):
 * 3D FOF -> halos (N_H >= nmin) -> f_l for every halo member -> for halos with
 * N_H >= nsearch_min: background cells, R, skew-Gaussian fit, ell -> 6D linking of the
 * outliers (ell >= ell_th) with lx2 = lx_sub^2 and lv2 = (alpha_lv sigma_host)^2.
 * Per-particle outputs are NaN / -1 outside the relevant halos. halo_stats [H][OR_HS]
 * (may be NULL) must hold n / max(nmin,1) + 1 rows. Returns H, or -1. */
int64_t or_pipeline(const int32_t *pos, const float *vel, int64_t n, int64_t link_d2,
                    double lx_sub, double alpha_lv, const or_params *P, int32_t *label3,
                    double *f_l, double *R, double *ell, int32_t *label6, double *halo_stats) {
  if (or_fof3d(pos, n, link_d2, label3) != 0) return -1;
  for (int64_t i = 0; i < n; ++i) {
    f_l[i] = NAN; R[i] = NAN; ell[i] = NAN; label6[i] = -1;
  }
  int64_t H = or_halos(label3, n, P->nmin, NULL, NULL);
  if (H < 0) return -1;
  int64_t *off = (int64_t *)malloc((size_t)(H + 1) * sizeof(int64_t));
  int32_t *mem = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  or_halos(label3, n, P->nmin, off, mem);
  for (int64_t h = 0; h < H; ++h) {
    int64_t nh = off[h + 1] - off[h];
    const int32_t *m = mem + off[h];
    int64_t *up = (int64_t *)malloc((size_t)nh * 3 * sizeof(int64_t));
    double *fl = (double *)malloc((size_t)nh * sizeof(double));
    double *r = (double *)malloc((size_t)nh * sizeof(double));
    or_unwrap(pos, m, nh, up);
    or_velden_halo(up, vel, m, nh, P->nse, P->nv, fl);
    for (int64_t k = 0; k < nh; ++k) f_l[m[k]] = fl[k];
    double frame[4];
    or_halo_frame(vel, m, nh, frame);
    double *hs = halo_stats ? halo_stats + OR_HS * h : NULL;
    if (hs) {
      for (int c = 0; c < OR_HS; ++c) hs[c] = NAN;
      hs[0] = (double)m[0];
      hs[1] = (double)nh;
      hs[2] = 0.0;
      for (int c = 0; c < 4; ++c) hs[5 + c] = frame[c];
    }
    if (nh >= P->nsearch_min) {
      int64_t nl = or_background_halo(up, vel, m, nh, fl, P->f_cell, P->ncell_min,
                                      P->split_rule, r, NULL, NULL, NULL);
      double fit[8];
      or_ell_fit(r, nh, P->fit_nbins_min, P->fit_nbins_max, P->fit_iters, fit);
      uint8_t *cand = (uint8_t *)malloc((size_t)nh);
      int32_t *l6 = (int32_t *)malloc((size_t)nh * sizeof(int32_t));
      for (int64_t k = 0; k < nh; ++k) {
        double e = (r[k] - fit[0]) / fit[1];
        R[m[k]] = r[k];
        ell[m[k]] = e;
        cand[k] = e >= P->ell_th; /* false for NaN */
      }
      double prm[5] = {lx_sub * lx_sub, (alpha_lv * frame[3]) * (alpha_lv * frame[3]),
                       frame[0], frame[1], frame[2]};
      or_fof6d_halo(up, vel, m, nh, cand, prm, P->v_ratio, P->theta_op, P->use_lv,
                    P->use_vr_theta, P->nmin, l6);
      for (int64_t k = 0; k < nh; ++k) label6[m[k]] = l6[k];
      if (hs) {
        hs[2] = 1.0;
        hs[3] = fit[0];
        hs[4] = fit[1];
        hs[9] = prm[0];
        hs[10] = prm[1];
        hs[11] = (double)nl;
      }
      free(cand);
      free(l6);
    }
    free(up);
    free(fl);
    free(r);
  }
  free(off);
  free(mem);
  return H;
}

/* Significance level of outlier groups (Eq. ellsig): mean of a unit Gaussian's tail
 * above ell_th, sqrt(2/pi) exp(-ell_th^2/2) / (1 - erf(ell_th/sqrt 2)). */
double or_ell_bar(double ell_th) {
  return sqrt(2.0 / OR_PI) * exp(-0.5 * ell_th * ell_th) / erfc(ell_th / sqrt(2.0));
}
