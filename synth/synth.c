/*
 * Seeded synthetic particle boxes: clustered dark-matter-like particle sets on a
 * periodic 2^21 integer lattice, standing in for N-body snapshots.
 *
 * This module only draws inputs. It holds none of the halo finder's arithmetic
 * (no linking, no densities, no background model); both the CUDA library and the
 * oracle consume what it writes.
 *
 * Random numbers: counter-based splitmix64 (Steele, Lea & Flood 2014), so every
 * particle's draws depend only on (seed, stream, counter) and the output is
 * identical for any thread count.
 *
 * Recipe (all lengths in lattice units, L = 2^21 per axis; velocities in km/s):
 *  - a halo of n_h particles has r200 = (3 n_h / (4 pi 200 nbar))^(1/3), nbar = N / L^3;
 *  - NFW positions: radius x r_s with m(x) = ln(1+x) - x/(1+x) inverted by bisection up
 *    to the concentration c, isotropic direction;
 *  - Plummer subhalos: r = a / sqrt(u^(-2/3) - 1) truncated at 10a, a = r200(n_sub)/5,
 *    centre drawn from the host's NFW profile;
 *  - velocities isotropic Gaussian (host sigma, subhalo sigma = host sigma * (n_sub/n_h)^(1/3)),
 *    subhalos carry a bulk offset;
 *  - the remaining particles are uniform with sigma_bg km/s;
 *  - positions are rounded to the lattice and wrapped; the particle order is scrambled
 *    by an affine bijection so halo members are not contiguous in index space.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SY_L 2097152.0
#define SY_LI 2097152LL
#define SY_PI 3.14159265358979323846

static inline uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return sm64(sm64(seed ^ sm64(stream * 0xD1B54A32D192ED03ULL + 1)) + ctr);
}
/* uniform in (0,1) */
static inline double u01(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return ((double)(draw(seed, stream, ctr) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
static inline double gauss(uint64_t seed, uint64_t stream, uint64_t ctr) {
  double a = u01(seed, stream, 2 * ctr), b = u01(seed, stream, 2 * ctr + 1);
  return sqrt(-2.0 * log(a)) * cos(2.0 * SY_PI * b);
}

/* blob kinds */
enum { BLOB_UNIFORM = 0, BLOB_NFW = 1, BLOB_PLUMMER = 2 };

typedef struct {
  int kind;
  int64_t start, count;
  double cx, cy, cz;      /* centre */
  double scale, rmax;     /* NFW: r_s and concentration c; Plummer: a and 10a */
  double vx, vy, vz;      /* bulk velocity */
  double sigma;           /* per-component velocity dispersion */
  int32_t host, sub;      /* truth ids (-1 = none) */
} blob_t;

static double nfw_m(double x) { return log1p(x) - x / (1.0 + x); }

/* radius in units of r_s for cumulative fraction u of an NFW profile truncated at c */
static double nfw_invert(double u, double c) {
  double target = u * nfw_m(c), lo = 0.0, hi = c;
  for (int it = 0; it < 44; ++it) {
    double mid = 0.5 * (lo + hi);
    if (nfw_m(mid) < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static void iso_dir(uint64_t seed, uint64_t stream, uint64_t ctr, double *d) {
  double cz = 2.0 * u01(seed, stream, ctr) - 1.0;
  double ph = 2.0 * SY_PI * u01(seed, stream, ctr + 1);
  double sz = sqrt(fmax(0.0, 1.0 - cz * cz));
  d[0] = sz * cos(ph); d[1] = sz * sin(ph); d[2] = cz;
}

static double r200_of(double nh, double nbar) {
  return cbrt(3.0 * nh / (4.0 * SY_PI * 200.0 * nbar));
}

/* power law dN/dM ~ M^-alpha on [lo, hi] by inverse CDF */
static double powlaw(double u, double lo, double hi, double alpha) {
  double e = 1.0 - alpha;
  return pow(pow(lo, e) + u * (pow(hi, e) - pow(lo, e)), 1.0 / e);
}

typedef struct {
  blob_t *b;
  int64_t nb, cap;
} blist;

static blob_t *push(blist *l) {
  if (l->nb == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 1024;
    l->b = (blob_t *)realloc(l->b, (size_t)l->cap * sizeof(blob_t));
  }
  memset(&l->b[l->nb], 0, sizeof(blob_t));
  l->b[l->nb].host = -1;
  l->b[l->nb].sub = -1;
  return &l->b[l->nb++];
}

/* Adds one host of nh particles (NFW, concentration c) with its subhalos (appended
 * after it). sub_mode 0: two subhalos of 5% mass each at a 2 sigma_host bulk offset in a
 * random direction (small clustered box); 1: power-law population holding ~10% of the
 * host mass, offsets ~ N(0, sigma_host^2) per axis (mass-function boxes). */
static void add_host(blist *l, uint64_t seed, int32_t hid, int64_t nh, double conc,
                     double sigma, double nbar, int sub_mode, int32_t *nsub_total,
                     double sigma_bg) {
  uint64_t hs = 1000003ULL * (uint64_t)(hid + 1);
  double r200 = r200_of((double)nh, nbar);
  double c[3] = {u01(seed, hs, 0) * SY_L, u01(seed, hs, 1) * SY_L, u01(seed, hs, 2) * SY_L};
  double bulk[3] = {sigma_bg * gauss(seed, hs, 3), sigma_bg * gauss(seed, hs, 4),
                    sigma_bg * gauss(seed, hs, 5)};
  int64_t subs[4096];
  int nsubs = 0;
  int64_t insub = 0;
  if (sub_mode == 0) {
    int64_t m = (int64_t)llround(0.05 * (double)nh);
    if (m >= 2) { subs[nsubs++] = m; subs[nsubs++] = m; insub = 2 * m; }
  } else if (nh >= 200) {
    int64_t target = (int64_t)llround(0.10 * (double)nh);
    for (int k = 0; k < 4096 && insub < target; ++k) {
      double mu = powlaw(u01(seed, hs, 100 + k), 1e-3, 1e-1, 1.9);
      int64_t m = (int64_t)llround(mu * (double)nh);
      if (m > target - insub) m = target - insub;
      if (m < 20) {
        if (target - insub < 20) break;
        continue;
      }
      subs[nsubs++] = m;
      insub += m;
    }
  }
  blob_t *h = push(l);
  h->kind = BLOB_NFW;
  h->count = nh - insub;
  h->cx = c[0]; h->cy = c[1]; h->cz = c[2];
  h->scale = r200 / conc;
  h->rmax = conc;
  h->vx = bulk[0]; h->vy = bulk[1]; h->vz = bulk[2];
  h->sigma = sigma;
  h->host = hid;
  for (int s = 0; s < nsubs; ++s) {
    uint64_t ss = hs + 7919ULL * (uint64_t)(s + 1);
    double rr = nfw_invert(u01(seed, ss, 0), conc) * (r200 / conc);
    double d[3];
    iso_dir(seed, ss, 1, d);
    double off[3];
    if (sub_mode == 0) {
      double vd[3];
      iso_dir(seed, ss, 3, vd);
      for (int a = 0; a < 3; ++a) off[a] = 2.0 * sigma * vd[a];
    } else {
      for (int a = 0; a < 3; ++a) off[a] = sigma * gauss(seed, ss, 5 + a);
    }
    blob_t *b = push(l);
    b->kind = BLOB_PLUMMER;
    b->count = subs[s];
    b->cx = c[0] + rr * d[0]; b->cy = c[1] + rr * d[1]; b->cz = c[2] + rr * d[2];
    b->scale = r200_of((double)subs[s], nbar) / 5.0;
    b->rmax = 10.0 * b->scale;
    b->vx = bulk[0] + off[0]; b->vy = bulk[1] + off[1]; b->vz = bulk[2] + off[2];
    b->sigma = sigma * cbrt((double)subs[s] / (double)nh);
    b->host = hid;
    b->sub = (*nsub_total)++;
  }
}

/* Particles in kind 2's nhost hosts (the N to pass to synth_box). */
int64_t synth_hosts_total(uint64_t seed, int nhost, double size_lo, double size_hi) {
  int64_t tot = 0;
  for (int h = 0; h < nhost; ++h)
    tot += (int64_t)llround(powlaw(u01(seed, 78, (uint64_t)h), size_lo, size_hi, 1.9));
  return tot;
}

static int64_t gcd64(int64_t a, int64_t b) {
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}

/*
 * kind 0: few hosts (nhost of them, concentration conc_lo, sizes log-uniform in
 *         [size_lo, size_hi], redrawn while the total exceeds 0.75 N), two subhalos each.
 * kind 1: hosts with sizes from dN/dM ~ M^-1.9 on [size_lo, size_hi] until frac_halo*N
 *         particles are in hosts; c uniform in [conc_lo, conc_hi];
 *         sigma_host = sigma_host0 (n_h/1000)^(1/3); power-law subhalos.
 * kind 2: exactly nhost hosts drawn as in kind 1 but without the frac_halo cap, and no
 *         background: N must be synth_hosts_total(seed, nhost, size_lo, size_hi)
 *         (pre-labelled halos: host_id gives each particle's halo).
 * Writes pos[N][3] (int32 lattice), vel[N][3] (float km/s), and optional truth ids
 * host_id[N], sub_id[N] (-1 = none). Returns the number of hosts, or -1 on bad input.
 */
int64_t synth_box(int64_t N, int kind, uint64_t seed, int nhost, double frac_halo,
                  double size_lo, double size_hi, double conc_lo, double conc_hi,
                  double sigma_host0, double sigma_bg, int32_t *pos, float *vel,
                  int32_t *host_id, int32_t *sub_id) {
  if (N <= 0 || !pos || !vel) return -1;
  double nbar = (double)N / (SY_L * SY_L * SY_L);
  blist l = {0, 0, 0};
  int32_t nsub = 0;
  int64_t in_halo = 0;
  int32_t hid = 0;
  if (kind == 0) {
    int64_t sizes[256];
    if (nhost > 256) nhost = 256;
    for (int attempt = 0; attempt < 10000; ++attempt) {
      int64_t tot = 0;
      for (int h = 0; h < nhost; ++h) {
        double u = u01(seed, 77, (uint64_t)attempt * 256 + h);
        sizes[h] = (int64_t)llround(exp(log(size_lo) + u * (log(size_hi) - log(size_lo))));
        tot += sizes[h];
      }
      if ((double)tot <= 0.75 * (double)N) break;
    }
    for (int h = 0; h < nhost; ++h) {
      if (in_halo + sizes[h] > N) break;
      add_host(&l, seed, hid++, sizes[h], conc_lo, sigma_host0, nbar, 0, &nsub, sigma_bg);
      in_halo += sizes[h];
    }
  } else if (kind == 2) {
    for (int h = 0; h < nhost; ++h) {
      int64_t nh = (int64_t)llround(powlaw(u01(seed, 78, (uint64_t)h), size_lo, size_hi, 1.9));
      if (in_halo + nh > N) { free(l.b); return -1; }
      double conc = conc_lo + (conc_hi - conc_lo) * u01(seed, 79, (uint64_t)h);
      double sig = sigma_host0 * cbrt((double)nh / 1000.0);
      add_host(&l, seed, hid++, nh, conc, sig, nbar, 1, &nsub, sigma_bg);
      in_halo += nh;
    }
    if (in_halo != N) { free(l.b); return -1; }
  } else {
    int64_t target = (int64_t)llround(frac_halo * (double)N);
    for (uint64_t k = 0; in_halo < target; ++k) {
      int64_t nh = (int64_t)llround(powlaw(u01(seed, 78, k), size_lo, size_hi, 1.9));
      if (nh > target - in_halo) nh = target - in_halo;
      if (nh < (int64_t)size_lo) break;
      double conc = conc_lo + (conc_hi - conc_lo) * u01(seed, 79, k);
      double sig = sigma_host0 * cbrt((double)nh / 1000.0);
      add_host(&l, seed, hid++, nh, conc, sig, nbar, 1, &nsub, sigma_bg);
      in_halo += nh;
    }
  }
  blob_t *bg = push(&l);
  bg->kind = BLOB_UNIFORM;
  bg->count = N - in_halo;
  bg->sigma = sigma_bg;
  int64_t off = 0;
  for (int64_t b = 0; b < l.nb; ++b) { l.b[b].start = off; off += l.b[b].count; }

  /* affine bijection on [0, N): generated particle g goes to slot (a g + c) mod N */
  int64_t a = (int64_t)(0x9E3779B97F4A7C15ULL % (uint64_t)N) | 1;
  while (a > 1 && gcd64(a, N) != 1) a += 2;
  if (N == 1) a = 1;
  int64_t cshift = (int64_t)(sm64(seed) % (uint64_t)N);

#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < N; ++g) {
    /* find the blob that owns g */
    int64_t lo = 0, hi = l.nb - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (l.b[mid].start <= g) lo = mid; else hi = mid - 1;
    }
    const blob_t *b = &l.b[lo];
    uint64_t st = 0xC0FFEEULL + (uint64_t)g;
    double p[3], v[3];
    if (b->kind == BLOB_UNIFORM) {
      for (int k = 0; k < 3; ++k) p[k] = u01(seed, st, k) * SY_L;
    } else {
      double r;
      if (b->kind == BLOB_NFW) {
        r = nfw_invert(u01(seed, st, 0), b->rmax) * b->scale;
      } else {
        double u = u01(seed, st, 0);
        do {
          r = b->scale / sqrt(pow(u, -2.0 / 3.0) - 1.0);
          if (r <= b->rmax) break;
          u *= 0.5; /* rare: fold the truncated tail back inside */
        } while (1);
      }
      double d[3];
      iso_dir(seed, st, 1, d);
      p[0] = b->cx + r * d[0];
      p[1] = b->cy + r * d[1];
      p[2] = b->cz + r * d[2];
    }
    v[0] = b->vx + b->sigma * gauss(seed, st, 8);
    v[1] = b->vy + b->sigma * gauss(seed, st, 9);
    v[2] = b->vz + b->sigma * gauss(seed, st, 10);
    int64_t slot = (int64_t)(((__int128)a * g + cshift) % N);
    for (int k = 0; k < 3; ++k) {
      int64_t q = (int64_t)floor(p[k]);
      q %= SY_LI;
      if (q < 0) q += SY_LI;
      pos[3 * slot + k] = (int32_t)q;
      vel[3 * slot + k] = (float)v[k];
    }
    if (host_id) host_id[slot] = b->host;
    if (sub_id) sub_id[slot] = b->sub;
  }
  int64_t nh_out = hid;
  free(l.b);
  return nh_out;
}
