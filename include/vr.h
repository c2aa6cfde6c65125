/*
 * vr.h — C ABI of the GB300 (sm_103a) VELOCIraptor substructure hot path.
 *
 * Method: Elahi et al. 2019, "Hunting for Galaxies and Halos in simulations with
 * VELOCIraptor", Sec. 2.1 (field halos, Eq. fof3d) and Sec. 2.2 (subhalos and streams:
 * local velocity density, background model Eqs. fvbg, S, meanpos-meandispvel,
 * cellinterp, log ratio R, skew-Gaussian fit Eqs. skewgaus/ell, phase-space linking
 * Eq. linkingcriteria with the 6D term of Eq. fof6d).
 *
 * Conventions for every call:
 *  - All array arguments are DEVICE pointers owned by the caller. Inputs are never
 *    modified. Particle arrays are indexed by particle index i in [0, n), n < 2^31.
 *  - Positions are int32 [n][3] (x, y, z interleaved) on a periodic lattice of 2^21
 *    points per axis, values in [0, 2^21). Velocities are float32 [n][3] (km/s).
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns a vr_status. Argument errors are detected before any work is
 *    enqueued. Device-side errors (unsupported geometry detected in a kernel) are
 *    reported by the NEXT call that synchronises (vr_sync or a call that reads sizes
 *    back), through its status and vr_last_error().
 *  - Scratch memory comes from the caller's workspace `ws` of `ws_bytes` bytes (device
 *    memory, 256-byte aligned); vr_workspace_size() gives the bytes needed for n
 *    particles. No call allocates device memory. Calls that share a workspace must be
 *    ordered on one stream.
 *  - Labels are canonical: the minimum particle index of the group.
 *  - A context (vr_ctx) holds pinned host staging for small read-backs and the last
 *    error string; it is not thread-safe (one host thread per context).
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VR_OK = 0,
  VR_ERR_INVALID_ARG = 1,        /* bad pointer, size or parameter */
  VR_ERR_CUDA = 2,               /* a CUDA runtime call failed */
  VR_ERR_WORKSPACE_TOO_SMALL = 3,/* ws_bytes < vr_workspace_size() */
  VR_ERR_TIMEOUT = 4,            /* a bounded device wait gave up */
  VR_ERR_DEGENERATE_CELL = 5,    /* reserved: reported as a count, never returned */
  VR_ERR_UNSUPPORTED = 6         /* geometry outside the supported envelope */
} vr_status;

typedef struct vr_ctx vr_ctx;

/* Search parameters. Defaults (vr_params_default) are the paper's (Table 1):
 * N_se = 256, N_v = 32, f_cell = 0.01, ell_th = 2.5, V_r = 2, Theta_op = 0.1 pi,
 * N_min = 20; the remaining fields fix readings the paper leaves open. */
typedef struct {
  int32_t nse;          /* N_se physical neighbours for f_l (Sec. 2.2), 1..1024 */
  int32_t nv;           /* N_v velocity neighbours among them, 1..64, nv <= nse */
  double f_cell;        /* background cell size as a fraction of N_H (Sec. 2.2) */
  int32_t ncell_min;    /* cells below this are raised to min(ncell_min, N_H/8) */
  int32_t nmin;         /* minimum group size N_min (Sec. 2.2), >= 1 */
  int32_t nsearch_min;  /* halos with N_H >= nsearch_min are searched (default 160) */
  double ell_th;        /* outlier threshold ell_th (Eq. linkingcriteria a) */
  double v_ratio;       /* speed ratio V_r (Eq. linkingcriteria c) */
  double theta_op;      /* opening angle Theta_op in radians, < pi/2 (Eq. linkingcriteria d) */
  int32_t use_lv;       /* 1: add the velocity term dv^2/lv^2 of Eq. fof6d to the link test */
  int32_t use_vr_theta; /* 1: apply the V_r and Theta_op criteria */
  int32_t split_rule;   /* 0: split cells along the axis of largest entropy S; 1: smallest */
  int32_t fit_nbins_min;/* R histogram bins: clamp(ceil(sqrt(N)), min, max) */
  int32_t fit_nbins_max;
  int32_t fit_iters;    /* Levenberg-Marquardt iterations for the skew-Gaussian fit */
} vr_params;

/* Per-halo output row of vr_outlier_ratio / vr_find_substructure (VR_HALO_COLS doubles,
 * halos in increasing label order): */
enum {
  VR_H_LABEL = 0,   /* halo label (minimum particle index) */
  VR_H_NH = 1,      /* N_H */
  VR_H_SEARCHED = 2,/* 1 if N_H >= nsearch_min (background, R, ell computed) */
  VR_H_RBAR = 3,    /* skew-Gaussian mode R-bar (Eq. skewgaus) */
  VR_H_SIGR = 4,    /* skew-Gaussian width sigma_R */
  VR_H_VFX = 5,     /* halo mean velocity (frame for V_r, Theta_op) */
  VR_H_VFY = 6,
  VR_H_VFZ = 7,
  VR_H_SIGMA = 8,   /* sigma_host = |Sigma_halo|^(1/6) (Table A2 sigma_v) */
  VR_H_LX2 = 9,     /* squared spatial linking length used by vr_fof6d */
  VR_H_LV2 = 10,    /* squared velocity linking length used by vr_fof6d */
  VR_H_NCELLS = 11, /* number of background cells */
  VR_HALO_COLS = 12
};

/* Fills p with the defaults above. */
void vr_params_default(vr_params *p);

/* Creates a context on CUDA device `device`. *out is NULL on failure. */
vr_status vr_create(vr_ctx **out, int device);
void vr_destroy(vr_ctx *ctx);

/* Last error message of ctx (empty string if none). Owned by ctx. */
const char *vr_last_error(const vr_ctx *ctx);

/* Host-side logging of ctx to stderr (the paper's code has a verbosity flag; the levels
 * here are this library's own): 0 = silent (the default), 1 = every error as it is
 * recorded (the text vr_last_error returns, prefixed "vr: "), 2 = also one line per
 * vr_fof3d / vr_find_substructure call with n and its status. Returns VR_ERR_INVALID_ARG
 * for a NULL ctx or a level outside [0, 2]. */
vr_status vr_set_log_level(vr_ctx *ctx, int level);

/* Bytes of workspace needed by any call below for n particles with parameters p
 * (p may be NULL for defaults). */
vr_status vr_workspace_size(vr_ctx *ctx, int64_t n, const vr_params *p, size_t *bytes);

/* Waits for `stream` and reports device-side errors raised by earlier calls. */
vr_status vr_sync(vr_ctx *ctx, void *stream);

/* 3D friends-of-friends (Sec. 2.1, Eq. fof3d): particles i, j are linked iff their
 * minimum-image squared separation is < link_d2 (lattice units squared; the strict
 * inequality of Eq. fof3d; link_d2 = floor(ell_x^2) + 1 for a non-integer ell_x^2);
 * groups are the connected components.
 *   pos    int32 [n][3], lattice positions in [0, 2^21)
 *   link_d2 1 <= link_d2 <= 2^38 (linking length at most 2^19 lattice units)
 *   label  int32 [n] out: minimum particle index of i's group
 * Errors: VR_ERR_INVALID_ARG for NULL pointers with n > 0, n < 0, n >= 2^31, or link_d2
 * out of range. n = 0 is a no-op. */
vr_status vr_fof3d(vr_ctx *ctx, const int32_t *pos, int64_t n, int64_t link_d2, int32_t *label,
                   void *ws, size_t ws_bytes, void *stream);

/* Local velocity density (Sec. 2.2): for every particle of a halo (3D group with at
 * least p->nmin members), the N_se nearest members of the same halo in position (by
 * squared separation, ties by particle index, the particle itself included,
 * N_se_eff = min(N_se, N_H)); h = distance in velocity to the N_v-th nearest of that
 * set; f_l = (1/N_se_eff) sum over the set of 15/(8 pi h^3)(1 - |dv|^2/h^2) for |dv| < h
 * (Epanechnikov kernel).
 *   label  int32 [n] 3D labels as written by vr_fof3d (canonical)
 *   f_l    float32 [n] out: f_l in (km/s)^-3; NaN for particles outside halos
 * Halos must span less than half the box per axis (positions are unwrapped about the
 * halo's minimum-index member); a halo may hold at most 2^22 particles.
 * Errors: VR_ERR_INVALID_ARG (pointers, n, parameters); VR_ERR_UNSUPPORTED (halo too
 * large or too extended, reported at the next synchronising call). */
vr_status vr_velden(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                    const int32_t *label, const vr_params *p, float *f_l, void *ws,
                    size_t ws_bytes, void *stream);

/* Outlier ratio (Sec. 2.2) for halos with N_H >= p->nsearch_min: entropy kd-tree cells of
 * N_cell = f_cell N_H particles (raised to min(ncell_min, N_H/8)), FP64 cell moments
 * (Eqs. meanpos, meanvel, meandispvel), inverse-distance interpolation over the
 * particle's cell and its face neighbours (Eq. cellinterp), FP64 Cholesky of the
 * interpolated dispersion tensor, R = ln f_l - ln f_bg (Eq. fvbg); then per halo a
 * skew-Gaussian fit of the binned R distribution (Eq. skewgaus) and
 * ell = (R - R-bar)/sigma_R (Eq. ell).
 *   f_l         float32 [n] from vr_velden
 *   R, ell      float32 [n] out; NaN outside searched halos (R is NaN where the tensor is
 *               not positive definite)
 *   halo_stats  double [n/nmin + 1][VR_HALO_COLS] out (rows for every halo with N_H >=
 *               nmin, in label order; columns VR_H_*; LX2/LV2 are NaN here)
 *   nhalo       int64 host pointer out (may be NULL): number of halos written
 * This call synchronises `stream` to read the halo count. */
vr_status vr_outlier_ratio(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *f_l,
                           int64_t n, const int32_t *label, const vr_params *p, float *R,
                           float *ell, double *halo_stats, int64_t *nhalo, void *ws,
                           size_t ws_bytes, void *stream);

/* Phase-space linking of outliers (Sec. 2.2, Eq. linkingcriteria; with p->use_lv the
 * velocity term of Eq. fof6d is added): inside each halo, candidates i, j (ell >=
 * ell_th; every member when ell is NULL) are linked iff dx^2/lx2 (+ dv^2/lv2) < 1 and,
 * with p->use_vr_theta, 1/V_r <= |u_i|/|u_j| <= V_r and the angle between u_i and u_j is
 * at most Theta_op, where u = v - v_frame. dx^2 is the exact squared lattice separation
 * of the unwrapped positions; the rest is FP64 without fused multiply-add, in the order
 * dv2 = (dvx^2 + dvy^2) + dvz^2, q = dx2/lx2 + dv2/lv2, s = (ux^2 + uy^2) + uz^2,
 * s_i <= V_r^2 s_j, dot >= 0 and dot^2 >= (cos^2(Theta_op) s_i) s_j.
 *   halo_params  double [H][VR_HALO_COLS] rows as written by vr_outlier_ratio, with
 *                VR_H_LX2, VR_H_LV2 and VR_H_VF* filled in; halos whose VR_H_SEARCHED is 0
 *                are skipped
 *   nhalo        number of rows
 *   label6       int32 [n] out: minimum particle index of the linked group for
 *                candidates in groups of >= p->nmin members, -1 otherwise */
vr_status vr_fof6d(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *ell,
                   int64_t n, const int32_t *label, const double *halo_params, int64_t nhalo,
                   const vr_params *p, int32_t *label6, void *ws, size_t ws_bytes,
                   void *stream);

/* Field halos (Sec. 2.1, Eq. fof6d): a 6DFOF inside every 3DFOF halo (labels of >=
 * p->nmin members) that splits dynamically unrelated bridges. For halo k,
 * sigma_v,k = |Sigma_k|^(1/6) of its velocity dispersion tensor (FP64, about the halo's
 * mean velocity, divided by N_H) and lv = alpha_v sigma_v,k (Table 1: alpha_v = 1.25);
 * members i, j are linked iff dx^2/lx^2 + dv^2/lv^2 < 1, evaluated as in vr_fof6d with
 * every member a candidate and V_r / Theta_op off. A halo with sigma_v,k = 0 has lv = 0
 * and links no pair (IEEE division). p->use_lv, p->use_vr_theta and p->ell_th are not
 * used.
 *   lx          spatial linking length in lattice units (0.2 of the mean spacing)
 *   label6      int32 [n] out: minimum particle index of the 6D group for members of
 *               groups of >= p->nmin, -1 otherwise (and outside halos)
 *   halo_stats  double [n/nmin + 1][VR_HALO_COLS] out: LABEL, NH, VF*, SIGMA; LX2 = lx^2,
 *               LV2 = (alpha_v sigma_v)^2, SEARCHED = 1; RBAR, SIGR NaN; NCELLS 0
 *   nhalo       int64 host pointer out (may be NULL): number of 3DFOF halos
 * Errors: VR_ERR_INVALID_ARG for lx <= 0 or alpha_v <= 0, as vr_fof6d otherwise. */
vr_status vr_fof6d_field(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                         const int32_t *label, double lx, double alpha_v, const vr_params *p,
                         int32_t *label6, double *halo_stats, int64_t *nhalo, void *ws,
                         size_t ws_bytes, void *stream);

/* The substructure search of Fig. 2 (first pass) for every halo: vr_velden, then
 * vr_outlier_ratio, then the per-halo linking lengths lx2 = lx_sub^2 and
 * lv2 = (alpha_lv sigma_host)^2, then vr_fof6d on the outliers. Outputs as in those
 * calls; halo_stats gets LX2/LV2 filled in. `batched` selects the launch form, with
 * identical results: 1 = batched, each stage is one launch over all halos; 0 = plain,
 * each stage is launched once per halo that has work in it (halo offsets are read back
 * to the host once). Any other value returns VR_ERR_INVALID_ARG. */
vr_status vr_find_substructure(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                               const int32_t *label, double lx_sub, double alpha_lv,
                               const vr_params *p, int batched, float *f_l, float *R,
                               float *ell, int32_t *label6, double *halo_stats, int64_t *nhalo,
                               void *ws, size_t ws_bytes, void *stream);

/* Two-stage linking (Sec. 2.2, "Linking particles": conservative criteria find the
 * candidate substructures; relaxed criteria then link previously untagged particles to
 * them, and substructures are joined only when the new connections exceed f_merge times
 * the original size of either). The relaxed pass takes, inside every halo whose
 * VR_H_SEARCHED is set, the candidates ell >= ell_th / gamma_ell plus every particle
 * already in a group, and the predicate of vr_fof6d with lx2 gamma_x^2 (evaluated as
 * (lx2 gamma_x) gamma_x), V_r gamma_vr and Theta_op gamma_theta (lv2 and frame
 * unchanged). In this order:
 *  1. the untagged candidates form connected components under the relaxed links among
 *     themselves;
 *  2. a component joins the group with the most relaxed links between its members and
 *     the group's (ties: the smaller label); with no such link it stays untagged;
 *  3. two grown groups A, B are joined iff the relaxed links between their members
 *     number more than f_merge N_o(A) or f_merge N_o(B), N_o the size on input; joins
 *     are transitive;
 *  4. each final group is labelled with its minimum particle index.
 * Table A1 defaults (vr_grow_params_default): gamma_ell 1, gamma_x 2, gamma_vr 1,
 * gamma_theta 1; f_merge 0.25 (Sec. 2.2). */
typedef struct {
  double gamma_ell, gamma_x, gamma_vr, gamma_theta, f_merge;
} vr_grow_params;

void vr_grow_params_default(vr_grow_params *g);

/*   ell, label, halo_params, nhalo  as for vr_fof6d
 *   label6  int32 [n] in/out: the stage-1 labels of vr_fof6d in, the grown labels out
 * Errors: VR_ERR_INVALID_ARG for a factor <= 0, f_merge < 0 or gamma_theta Theta_op >=
 * pi/2; VR_ERR_UNSUPPORTED if a link-count table overflows (more distinct (component,
 * group) or (group, group) pairs than n). This call synchronises `stream`. */
vr_status vr_grow_groups(vr_ctx *ctx, const int32_t *pos, const float *vel, const float *ell,
                         int64_t n, const int32_t *label, const double *halo_params,
                         int64_t nhalo, const vr_params *p, const vr_grow_params *gp,
                         int32_t *label6, void *ws, size_t ws_bytes, void *stream);

/* Core search (Sec. 2.3, "Core Identification", Eq. coreloop) inside every halo of >=
 * p->nsearch_min members. The background starts as the members outside substructure
 * (label6 < 0; every member when label6 is NULL). Loop l = 0 .. n_loop - 1: a 6DFOF
 * (Eq. fof6d, predicate and rounding as in vr_fof6d, V_r / Theta_op off) over the
 * background with lx_l = alpha_x^l lx and lv_l = alpha_v,C^l lv, lv = alpha_v
 * sigma_v (sigma_v = |Sigma|^(1/6) of the halo), each by repeated multiplication;
 * groups count with >= p->nmin and >= f_c N_H alpha_n^l members (also by repeated
 * multiplication, compared as reals). Without such a group the halo's search stops.
 * Otherwise its largest group (ties: smaller label) is the next background, the
 * "primary core", and every other group is a candidate core of level l. The last
 * primary core is labelled at the end. Table 1 defaults (vr_core_params_default):
 * alpha_x,C 0.8, alpha_v,C 1.0, n_loop,C 5, f_C 0.02, alpha_N,C 1.2. */
typedef struct {
  double alpha_x, alpha_v;  /* length factors per loop (alpha_x,C, alpha_v,C) */
  int32_t n_loop;           /* loops n_loop,C */
  double f_c, alpha_n;      /* N_min,C = f_c N_H alpha_n^l */
} vr_core_params;

void vr_core_params_default(vr_core_params *c);

/*   label6      int32 [n] substructure labels (may be NULL)
 *   lx, alpha_v the halo linking length (lattice units) and the velocity factor of the
 *               field 6DFOF (Table 1: 0.2 mean spacing, 1.25)
 *   core, level int32 [n] out: minimum particle index of the member's core and the loop
 *               at which it was found; -1 for particles in no core
 *   ncores      int64 host pointer out (may be NULL): candidate cores + primary cores
 *   halo_stats  double [n/nmin + 1][VR_HALO_COLS] out: frame rows; LX2, LV2 and
 *               SEARCHED hold the last loop's values
 *   nhalo       int64 host pointer out (may be NULL)
 * This call synchronises `stream`. */
vr_status vr_core_search(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                         const int32_t *label, const int32_t *label6, double lx, double alpha_v,
                         const vr_params *p, const vr_core_params *cp, int32_t *core,
                         int32_t *level, int64_t *ncores, double *halo_stats, int64_t *nhalo,
                         void *ws, size_t ws_bytes, void *stream);

/* Core cleaning and core growth (Sec. 2.3, "Cleaning the Catalogue" and "Core Growth &
 * Mass Reconstruction"; Eqs. coremeanphase, coredispphase, coredist, coresig), run
 * after the core search of vr_core_search inside every searched halo. Phase-space
 * points are X = (x, y, z, vx, vy, vz): the member's position unwrapped about the halo
 * (lattice units) and its velocity. A core's mean and dispersion tensor are the plain
 * mean and 1/M second moment of its members' X (unit masses), its distance
 * D^2 = (X - mean)^T Sigma^-1 (X - mean) (Eq. coredist).
 *  - Cleaning (Eq. coresig): a candidate core n of level l_n is kept iff
 *    D^2(mean_p) >= beta_c under core n's tensor, mean_p the mean of the primary group
 *    of loop l_n (the members searched at loop l_n + 1 plus the final primary core). A
 *    core whose tensor is not positive definite is dropped; a dropped core's members
 *    return to the untagged background.
 *  - Growth, in halos that keep a candidate core: for l = n_loop - 1 down to 0, every
 *    untagged member last searched at loop l goes to the active core (the primary core
 *    and the kept candidate cores of level >= l) of smallest D^2, ties to the smaller
 *    label, cores without a positive-definite tensor skipped; all members of a level
 *    use the tensors held at the start of that level.
 *  - mode (Table A1, Use_phase_tensor_core_growth): 2 = every active core's mean and
 *    tensor recomputed from its current members at each level (default); 1 = the
 *    tensors of the cores as found; 0 = the scalar form D^2 = |x - xbar|^2 / s_x^2 +
 *    |v - vbar|^2 / s_v^2, s_x^2 and s_v^2 the mean diagonal of the position and velocity
 *    blocks of the core as found (the paper prints this form without squares; read as
 *    squared).
 * Means and tensors are FP64 sums in an order of the library's choosing, so a D^2 can
 * differ from a sequential sum in its last bits: an assignment whose two smallest D^2
 * differ by a few ulp may go either way. Table 1 / A1 defaults
 * (vr_core_grow_params_default): beta_c = 1, mode = 2. */
typedef struct {
  double beta_c;  /* significance beta_C of Eq. coresig */
  int32_t mode;   /* 0, 1 or 2, as above */
} vr_core_grow_params;

void vr_core_grow_params_default(vr_core_grow_params *g);

/*   pos .. level, halo_stats, nhalo: as for vr_core_search (same outputs)
 *   grown      int32 [n] out: the core label of each particle after cleaning and growth,
 *              -1 for none (substructure members, members of halos that were not
 *              searched, untagged members of halos without growth)
 *   nkept      int64 host pointer out (may be NULL): cores kept (kept candidate cores +
 *              primary cores)
 * Workspace: vr_workspace_size. This call synchronises `stream`. Errors:
 * VR_ERR_INVALID_ARG for the core-search parameter checks, beta_c < 0 or NaN, or a mode
 * other than 0, 1, 2. */
vr_status vr_core_grow(vr_ctx *ctx, const int32_t *pos, const float *vel, int64_t n,
                       const int32_t *label, const int32_t *label6, double lx, double alpha_v,
                       const vr_params *p, const vr_core_params *cp, const vr_core_grow_params *gp,
                       int32_t *core, int32_t *level, int32_t *grown, int64_t *nkept,
                       double *halo_stats, int64_t *nhalo, void *ws, size_t ws_bytes,
                       void *stream);

/* Cleaning of outlier groups (Sec. 2.2, "Cleaning the catalogue", Eq. ellsig). A group
 * of N particles (equal labels >= 0 in label6) is significant iff
 *   <ell> >= ell_bar(p->ell_th) (1 + beta/sqrt(N)),
 * ell_bar(t) = sqrt(2/pi) exp(-t^2/2) / erfc(t/sqrt 2), the mean of a unit Gaussian
 * above t (2.822744797663897 at t = 2.5). A group that is not significant loses its
 * particles in order of smallest ell (ties: smaller particle index first) until it is;
 * a group left with fewer than p->nmin particles is removed. Removed particles get -1;
 * the particles kept get the minimum particle index among them. <ell> is the FP64 sum
 * of the FP32 ell values (exact, hence independent of the order of additions, while a
 * group's sum stays below 2^53 times the FP32 spacing of its smallest ell: 2^31 for
 * ell >= 2) divided by N; the threshold is ell_bar * (1 + beta / sqrt(N)), each
 * operation rounded once.
 *   ell      float32 [n]; must not be NaN for grouped particles (outlier groups hold
 *            ell >= ell_th by construction)
 *   beta     beta_ell >= 0 (Table 1: 1)
 *   label6   int32 [n] in/out
 *   ngroups  int64 host pointer out (may be NULL): groups kept
 * This call synchronises `stream`. Errors: VR_ERR_INVALID_ARG for beta < 0. */
vr_status vr_clean_groups(vr_ctx *ctx, const float *ell, int64_t n, const vr_params *p,
                          double beta, int32_t *label6, int64_t *ngroups, void *ws,
                          size_t ws_bytes, void *stream);

/* ----------------------------------------------------- allocation-free 3D FOF
 * No counterpart in the paper. For callers that cannot allocate device memory at all
 * (for example code running where cudaMalloc is forbidden or unavailable, such as inside
 * another library's allocation-free section, or a host that has handed all device
 * memory to its own pool): the same result as vr_fof3d, but with no context, no
 * workspace argument and no allocation. Its scratch is one static device array of
 * VR_FOF3D_NOALLOC_BYTES bytes compiled into this library, which every GPU that loads
 * the library holds until the process exits.
 *   pos, n, link_d2, label: as for vr_fof3d, with n <= VR_FOF3D_NOALLOC_MAX_N
 *   stream: cudaStream_t on the current device (NULL = legacy default stream)
 * Works on the calling thread's current device. Every call looks up the array's device
 * address in the current context (cudaGetSymbolAddress, which allocates nothing), so
 * calls after a cudaDeviceReset find the reloaded array. All calls share the one array and every call overwrites it: calls whose
 * work overlaps on the GPU (other streams, or host threads on the same device) race and
 * must be serialised by the caller. Returns VR_ERR_INVALID_ARG for n above the maximum
 * or bad arguments, VR_ERR_CUDA if the address lookup or a launch fails; the status code
 * is the only error report. */
#define VR_FOF3D_NOALLOC_MAX_N 131072
#define VR_FOF3D_NOALLOC_BYTES (8u << 20)
vr_status vr_fof3d_noalloc(const int32_t *pos, int64_t n, int64_t link_d2, int32_t *label,
                           void *stream);

/* ---------------------------------------------------------------- measurement
 * (no counterpart in the paper: instrumentation of this library)
 * Per-kernel device timing with CUDA events recorded on the launching stream; off by
 * default. Kernel names: "fof_link", "velden_big", "velden_small", "halo_frame",
 * "cells_build", "cells_build_big", "ratio", "ell_fit", "link6", "clean", "core_link". */

/* Enables (1) or disables (0) event timing of the named kernels for this context. */
vr_status vr_timing_enable(vr_ctx *ctx, int enable);

/* Device time in ms summed over the launches of kernel `name` recorded since the last
 * vr_timing_reset, and the number of those launches. Waits for the recorded events. */
vr_status vr_timing_read(vr_ctx *ctx, const char *name, double *ms, int64_t *launches);

/* Drops all recorded timings. */
vr_status vr_timing_reset(vr_ctx *ctx);

/* Number of kernels this library has launched in the calling process so far (every
 * kernel, including those of the sort and scan primitives). */
int64_t vr_launch_count(void);

/* ---------------------------------------------------------------- autotuning
 * (no counterpart in the paper: the launch shapes of this library's batched form)
 * The f_l kernel runs one launch per halo-size bin (halos of more than 65536 members,
 * 4097-65536, N_se+1-4096), each with its own shape (candidates computed side by side,
 * register cap, warps per block); the 6D linker has one shape (32-candidate tiles per
 * block). A shape changes how the same work is laid out on the GPU, never the arithmetic
 * or its order: every shape gives bit-identical results.
 * vr_autotune(ctx, 1): from the next call on, the first launch of each bin (and of the
 * linker) with work runs every candidate shape on the caller's data, timed with CUDA
 * events on `stream`, and keeps the fastest for later calls (that call takes several
 * times longer and synchronises its stream). vr_autotune(ctx, 0) returns to the default
 * shapes. Errors: VR_ERR_INVALID_ARG for enable not 0 or 1. */
vr_status vr_autotune(vr_ctx *ctx, int enable);

/* Every later launch uses f_l shape `velden_shape` and linker shape `link_shape` (indices
 * into the candidate lists of vr_tuning_report; -1 = not forced). For testing that the
 * shapes agree. Errors: VR_ERR_INVALID_ARG for an index out of range. */
vr_status vr_tuning_force(vr_ctx *ctx, int velden_shape, int link_shape);

/* Writes a JSON object with the candidate shapes, the shape in use per bin and the
 * measured milliseconds (-1 where not measured) into buf (len bytes, NUL-terminated).
 * Errors: VR_ERR_INVALID_ARG if buf is too small. */
vr_status vr_tuning_report(const vr_ctx *ctx, char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */
