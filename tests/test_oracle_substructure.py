"""Pins for the oracle's phase-space outlier search (Sec. 2.2).

Each part is tied to something other than the oracle itself: hand-placed points with
analytic sums, closed-form Gaussian densities, numpy/scipy library routes, planted
distributions and the paper's printed defaults (tests/golden/table1_defaults.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "table1_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def test_defaults_match_table1():
    g = _golden()
    p = oracle.Params.default()
    assert p.nse == g["nse"] and p.nv == g["nv"] and p.nmin == g["nmin"]
    assert p.f_cell == g["f_cell"] and p.ell_th == g["ell_th"] and p.v_ratio == g["v_ratio"]
    assert abs(p.theta_op - g["theta_op_pi"] * math.pi) < 1e-15
    assert abs(math.degrees(p.theta_op) - 18.0) < 1e-12  # Sec. 2.2 states 18 degrees


# ----------------------------------------------------------------- k-NN

def test_knn_matches_full_sort():
    rng = np.random.default_rng(5)
    nh = 700
    upos = rng.integers(-3000, 3000, size=(nh, 3)).astype(np.int64)
    upos[10] = upos[11]  # a coincident pair: tie broken by index
    members = np.sort(rng.choice(100000, nh, replace=False)).astype(np.int32)
    for k in (0, 10, 11, 350, nh - 1):
        got = oracle.knn_one(upos, members, k, 256)
        d2 = ((upos - upos[k]) ** 2).sum(1)
        order = np.lexsort((members, d2))[:256]
        assert np.array_equal(got, members[order])
        assert got[0] == members[k] or d2[np.searchsorted(members, got[0])] == 0


def test_knn_small_halo_is_whole_halo():
    rng = np.random.default_rng(6)
    upos = rng.integers(0, 100, size=(40, 3)).astype(np.int64)
    members = np.arange(40, dtype=np.int32) * 3
    got = oracle.knn_one(upos, members, 7, 256)
    assert sorted(got.tolist()) == members.tolist()


# ------------------------------------------------------------ f_l (Epanechnikov)

def _halo_with_velocities(dv):
    """Members at distinct positions (all within N_se), velocities v_k + dv[j]."""
    nh = len(dv)
    upos = np.stack([np.arange(nh), np.zeros(nh), np.zeros(nh)], 1).astype(np.int64)
    vel = np.asarray(dv, np.float32) + np.float32(250.0)
    members = np.arange(nh, dtype=np.int32)
    return upos, vel, members


def test_epanechnikov_hand_placed():
    # query 0 at rest; others at speeds 0.5, 0.5, 2, 2, 3, 3, 3 along axes.
    dv = [[0, 0, 0], [0.5, 0, 0], [0, -0.5, 0], [2, 0, 0], [0, 0, -2], [3, 0, 0], [0, 3, 0],
          [0, 0, 3]]
    upos, vel, members = _halo_with_velocities(dv)
    # N_se = 8 (whole halo), N_v = 4: h = 4th smallest |dv| (self included) = 2;
    # terms: self 1, two at r = 0.5 give 1 - 0.25/4 each, r = h gives 0.
    h = 2.0
    norm = 15.0 / (8.0 * math.pi * h ** 3)
    expect = norm * (1.0 + 2.0 * (1.0 - 0.25 / 4.0)) / 8.0
    got = oracle.velden_one(upos, vel, members, 0, nse=8, nv=4)
    assert abs(got - expect) < 1e-14 * expect
    # N_se = 4 drops the two farthest members in position (indices 6, 7 at x = 6, 7)
    got4 = oracle.velden_one(upos, vel, members, 0, nse=4, nv=4)
    # set {0,1,2,3}: |dv| = 0, .5, .5, 2 -> h = 2, same three terms, normalised by 4
    assert abs(got4 - norm * (1.0 + 2.0 * (1.0 - 0.25 / 4.0)) / 4.0) < 1e-14 * expect * 2
    # N_v = 2: h = 0.5 -> only self contributes
    h = 0.5
    got2 = oracle.velden_one(upos, vel, members, 0, nse=8, nv=2)
    assert abs(got2 - 15.0 / (8.0 * math.pi * h ** 3) / 8.0) < 1e-12 * got2


def test_velden_halo_equals_one_by_one():
    rng = np.random.default_rng(9)
    nh = 400
    upos = rng.integers(0, 20000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, 50, size=(nh, 3)).astype(np.float32)
    members = np.arange(nh, dtype=np.int32)
    allf = oracle.velden_halo(upos, vel, members, 64, 16)
    for k in (0, 17, 399):
        assert allf[k] == oracle.velden_one(upos, vel, members, k, 64, 16)


def test_velden_gaussian_closed_form():
    """Positions independent of velocities: the N_se set is a random sample of the
    isotropic Gaussian, so f_l estimates (2 pi s^2)^(-3/2) exp(-v^2 / 2 s^2) (Eq. fvbg with
    Sigma = s^2 I). The 1/N_se normalisation gives a mean log ratio near zero; the 1/N_v
    reading would sit at ln(N_se/N_v) = 2.08."""
    rng = np.random.default_rng(12)
    nh, s = 20000, 80.0
    upos = rng.integers(0, 200000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, s, size=(nh, 3)).astype(np.float32)
    members = np.arange(nh, dtype=np.int32)
    ks = rng.choice(nh, 600, replace=False)
    r = []
    for k in ks:
        f = oracle.velden_one(upos, vel, members, int(k))
        v2 = float((vel[k].astype(np.float64) ** 2).sum())
        ftrue = (2 * math.pi * s * s) ** -1.5 * math.exp(-v2 / (2 * s * s))
        r.append(math.log(f / ftrue))
    r = np.array(r)
    assert abs(r.mean()) < 0.25, r.mean()
    assert 0.1 < r.std() < 1.0


# ------------------------------------------------------ background Gaussian model

def test_ln_fbg_isotropic_closed_form():
    s2 = 37.0 ** 2
    v = np.array([10.0, -20.0, 5.0])
    vb = np.array([1.0, 2.0, 3.0])
    got = oracle.ln_fbg(v, vb, [s2, s2, s2, 0, 0, 0])
    d2 = ((v - vb) ** 2).sum()
    expect = -d2 / (2 * s2) - 1.5 * math.log(2 * math.pi * s2)
    assert abs(got - expect) < 1e-13 * abs(expect)


def test_ln_fbg_rotated_anisotropic():
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    S = q @ np.diag([900.0, 2500.0, 100.0]) @ q.T
    v = np.array([33.0, -12.0, 40.0])
    vb = np.array([-5.0, 4.0, 8.0])
    six = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
    got = oracle.ln_fbg(v, vb, six)
    d = v - vb
    expect = -0.5 * d @ np.linalg.inv(S) @ d - 1.5 * math.log(2 * math.pi) - 0.5 * math.log(
        np.linalg.det(S))
    assert abs(got - expect) < 1e-12 * abs(expect)
    # not positive definite -> NaN
    assert math.isnan(oracle.ln_fbg(v, vb, [1.0, 1.0, 1.0, 2.0, 0.0, 0.0]))


def test_ncell_rule():
    # Sec. 2.2: N_cell = f_cell N_H, raised below 100 up to N_H/8
    assert oracle.ncell(1000000) == 10000
    assert oracle.ncell(50000) == 500
    assert oracle.ncell(1000) == 100
    assert oracle.ncell(799) == 99
    assert oracle.ncell(160) == 20


def _blob(nh, seed, spread=5000, sv=60.0):
    rng = np.random.default_rng(seed)
    upos = rng.integers(0, spread, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, sv, size=(nh, 3)).astype(np.float32)
    return upos, vel, np.arange(nh, dtype=np.int32)


def test_cells_balanced_median_splits_and_moments():
    nh = 1600
    upos, vel, members = _blob(nh, 21, spread=1 << 20)  # distinct coordinates (a.s.)
    f = np.ones(nh)
    R, leaf, cs = oracle.background_halo(upos, vel, members, f)
    # N_cell = 100: 1600 -> 800 -> 400 -> 200 -> 100, median splits
    assert cs.shape[0] == 16
    assert np.all(np.bincount(leaf) == 100)
    # moments (Eqs. meanpos, meanvel, meandispvel), recomputed by numpy per leaf
    for l in range(16):
        sel = leaf == l
        assert cs[l, 0] == sel.sum()
        assert np.allclose(cs[l, 1:4], upos[sel].mean(0), rtol=1e-14)
        v = vel[sel].astype(np.float64)
        assert np.allclose(cs[l, 4:7], v.mean(0), rtol=1e-12, atol=1e-12)
        C = np.cov(v.T, bias=True)
        assert np.allclose(cs[l, 7:13], [C[0, 0], C[1, 1], C[2, 2], C[0, 1], C[0, 2], C[1, 2]],
                           rtol=1e-10)
    # each leaf is a box: leaves are separable, no member of another leaf inside a
    # leaf's bounding box
    for l in range(16):
        sel = leaf == l
        lo, hi = upos[sel].min(0), upos[sel].max(0)
        inside = np.all((upos >= lo) & (upos <= hi), 1)
        assert np.all(leaf[inside] == l)


def test_entropy_axis_choice():
    """Root split into 2 cells (f_cell = 0.5, N_cell = 100): x uniform (S near 1), y two tight clumps (S low), z one
    value (zero extent, never split). argmax S splits x; argmin S splits y."""
    rng = np.random.default_rng(4)
    nh = 200
    x = rng.permutation(np.arange(nh) * 100)
    y = np.where(np.arange(nh) % 2 == 0, 0, 50000) + rng.integers(0, 10, nh)
    z = np.full(nh, 7)
    upos = np.stack([x, y, z], 1).astype(np.int64)
    vel = rng.normal(0, 10, size=(nh, 3)).astype(np.float32)
    members = np.arange(nh, dtype=np.int32)
    for rule, axis in ((0, 0), (1, 1)):
        R, leaf, cs = oracle.background_halo(upos, vel, members, np.ones(nh), f_cell=0.5,
                                             split_rule=rule)
        assert cs.shape[0] == 2
        a0 = upos[leaf == 0, axis]
        a1 = upos[leaf == 1, axis]
        assert a0.max() < a1.min()
        assert len(a0) == 100  # median split in (coordinate, index) order


def test_interpolation_two_cells():
    """Two leaves split along one axis: every member interpolates over its own cell and
    the cell across the split face (Eq. cellinterp), with w = 1/|x - xbar|."""
    rng = np.random.default_rng(8)
    nh = 200
    upos = rng.integers(0, 100000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, 40, size=(nh, 3)).astype(np.float32)
    vel[upos[:, 0] > 50000] += np.float32(30.0)
    members = np.arange(nh, dtype=np.int32)
    f = np.exp(rng.normal(-14, 0.3, nh))
    R, leaf, cs = oracle.background_halo(upos, vel, members, f, f_cell=0.5)
    assert cs.shape[0] == 2
    for k in range(0, nh, 7):
        x = upos[k].astype(np.float64)
        w = np.array([1 / np.linalg.norm(x - cs[c, 1:4]) for c in (0, 1)])
        vb = (w[:, None] * cs[:, 4:7]).sum(0) / w.sum()
        s6 = (w[:, None] * cs[:, 7:13]).sum(0) / w.sum()
        S = np.array([[s6[0], s6[3], s6[4]], [s6[3], s6[1], s6[5]], [s6[4], s6[5], s6[2]]])
        d = vel[k].astype(np.float64) - vb
        lnfbg = -0.5 * d @ np.linalg.solve(S, d) - 1.5 * math.log(2 * math.pi) - 0.5 * math.log(
            np.linalg.det(S))
        assert abs(R[k] - (math.log(f[k]) - lnfbg)) < 1e-10 * max(1, abs(R[k]))


def _leaf_of_point(boxes, p):
    """Index of the one leaf whose half-open region holds p, by a scan over every leaf."""
    inside = np.all((boxes[:, :3] <= p) & (p < boxes[:, 3:]), axis=1)
    hit = np.flatnonzero(inside)
    assert len(hit) == 1, (p, hit)
    return int(hit[0])


def test_interpolation_multilevel_tree_brute_force():
    """Face neighbours in a deep tree (Sec. 2.2, Eq. cellinterp), found without the tree:
    for every member, the leaf holding its position moved to lo - 1 / hi of its own leaf
    along each axis is found by scanning every leaf's half-open region; points outside
    the root region are skipped and a leaf reached through two faces is counted once.
    The moments are recomputed by numpy from the leaf membership, the interpolation and
    ln f_bg (Eq. fvbg) by numpy's solve and determinant, and R must match to 1e-12."""
    rng = np.random.default_rng(77)
    nh = 12800  # N_cell = 128: seven levels of median splits, 128 leaves
    # distinct coordinates on every axis, a dense clump plus a wider halo, anisotropic
    core = rng.normal(0, [3000, 9000, 5000], size=(nh // 2, 3))
    outer = rng.normal(0, [30000, 12000, 20000], size=(nh - nh // 2, 3))
    p = np.concatenate([core, outer]) + 200000
    upos = np.empty((nh, 3), np.int64)
    for a in range(3):  # make each axis's coordinates distinct, keeping their order
        order = np.argsort(p[:, a], kind="stable")
        x = np.round(p[order, a]).astype(np.int64)
        x = x + np.arange(nh)  # strictly increasing in sorted order
        upos[order, a] = x
    vel = rng.normal(0, 60, size=(nh, 3)).astype(np.float32)
    vel[upos[:, 1] > np.median(upos[:, 1])] += np.float32([40, -10, 5])
    members = np.arange(nh, dtype=np.int32)
    f = np.exp(rng.normal(-14, 0.4, nh))
    R, leaf, cs, boxes = oracle.background_halo(upos, vel, members, f, boxes=True)
    nl = cs.shape[0]
    assert nl == 128 and np.all(np.bincount(leaf, minlength=nl) == 100)

    # the leaf regions tile the root region [min, max + 1) exactly and hold their members
    root_lo, root_hi = upos.min(0), upos.max(0) + 1
    assert np.all(boxes[:, :3] >= root_lo) and np.all(boxes[:, 3:] <= root_hi)
    vol = np.prod((boxes[:, 3:] - boxes[:, :3]).astype(np.float64), axis=1)
    assert vol.sum() == np.prod((root_hi - root_lo).astype(np.float64))
    for i in range(nl):
        for j in range(i + 1, nl):
            overlap = np.all(np.maximum(boxes[i, :3], boxes[j, :3])
                             < np.minimum(boxes[i, 3:], boxes[j, 3:]))
            assert not overlap
    for m in range(nh):
        assert _leaf_of_point(boxes, upos[m]) == leaf[m]

    # moments per leaf (Eqs. meanpos, meanvel, meandispvel) by numpy
    mom = np.zeros((nl, 13))
    for l in range(nl):
        sel = leaf == l
        v = vel[sel].astype(np.float64)
        C = np.cov(v.T, bias=True)
        mom[l] = [sel.sum(), *upos[sel].mean(0), *v.mean(0),
                  C[0, 0], C[1, 1], C[2, 2], C[0, 1], C[0, 2], C[1, 2]]
    assert np.allclose(cs, mom, rtol=1e-11, atol=1e-9)

    # a split made at the root: a plane that no leaf region straddles
    root_planes = [(a, x) for a in range(3) for x in np.unique(boxes[:, a])
                   if x > root_lo[a] and np.all((boxes[:, 3 + a] <= x) | (boxes[:, a] >= x))]
    assert root_planes
    n_far, n_cross_root, n_dup, nneigh = 0, 0, 0, []
    for m in range(nh):
        own = leaf[m]
        cells = [own]
        for a in range(3):
            for side in (0, 1):
                q = upos[m].copy()
                q[a] = boxes[own, a] - 1 if side == 0 else boxes[own, 3 + a]
                if np.any(q < root_lo) or np.any(q >= root_hi):
                    continue
                c = _leaf_of_point(boxes, q)
                n_dup += c in cells
                if c not in cells:
                    cells.append(c)
                    other = [b for b in range(3) if b != a]
                    # not a mirror image of the own leaf: its region differs across the face,
                    # so the split between them was made two or more levels up
                    if np.any(boxes[c, other] != boxes[own, other]) or np.any(
                            boxes[c, [3 + b for b in other]] != boxes[own, [3 + b for b in other]]):
                        n_far += 1
                    for (ra, rx) in root_planes:
                        if (boxes[own, ra] >= rx) != (boxes[c, ra] >= rx):
                            n_cross_root += 1
        nneigh.append(len(cells))
        X = upos[m].astype(np.float64)
        r = np.array([np.linalg.norm(X - mom[c, 1:4]) for c in cells])
        if np.any(r == 0.0):
            use = [cells[int(np.flatnonzero(r == 0.0)[0])]]
            w = np.ones(1)
        else:
            use, w = cells, 1.0 / r
        w = w / w.sum()
        vb = (w[:, None] * mom[use, 4:7]).sum(0)
        s6 = (w[:, None] * mom[use, 7:13]).sum(0)
        S = np.array([[s6[0], s6[3], s6[4]], [s6[3], s6[1], s6[5]], [s6[4], s6[5], s6[2]]])
        d = vel[m].astype(np.float64) - vb
        lnfbg = (-0.5 * d @ np.linalg.solve(S, d) - 1.5 * math.log(2 * math.pi)
                 - 0.5 * math.log(np.linalg.det(S)))
        expect = math.log(f[m]) - lnfbg
        assert abs(R[m] - expect) <= 1e-12 * max(1.0, abs(expect)), (m, R[m], expect)
    assert n_far > 1000 and n_cross_root > 100
    # leaves are disjoint boxes, so distinct faces of one leaf never reach the same
    # neighbour; some members have neighbours across four faces
    assert n_dup == 0 and max(nneigh) >= 5 and np.mean(nneigh) > 3.5


def test_R_near_zero_on_smooth_gaussian_halo():
    """A halo-free Gaussian velocity field: R = ln(f_l/f_bg) should scatter around 0."""
    nh = 12000
    rng = np.random.default_rng(30)
    # uniform ball of positions, isotropic Gaussian velocities independent of position
    p = rng.normal(size=(nh, 3))
    p = p / np.linalg.norm(p, axis=1, keepdims=True) * rng.random((nh, 1)) ** (1 / 3) * 40000
    upos = np.round(p).astype(np.int64)
    vel = rng.normal(0, 70.0, size=(nh, 3)).astype(np.float32)
    members = np.arange(nh, dtype=np.int32)
    f = oracle.velden_halo(upos, vel, members)
    R, leaf, cs = oracle.background_halo(upos, vel, members, f)
    assert abs(np.mean(R)) < 0.25, np.mean(R)
    fit = oracle.ell_fit(R)
    ell = (R - fit[0]) / fit[1]
    # outlier fraction of a smooth halo: about the Gaussian tail above 2.5 (Eq. ell)
    frac = np.mean(ell >= 2.5)
    assert frac < 0.10


# ---------------------------------------------------------- skew-Gaussian fit

def test_skew_gaussian_fit_recovers_planted():
    rng = np.random.default_rng(1)
    n, mu, sg, s = 200000, 0.3, 0.5, 1.6
    # left half-normal of width s*sg with weight s/(1+s), right of width sg
    left = rng.random(n) < s / (1 + s)
    z = np.abs(rng.normal(size=n))
    R = np.where(left, mu - z * s * sg, mu + z * sg)
    fit = oracle.ell_fit(R)
    assert abs(fit[0] - mu) < 0.02
    assert abs(fit[1] - sg) / sg < 0.03
    assert abs(fit[2] - s) / s < 0.05
    assert fit[6] == 200  # nbins clamp


def _f_sg(x, A, mu, sg, s):
    """Eq. skewgaus: width s*sigma left of the mode, sigma right of it."""
    w = np.where(x < mu, s * sg, sg)
    return A * np.exp(-((x - mu) ** 2) / (2 * w * w))


@pytest.mark.parametrize("A,mu,sg,s", [(500.0, 0.3, 0.5, 1.6), (4321.0, -1.2, 0.8, 0.7),
                                       (37.5, 2.0, 0.25, 1.0)])
def test_sg_fit_exact_counts(A, mu, sg, s):
    """Noise-free counts A f_SG at the bin centres x_b = lo + (b + 1/2) width of the
    documented binning: the fit must return (Rbar, sigma_R, s, A) to 1e-8 relative. A bin
    centre taken at the edge, or any offset in it, moves Rbar by up to half a bin."""
    nb = 60
    lo, width = mu - 6 * sg * max(s, 1.0), 12 * sg * max(s, 1.0) / nb
    x = lo + (np.arange(nb) + 0.5) * width
    counts = _f_sg(x, A, mu, sg, s)
    fit = oracle.sg_fit(counts, lo, width, sigma0=1.3 * sg)
    for got, want in zip(fit, (mu, sg, s, A)):
        assert abs(got - want) <= 1e-8 * max(1.0, abs(want)), (fit, (mu, sg, s, A))


def test_ell_bins_documented_binning():
    """The binning step of the fit, recomputed by numpy: finite values only, median,
    MAD' = 1.4826 median |R - median|, clamp(ceil(sqrt N), 10, 200) bins on
    median -/+ 6 MAD', bin = floor((R - lo) / width)."""
    rng = np.random.default_rng(12)
    for n in (7, 99, 2500, 60000):
        R = np.concatenate([rng.standard_t(5, n) * 0.7 + 0.2, [np.nan, np.inf, -np.inf]])
        counts, meta = oracle.ell_bins(R)
        a = R[np.isfinite(R)]
        med = np.median(a)
        mad = 1.4826 * np.median(np.abs(a - med))
        nb = int(min(max(math.ceil(math.sqrt(len(a))), 10), 200))
        lo, width = med - 6 * mad, 12 * mad / nb
        assert meta[0] == med and meta[1] == mad and meta[4] == nb
        assert meta[2] == lo and meta[3] == width
        f = np.floor((a - lo) / width)
        f = f[(f >= 0) & (f < nb)].astype(np.int64)
        assert np.array_equal(counts, np.bincount(f, minlength=nb).astype(np.float64))
        # the fit is this binning followed by the count fit started at sigma = MAD'
        fit = oracle.ell_fit(R)
        assert np.array_equal(fit[:4], oracle.sg_fit(counts, lo, width, mad))
        assert fit[4] == lo and fit[5] == width and fit[6] == nb and fit[7] == mad


def test_fit_degenerate():
    fit = oracle.ell_fit(np.full(50, 1.25))
    assert fit[0] == 1.25 and math.isnan(fit[1])


def test_ell_bar_closed_form():
    # Eq. ellsig: tail mean of a unit Gaussian above ell_th
    e = 2.5
    expect = math.sqrt(2 / math.pi) * math.exp(-e * e / 2) / (1 - math.erf(e / math.sqrt(2)))
    assert abs(oracle.ell_bar(e) - expect) < 1e-13 * expect
    # cross-check by quadrature of the two integrals
    from scipy.integrate import quad

    num = quad(lambda x: x * math.exp(-x * x / 2), e, np.inf)[0]
    den = quad(lambda x: math.exp(-x * x / 2), e, np.inf)[0]
    assert abs(oracle.ell_bar(e) - num / den) < 1e-9


# ------------------------------------------------------------ 6D linking

def _pair(dx, v1, v2):
    upos = np.array([[0, 0, 0], [dx, 0, 0]], np.int64)
    vel = np.array([v1, v2], np.float32)
    return upos, vel, np.array([0, 1], np.int32)


def test_link6_each_criterion_boundary():
    prm = np.array([100.0 ** 2, 1e30, 0, 0, 0])  # lx = 100, velocity term negligible
    cand = np.ones(2, np.uint8)
    kw = dict(nmin=1)
    # Eq. linkingcriteria b: strict
    assert list(oracle.fof6d_halo(*_pair(99, [100, 0, 0], [100, 0, 0]), cand, prm, **kw)) == [0, 0]
    assert list(oracle.fof6d_halo(*_pair(100, [100, 0, 0], [100, 0, 0]), cand, prm, **kw)) == [0, 1]
    # Eq. linkingcriteria c: speed ratio 2 inclusive
    assert list(oracle.fof6d_halo(*_pair(1, [100, 0, 0], [200, 0, 0]), cand, prm, **kw)) == [0, 0]
    assert list(oracle.fof6d_halo(*_pair(1, [100, 0, 0], [201, 0, 0]), cand, prm, **kw)) == [0, 1]
    # Eq. linkingcriteria d: opening angle 18 degrees
    for ang, linked in ((17.9, True), (18.1, False)):
        a = math.radians(ang)
        v2 = [100 * math.cos(a), 100 * math.sin(a), 0]
        got = oracle.fof6d_halo(*_pair(1, [100, 0, 0], v2), cand, prm, **kw)
        assert (got[1] == 0) == linked, ang
    # the frame: u = v - v_frame; opposite in the frame -> not linked
    prm2 = prm.copy()
    prm2[2:] = [100, 0, 0]
    assert list(oracle.fof6d_halo(*_pair(1, [110, 0, 0], [90, 0, 0]), cand, prm2, **kw)) == [0, 1]
    # Eq. fof6d velocity term: dx^2/lx^2 + dv^2/lv^2 < 1
    prm3 = np.array([100.0 ** 2, 10.0 ** 2, 0, 0, 0])
    # dx = 60 (0.36), dv = 8 (0.64): sum exactly 1 -> not linked; dv = 7.9 linked
    assert list(oracle.fof6d_halo(*_pair(60, [100, 0, 0], [108, 0, 0]), cand, prm3, **kw)) == [0, 1]
    assert list(oracle.fof6d_halo(*_pair(60, [100, 0, 0], [107.9, 0, 0]), cand, prm3,
                                  **kw)) == [0, 0]
    assert list(oracle.fof6d_halo(*_pair(60, [100, 0, 0], [108, 0, 0]), cand, prm3, use_lv=0,
                                  **kw)) == [0, 0]
    # non-candidates never link
    assert list(oracle.fof6d_halo(*_pair(1, [100, 0, 0], [100, 0, 0]), np.array([1, 0], np.uint8),
                                  prm, **kw)) == [0, -1]


def _brute_6d(upos, vel, members, cand, prm, vr=2.0, th=0.1 * math.pi, nmin=20):
    """Independent numpy route: pairwise predicate matrix + scipy components."""
    from scipy.sparse.csgraph import connected_components

    idx = np.flatnonzero(cand)
    x = upos[idx].astype(np.int64)
    v = vel[idx].astype(np.float64)
    dx2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(2)
    dv = v[:, None, :] - v[None, :, :]
    dv2 = (dv[..., 0] * dv[..., 0] + dv[..., 1] * dv[..., 1]) + dv[..., 2] * dv[..., 2]
    q = dx2.astype(np.float64) / prm[0] + dv2 / prm[1]
    u = v - prm[2:5]
    s = (u[:, 0] * u[:, 0] + u[:, 1] * u[:, 1]) + u[:, 2] * u[:, 2]
    dot = u @ u.T
    c2 = math.cos(th) ** 2
    ok = (q < 1) & (s[:, None] > 0) & (s[None, :] > 0)
    ok &= (s[:, None] <= vr * vr * s[None, :]) & (s[None, :] <= vr * vr * s[:, None])
    ok &= (dot >= 0) & (dot * dot >= (c2 * s[:, None]) * s[None, :])
    _, comp = connected_components(ok, directed=False)
    out = np.full(len(members), -1, np.int32)
    for c in np.unique(comp):
        sel = idx[comp == c]
        if len(sel) >= nmin:
            out[sel] = members[sel].min()
    return out


def test_fof6d_matches_independent_route():
    rng = np.random.default_rng(44)
    nh = 3000
    # two cold streams plus a hot background, in one halo
    upos = rng.integers(0, 60000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, 100, size=(nh, 3)).astype(np.float32)
    s1 = slice(0, 300)
    upos[s1] = rng.normal(20000, 1500, size=(300, 3)).astype(np.int64)
    vel[s1] = (np.array([150, 40, 0]) + rng.normal(0, 8, size=(300, 3))).astype(np.float32)
    members = np.sort(rng.choice(10 ** 6, nh, replace=False)).astype(np.int32)
    cand = (rng.random(nh) < 0.15).astype(np.uint8)
    cand[s1] = 1
    prm = np.array([1500.0 ** 2, 60.0 ** 2, 5.0, -3.0, 1.0])
    vel_all = np.zeros((10 ** 6, 3), np.float32)  # velocities are indexed by particle
    vel_all[members] = vel
    got = oracle.fof6d_halo(upos, vel_all, members, cand, prm)
    exp = _brute_6d(upos, vel, members, cand, prm)
    assert np.array_equal(got, exp)
    assert (got >= 0).sum() >= 200


def test_halo_frame_sigma_host():
    """sigma_host = |Sigma|^(1/6) (Table A2's sigma_v) with Sigma about the mean / N_H."""
    rng = np.random.default_rng(2)
    vel = (rng.normal(0, 1, size=(5000, 3)) * [30.0, 60.0, 90.0] + [10, -20, 5]).astype(np.float32)
    members = np.arange(5000, dtype=np.int32)
    fr = oracle.halo_frame(vel, members)
    v = vel.astype(np.float64)
    assert np.allclose(fr[:3], v.mean(0), rtol=1e-12)
    C = np.cov(v.T, bias=True)
    assert abs(fr[3] - np.linalg.det(C) ** (1 / 6)) < 1e-10 * fr[3]
    assert abs(fr[3] - (30 * 60 * 90) ** (1 / 3)) / fr[3] < 0.03


def test_pipeline_recovers_planted_subhalos():
    """Sanity (not parity): the 32^3 clustered box plants two cold Plummer subhalos per
    host; most substructure groups found should be dominated by one planted subhalo."""
    import synth

    box = synth.named("c32")
    out = oracle.pipeline(box.pos, box.vel, box.link_d2, box.lx_sub)
    lab6 = out["label6"]
    groups = np.unique(lab6[lab6 >= 0])
    assert len(groups) >= 6
    pure = 0
    for g in groups:
        sid = box.sub_id[lab6 == g]
        vals, cnt = np.unique(sid, return_counts=True)
        if vals[np.argmax(cnt)] >= 0 and cnt.max() >= 0.8 * len(sid):
            pure += 1
    assert pure >= 0.7 * len(groups)
    # per-particle outputs are defined exactly on halo members
    inhalo = np.isfinite(out["f_l"])
    assert inhalo.sum() == out["halos"][:, 1].sum()
