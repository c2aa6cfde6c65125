"""Pins for the oracle's core cleaning and core growth (Sec. 2.3, "Core Growth & Mass
Reconstruction" and "Cleaning the Catalogue"; Eqs. coremeanphase, coredispphase,
coredist, coresig; Table 1 beta_C = 1; Table A1 core growth mode 2).

Tied to: distances worked out by hand on symmetric seed sets; numpy's own inverse and
covariance routines on random seeds; the paper's Gaussian-mixture comparison of tensor
and scalar distances, rebuilt on synthetic draws; an independent brute-force route
(6D links by a union-find written here, numpy moments and linear solves) on small halos;
exact power-of-two rescalings, under which every decision is unchanged.
"""
import numpy as np
import pytest

import oracle


# ------------------------------------------------------------ assignment step

def _cross(center, sig):
    """12 seed points at center +- sig_a e_a: mean = center, S = diag(sig^2 / 6)."""
    pts = []
    for a in range(6):
        for s in (1.0, -1.0):
            p = np.array(center, np.float64)
            p[a] += s * sig[a]
            pts.append(p)
    return np.array(pts)


def test_distance_worked_by_hand():
    """Core 0 at the origin with S0 = diag(1/6, ..., 1/6) (sig = 1); core 1 at x = 10 with
    S1 = diag(24, 1/6, ...) (sig_x = 12). The point (t, 0, ..., 0) has D0^2 = 6 t^2 and
    D1^2 = (t - 10)^2 / 24: equal at 6 t^2 = (t - 10)^2 / 24, i.e. 12 t = -(t - 10) for
    t > 0: t = 10/13. Points just below go to core 0, just above to core 1. In the scalar
    form (mode 0), s_x^2(core 1) = (24 + 2/6) / 3 and s_x^2(core 0) = 1/6."""
    s0 = _cross(np.zeros(6), np.ones(6))
    s1 = _cross([10, 0, 0, 0, 0, 0], [12, 1, 1, 1, 1, 1])
    t = np.array([10 / 13 - 1e-6, 10 / 13 + 1e-6, 0.0, 9.0])
    q = np.zeros((len(t), 6))
    q[:, 0] = t
    X = np.vstack([s0, s1, q])
    init = np.array([0] * 12 + [1] * 12 + [-1] * len(t), np.int32)
    out, npd = oracle.core_assign(X, init, 2, mode=1)
    assert npd == 2
    assert list(out[24:]) == [0, 1, 0, 1]
    # scalar form: D0^2 = t^2 / (1/6), D1^2 = (t - 10)^2 / ((24 + 1/3) / 3)
    sx1 = (24 + 2 / 6) / 3
    t0 = 10 / (1 + np.sqrt(6 * sx1))  # positive root of 6 t^2 = (10 - t)^2 / sx1
    q[:, 0] = [t0 - 1e-6, t0 + 1e-6, 0.0, 9.0]
    X = np.vstack([s0, s1, q])
    out, _ = oracle.core_assign(X, init, 2, mode=0)
    assert list(out[24:]) == [0, 1, 0, 1]


def test_distance_matches_numpy_inverse():
    """Random anisotropic seeds: the assignment is argmin of (x - mean) S^-1 (x - mean)
    with mean and S from numpy (np.cov, bias=True) and S^-1 from np.linalg.inv."""
    rng = np.random.default_rng(11)
    k, ns = 4, 60
    seeds, init = [], []
    for c in range(k):
        A = rng.normal(size=(6, 6))
        seeds.append(rng.normal(size=(ns, 6)) @ A + rng.normal(0, 3, 6))
        init += [c] * ns
    q = rng.normal(0, 4, size=(3000, 6))
    X = np.vstack(seeds + [q])
    init = np.array(init + [-1] * len(q), np.int32)
    for mode in (0, 1):
        out, npd = oracle.core_assign(X, init, k, mode=mode)
        assert npd == k
        D = np.empty((len(q), k))
        for c in range(k):
            m = seeds[c].mean(0)
            S = np.cov(seeds[c].T, bias=True)
            d = q - m
            if mode == 1:
                D[:, c] = np.einsum("ij,jk,ik->i", d, np.linalg.inv(S), d)
            else:
                D[:, c] = ((d[:, :3] ** 2).sum(1) / (np.trace(S[:3, :3]) / 3)
                           + (d[:, 3:] ** 2).sum(1) / (np.trace(S[3:, 3:]) / 3))
        srt = np.sort(D, 1)
        clear = (srt[:, 1] - srt[:, 0]) > 1e-9 * srt[:, 1]
        assert clear.mean() > 0.99
        assert np.array_equal(out[len(init) - len(q):][clear], D.argmin(1)[clear]), mode


def test_degenerate_tensor_attracts_nothing():
    """A core whose seeds lie in a 5D plane has a singular tensor: no point goes to it."""
    rng = np.random.default_rng(2)
    a = rng.normal(size=(50, 6))
    b = rng.normal(size=(50, 6)) + 0.1
    b[:, 5] = 0.0
    q = rng.normal(size=(200, 6))
    X = np.vstack([a, b, q])
    init = np.array([0] * 50 + [1] * 50 + [-1] * 200, np.int32)
    out, npd = oracle.core_assign(X, init, 2, mode=1)
    assert npd == 1 and (out[100:] == 0).all()


def _mixture(rng, n_each, minor):
    """Two 6D Gaussians (the comparison of Sec. 2.3): population 0 spherical (unit
    dispersion), population 1 with principal axes (1, 1, 1, 1, 1, minor) in a random
    orientation; means 2 apart (2 unit dispersions)."""
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
    ax = np.array([1, 1, 1, 1, 1, minor])
    d = rng.normal(size=6)
    d *= 2.0 / np.linalg.norm(d)
    p0 = rng.normal(size=(n_each, 6))
    p1 = (rng.normal(size=(n_each, 6)) * ax) @ Q.T + d
    return p0, p1


def _purity_recovery(out, truth):
    pur, rec = [], []
    for c in (0, 1):
        got = out == c
        pur.append(((truth == c) & got).sum() / max(got.sum(), 1))
        rec.append(((truth == c) & got).sum() / (truth == c).sum())
    return np.array(pur), np.array(rec)


def _paper_mixture():
    """The paper's printed figures (tests/golden/core_growth_mixture.txt)."""
    import os

    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "core_growth_mixture.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                q, pop, sc, te = line.split()
                out[(q, pop)] = (float(sc), float(te))
    return out


def test_defaults_match_the_paper():
    import os

    g = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "table1_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                g[k] = float(v)
    d = oracle.CORE_DEFAULTS
    assert (d["ax"], d["av"], d["n_loop"], d["f_c"], d["an"]) == (
        g["alpha_xC"], g["alpha_vC"], g["n_loopC"], g["f_C"], g["alpha_NC"])
    assert (oracle.CORE_GROW_DEFAULTS["beta_c"], oracle.CORE_GROW_DEFAULTS["mode"]) == (
        g["beta_C"], g["core_growth_mode"])


def test_gaussian_mixture_tensor_vs_scalar():
    """Sec. 2.3's comparison, rebuilt: seeds of 100 particles per population set the
    dispersions, every other particle is assigned in one step. The paper reports, for a
    spherical and an aspherical population (minor axis ratio 0.03) two tensor-normalised
    dispersions apart, purities 0.76 / 0.92 (scalar) and 0.79 / 0.93 (tensor) and
    recoveries 0.94 / 0.70 and 0.95 / 0.76. It does not give the other axes, the
    orientation or the draw, and in our draws (axes 1, 1, 1, 1, 1, 0.03; random
    orientation) the spherical population's purity and the aspherical one's recovery
    move either way by a few per cent with the seed. What holds on every draw is pinned:
    the tensor distance raises the aspherical population's purity (~0.88 -> ~0.99) and
    the spherical population's recovery (~0.88 -> ~0.99), because it stops assigning the
    spherical population's particles off the thin axis to the aspherical core."""
    paper = _paper_mixture()
    # the two figures pinned here move up from scalar to tensor in the paper too
    assert paper[("purity", "aspherical")][1] > paper[("purity", "aspherical")][0]
    assert paper[("recovery", "spherical")][1] > paper[("recovery", "spherical")][0]
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        p0, p1 = _mixture(rng, 20000, 0.03)
        X = np.vstack([p0, p1])
        truth = np.array([0] * len(p0) + [1] * len(p1))
        init = np.full(len(X), -1, np.int32)
        init[:100] = 0
        init[len(p0):len(p0) + 100] = 1
        free = init < 0
        res = []
        for mode in (0, 1):
            out, npd = oracle.core_assign(X, init, 2, mode=mode)
            assert npd == 2
            res.append(_purity_recovery(out[free], truth[free]))
        (ps, rs), (pt, rt) = res
        assert pt[1] > ps[1] + 0.05 and rt[0] > rs[0] + 0.05, (seed, res)
        assert (pt > 0.5).all() and (rt > 0.5).all()
        assert (ps > 0.5).all() and (rs > 0.5).all()


# ------------------------------------------------------------ whole growth step

def _find(par, x):
    while par[x] != x:
        x = par[x]
    return x


def _brute_search(upos, vel, members, lab6, lx, lv, ax=0.8, av=1.0, n_loop=5, f_c=0.02,
                  an=1.2, nmin=20):
    """Core search by pairwise 6D links; also the last loop at which each member was in
    the searched background and the primary core's label."""
    nh = len(members)
    v = vel[members].astype(np.float64)
    bg = np.ones(nh, bool) if lab6 is None else (np.asarray(lab6) < 0)
    core = np.full(nh, -1, np.int32)
    lev = np.full(nh, -1, np.int32)
    searched = np.full(nh, -1, np.int32)
    lxl, lvl, thr = lx, lv, f_c * nh
    prim, plev = None, -1
    for l in range(n_loop):
        if l > 0:
            lxl, lvl, thr = lxl * ax, lvl * av, thr * an
        idx = np.flatnonzero(bg)
        searched[idx] = l
        par = {int(i): int(i) for i in idx}
        for a in range(len(idx)):
            i = idx[a]
            d = upos[idx[a + 1:]] - upos[i]
            dv = v[idx[a + 1:]] - v[i]
            q = (d * d).sum(1) / (lxl * lxl) + ((dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1])
                                                + dv[:, 2] * dv[:, 2]) / (lvl * lvl)
            for j in idx[a + 1:][q < 1.0]:
                ra, rb = _find(par, int(i)), _find(par, int(j))
                if ra != rb:
                    par[max(ra, rb)] = min(ra, rb)
        groups = {}
        for i in idx:
            groups.setdefault(_find(par, int(i)), []).append(int(i))
        good = {r: g for r, g in groups.items() if len(g) >= nmin and len(g) >= thr}
        if not good:
            break
        big = min(good, key=lambda r: (-len(good[r]), r))
        bg[:] = False
        for r, g in good.items():
            if r == big:
                bg[g] = True
            else:
                core[g] = members[r]
                lev[g] = l
        prim, plev = members[big], l
    if prim is not None:
        core[bg] = prim
        lev[bg] = plev
    return core, lev, searched, (-1 if prim is None else int(prim))


def _mahal(X, sel):
    m = X[sel].mean(0)
    S = np.cov(X[sel].T, bias=True)
    return m, S


def _d2(mode, m, S, Y):
    d = Y - m
    if mode == 0:
        return ((d[:, :3] ** 2).sum(1) / (np.trace(S[:3, :3]) / 3)
                + (d[:, 3:] ** 2).sum(1) / (np.trace(S[3:, 3:]) / 3))
    return np.einsum("ij,ij->i", d, np.linalg.solve(S, d.T).T)


def _brute_grow(upos, vel, members, lab6, lx, lv, beta_c=1.0, mode=2, n_loop=5, **kw):
    core, lev, searched, prim = _brute_search(upos, vel, members, lab6, lx, lv, n_loop=n_loop,
                                              **kw)
    grown = core.copy()
    if prim < 0:
        return core, lev, grown, []
    X = np.hstack([upos.astype(np.float64), vel[members].astype(np.float64)])
    labels = sorted(set(core[core >= 0].tolist()))
    clev = {c: int(lev[core == c][0]) for c in labels}
    init = {c: _mahal(X, core == c) for c in labels}
    alive = {c: True for c in labels}
    d2s = []
    for c in labels:
        if c == prim:
            continue
        mp = X[(searched >= clev[c] + 1) | (core == prim)].mean(0)
        m, S = init[c]
        d = mp - m
        d2s.append(float(d @ np.linalg.solve(S, d)))
        alive[c] = bool(np.linalg.eigvalsh(S).min() > 0) and d2s[-1] >= beta_c
    for c in labels:
        if not alive[c]:
            grown[core == c] = -1
    if not any(alive[c] for c in labels if c != prim):
        return core, lev, grown, d2s
    for l in range(n_loop - 1, -1, -1):
        act = [c for c in labels if alive[c] and (c == prim or clev[c] >= l)]
        todo = np.flatnonzero((grown < 0) & (searched == l))
        if len(todo) == 0:
            continue
        D = np.empty((len(todo), len(act)))
        for k, c in enumerate(act):
            m, S = _mahal(X, grown == c) if mode == 2 else init[c]
            D[:, k] = _d2(mode, m, S, X[todo])
        grown[todo] = np.array(act)[D.argmin(1)]  # act is in increasing label order
    return core, lev, grown, d2s


def _clumpy_halo(seed, nh=700, nclump=3):
    rng = np.random.default_rng(seed)
    upos = rng.normal(0, 3000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, 50, size=(nh, 3)).astype(np.float32)
    for c in range(nclump):
        s = slice(120 * c, 120 * c + 100)
        upos[s] = rng.normal(rng.uniform(-4000, 4000, 3), 500, size=(100, 3)).astype(np.int64)
        vel[s] = (rng.normal(0, 60, 3) + rng.normal(0, 8, size=(100, 3))).astype(np.float32)
    members = np.arange(nh, dtype=np.int32) * 3 + 2
    vel_all = np.zeros((members.max() + 1, 3), np.float32)
    vel_all[members] = vel
    lab6 = np.where(rng.random(nh) < 0.05, 1, -1).astype(np.int32)
    return upos, vel_all, members, lab6


@pytest.mark.parametrize("mode", [2, 1, 0])
def test_matches_brute_force_route(mode):
    """Default beta_C = 1, then beta_C between two candidate cores' D^2 to their primary
    group, so that cleaning keeps one and drops the other."""
    checked = dropped = 0
    for seed in (1, 2, 3, 4):
        upos, vel, members, lab6 = _clumpy_halo(seed)
        lv = 1.25 * oracle.halo_frame(vel, members)[3]
        for lx in (600.0, 900.0):
            betas = [1.0]
            for beta in betas:
                core, lev, grown, gap, nk = oracle.core_grow_halo(upos, vel, members, lab6, lx,
                                                                  lv, mode=mode, beta_c=beta)
                b = _brute_grow(upos, vel, members, lab6, lx, lv, mode=mode, beta_c=beta)
                assert np.array_equal(core, b[0]) and np.array_equal(lev, b[1])
                assert not np.any(gap[np.isfinite(gap)] < 1e-6), "near tie: pick another seed"
                assert np.array_equal(grown, b[2]), (seed, lx, mode, beta)
                assert nk == len(set(grown[grown >= 0].tolist()))
                checked += int((grown != core).sum())
                if beta == 1.0:
                    nk1 = nk
                else:
                    dropped += nk1 - nk
                d2 = sorted(b[3])
                if beta == 1.0 and len(d2) >= 2:
                    k = len(d2) // 2 - 1
                    assert d2[k + 1] > d2[k] * (1 + 1e-6)
                    betas.append(float(np.sqrt(d2[k] * d2[k + 1])))
    assert checked > 100  # growth assigned particles in these halos
    assert dropped > 0  # and cleaning dropped cores


def _blobs_with_halo():
    """Two 7^3 lattices (spacing 500), 3500 apart in x, moving at +-200 km/s with 0.3 km/s
    dispersion, plus 60 diffuse members: 30 near each blob in position and velocity but
    off the lattice far enough (>= 800) that no 6D link reaches them."""
    rng = np.random.default_rng(8)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3) * 500
    nb = len(g)
    base = np.array([100000, 100000, 100000])
    upos = [g + base, g + base + [3500, 0, 0]]
    vel = [rng.normal(0, 0.3, size=(nb, 3)) + [200, 0, 0],
           rng.normal(0, 0.3, size=(nb, 3)) - [200, 0, 0]]
    for sgn, off in ((1, 0), (-1, 3500)):
        c = base + [off + 1500, 1500, 1500]
        d = rng.normal(size=(30, 3))
        d = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(4000, 5000, (30, 1))
        upos.append(np.round(c + d).astype(np.int64))
        vel.append(rng.normal(0, 30, size=(30, 3)) + [sgn * 200, 0, 0])
    upos = np.vstack(upos).astype(np.int64)
    vel = np.vstack(vel).astype(np.float32)
    return upos, vel, np.arange(len(upos), dtype=np.int32), nb


def test_two_blobs_grown_by_hand():
    """Loop 0 finds blob A (label 0, the primary core) and blob B (label 343, a core of
    level 0); the 60 diffuse members link to nothing and leave the background at loop 0.
    B's mean is ~400 km/s from the primary group's mean against a 0.3 km/s dispersion:
    D^2 >> beta_C, B is kept. Growth at level 0 gives each diffuse member the blob that
    moves with it (velocities +-200 vs dispersions 0.3: the velocity term decides)."""
    upos, vel, members, nb = _blobs_with_halo()
    lv = 1.25 * oracle.halo_frame(vel, members)[3]
    core, lev, grown, gap, nk = oracle.core_grow_halo(upos, vel, members, None, 700.0, lv)
    assert (core[:nb] == 0).all() and (core[nb:2 * nb] == nb).all()
    assert (core[2 * nb:] == -1).all() and nk == 2
    assert (grown[:2 * nb] == core[:2 * nb]).all()
    assert (grown[2 * nb:2 * nb + 30] == 0).all() and (grown[2 * nb + 30:] == nb).all()
    # beta_C above every distance: B is dropped, no candidate core is left, no growth
    core2, _, grown2, _, nk2 = oracle.core_grow_halo(upos, vel, members, None, 700.0, lv,
                                                      beta_c=1e300)
    assert np.array_equal(core2, core) and nk2 == 1
    assert (grown2[:nb] == 0).all() and (grown2[nb:] == -1).all()


def test_single_core_is_not_grown():
    upos, vel, members, nb = _blobs_with_halo()
    keep = np.r_[0:nb, 2 * nb:2 * nb + 30]
    up, mem = upos[keep], np.arange(len(keep), dtype=np.int32)
    v = vel[keep]
    lv = 1.25 * oracle.halo_frame(v, mem)[3]
    core, lev, grown, gap, nk = oracle.core_grow_halo(up, v, mem, None, 700.0, lv)
    assert nk == 1 and np.array_equal(grown, core) and (grown[nb:] == -1).all()
    assert np.isnan(gap).all()


def test_exact_rescaling_changes_nothing():
    """Positions x2 (lx x2) and velocities x4 (lv x4): every 6D link term and every
    D^2 is computed from exactly scaled operands, so all decisions are identical."""
    upos, vel, members, lab6 = _clumpy_halo(5)
    lv = 1.25 * oracle.halo_frame(vel, members)[3]
    for mode in (2, 0):
        a = oracle.core_grow_halo(upos, vel, members, lab6, 700.0, lv, mode=mode)
        b = oracle.core_grow_halo(upos * 2, vel * 4, members, lab6, 1400.0, lv * 4, mode=mode)
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)
        assert (a[2] != a[0]).sum() > 0
