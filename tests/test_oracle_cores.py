"""Pins for the oracle's core search (Sec. 2.3, "Core Identification", Eq. coreloop;
Table 1: alpha_x,C = 0.8, alpha_v,C = 1.0, n_loop,C = 5, f_C = 0.02, alpha_N,C = 1.2).

Tied to: two bridged lattice blobs whose loop-by-loop outcome is worked out by hand; an
independent brute-force route (pairwise 6D links, a union-find written here) on small
halos; the degenerate cases (no background, a single blob).
"""
import numpy as np

import oracle


def _brute(upos, vel, members, lab6, lx, lv, ax=0.8, av=1.0, n_loop=5, f_c=0.02, an=1.2, nmin=20):
    nh = len(members)
    v = vel[members].astype(np.float64)
    bg = np.ones(nh, bool) if lab6 is None else (np.asarray(lab6) < 0)
    core = np.full(nh, -1, np.int32)
    lev = np.full(nh, -1, np.int32)
    lxl, lvl, thr = lx, lv, f_c * nh
    prim, plev = None, -1
    for l in range(n_loop):
        if l > 0:
            lxl, lvl, thr = lxl * ax, lvl * av, thr * an
        idx = np.flatnonzero(bg)
        par = {int(i): int(i) for i in idx}

        def find(x):
            while par[x] != x:
                x = par[x]
            return x

        for a in range(len(idx)):
            i = idx[a]
            d = upos[idx[a + 1:]] - upos[i]
            dv = v[idx[a + 1:]] - v[i]
            q = (d * d).sum(1) / (lxl * lxl) + ((dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1])
                                                + dv[:, 2] * dv[:, 2]) / (lvl * lvl)
            for j in idx[a + 1:][q < 1.0]:
                ra, rb = find(int(i)), find(int(j))
                if ra != rb:
                    par[max(ra, rb)] = min(ra, rb)
        groups = {}
        for i in idx:
            groups.setdefault(find(int(i)), []).append(int(i))
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
    return core, lev


def _blobs():
    """Two 7^3 lattices (spacing 500) side by side, moving apart at +-200 with 0.3 km/s
    internal dispersion: one 3D halo of 686 members."""
    rng = np.random.default_rng(8)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3) * 500
    nb = len(g)
    upos = np.vstack([g + 100000, g + 100000 + [3500, 0, 0]]).astype(np.int64)
    vel = np.vstack([rng.normal(0, 0.3, size=(nb, 3)) + [200, 0, 0],
                     rng.normal(0, 0.3, size=(nb, 3)) - [200, 0, 0]]).astype(np.float32)
    return upos, vel, np.arange(2 * nb, dtype=np.int32), nb


def test_two_blobs_worked_by_hand():
    """sigma_v = |Sigma|^(1/6) ~ (200 * 0.3 * 0.3)^(1/3) ~ 2.6, lv = 1.25 sigma_v ~ 3.3
    km/s; neighbours differ by |dv| ~ 0.7, a velocity term ~ 0.05. Loop 0 (lx = 700)
    finds the two blobs as groups of 343 (>= f_C N_H = 13.7; across the blobs |dv| ~ 400):
    equal sizes, so the smaller label (0) is the primary core and blob B a core of level
    0; loop 1 (lx = 560, spatial term 0.80 for neighbours) finds blob A whole again; loop
    2 (lx = 448 < 500) links nothing: stop. A is the primary core of level 1."""
    upos, vel, members, nb = _blobs()
    lv = 1.25 * oracle.halo_frame(vel, members)[3]
    assert 2.0 < lv / 1.25 < 3.5
    core, lev, nc = oracle.core_search_halo(upos, vel, members, None, 700.0, lv)
    assert nc == 2
    assert (core[:nb] == 0).all() and (lev[:nb] == 1).all()
    assert (core[nb:] == nb).all() and (lev[nb:] == 0).all()
    b = _brute(upos, vel, members, None, 700.0, lv)
    assert np.array_equal(core, b[0]) and np.array_equal(lev, b[1])


def test_substructure_is_not_background():
    upos, vel, members, nb = _blobs()
    lv = 1.25 * oracle.halo_frame(vel, members)[3]
    lab6 = np.full(2 * nb, -1, np.int32)
    lab6[nb:] = nb  # blob B is substructure
    core, lev, nc = oracle.core_search_halo(upos, vel, members, lab6, 700.0, lv)
    assert nc == 1 and (core[:nb] == 0).all() and (core[nb:] == -1).all()
    lab6[:] = 0  # everything is substructure: no background, no core
    core, lev, nc = oracle.core_search_halo(upos, vel, members, lab6, 700.0, lv)
    assert nc == 0 and (core == -1).all() and (lev == -1).all()


def test_matches_brute_force_random_halos():
    for seed in (1, 2, 3):
        rng = np.random.default_rng(seed)
        nh = 600
        upos = rng.normal(0, 3000, size=(nh, 3)).astype(np.int64)
        vel = rng.normal(0, 50, size=(nh, 3)).astype(np.float32)
        for c in range(3):  # three dense cold clumps
            s = slice(100 * c, 100 * c + 90)
            upos[s] = rng.normal(rng.uniform(-4000, 4000, 3), 400, size=(90, 3)).astype(np.int64)
            vel[s] = (rng.normal(0, 60, 3) + rng.normal(0, 8, size=(90, 3))).astype(np.float32)
        members = np.arange(nh, dtype=np.int32) * 2 + 1
        vel_all = np.zeros((members.max() + 1, 3), np.float32)
        vel_all[members] = vel
        lab6 = np.where(rng.random(nh) < 0.05, 1, -1).astype(np.int32)
        lv = 1.25 * oracle.halo_frame(vel_all, members)[3]
        for lx in (500.0, 900.0):
            core, lev, _ = oracle.core_search_halo(upos, vel_all, members, lab6, lx, lv)
            b = _brute(upos, vel_all, members, lab6, lx, lv)
            assert np.array_equal(core, b[0]) and np.array_equal(lev, b[1]), (seed, lx)
