"""Pins for the oracle's two-stage linking (Sec. 2.2, "Linking particles": the relaxed
pass that grows the conservative candidate substructures, and the merge threshold
f_merge,th = 0.25; gamma factors of Table A1).

Tied to: the identity at gamma = 1 (the relaxed pass equals the conservative one, so
nothing can grow or join); an independent brute-force route; hand-built trails, bridges
and competing groups whose outcome follows from counting links by hand.
"""
import math

import numpy as np

import oracle

GAM1 = (1.0, 1.0, 1.0, 1.0)


def _brute(upos, vel, members, ell, lab1, prm, ell_th, v_ratio, theta_op, use_lv, use_vt,
           gam, f_merge):
    nh = len(members)
    thr = ell_th / gam[0]
    lx2, lv2 = prm[0] * gam[1] * gam[1], prm[1]
    vr2 = (v_ratio * gam[2]) ** 2
    c2 = math.cos(theta_op * gam[3]) ** 2
    cand = [lab1[i] >= 0 or ell[i] >= thr for i in range(nh)]
    v = vel[members].astype(np.float64)
    edges = []
    for i in range(nh):
        for j in range(i + 1, nh):
            if not (cand[i] and cand[j]):
                continue
            d = upos[i] - upos[j]
            q = float(d @ d) / lx2
            if use_lv:
                dv = v[i] - v[j]
                q = q + ((dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2]) / lv2
            if not q < 1.0:
                continue
            if use_vt:
                ui, uj = v[i] - prm[2:5], v[j] - prm[2:5]
                si = (ui[0] * ui[0] + ui[1] * ui[1]) + ui[2] * ui[2]
                sj = (uj[0] * uj[0] + uj[1] * uj[1]) + uj[2] * uj[2]
                dot = (ui[0] * uj[0] + ui[1] * uj[1]) + ui[2] * uj[2]
                if not (si > 0 and sj > 0 and si <= vr2 * sj and sj <= vr2 * si and dot >= 0
                        and dot * dot >= (c2 * si) * sj):
                    continue
            edges.append((i, j))
    par = list(range(nh))

    def find(x):
        while par[x] != x:
            x = par[x]
        return x

    for i, j in edges:
        if lab1[i] < 0 and lab1[j] < 0:
            a, b = find(i), find(j)
            par[max(a, b)] = min(a, b)
    cnt = {}
    for i, j in edges:
        if (lab1[i] < 0) != (lab1[j] < 0):
            u, t = (i, j) if lab1[i] < 0 else (j, i)
            k = (find(u), int(lab1[t]))
            cnt[k] = cnt.get(k, 0) + 1
    best = {}
    for (c, g), n in sorted(cnt.items()):
        if c not in best or n > best[c][1]:
            best[c] = (g, n)
    grown = [int(lab1[i]) if lab1[i] >= 0 else (best[find(i)][0] if cand[i] and find(i) in best else -1)
             for i in range(nh)]
    n0 = {}
    for i in range(nh):
        if lab1[i] >= 0:
            n0[int(lab1[i])] = n0.get(int(lab1[i]), 0) + 1
    cross = {}
    for i, j in edges:
        a, b = grown[i], grown[j]
        if a >= 0 and b >= 0 and a != b:
            k = (min(a, b), max(a, b))
            cross[k] = cross.get(k, 0) + 1
    gp = {g: g for g in n0}

    def gfind(x):
        while gp[x] != x:
            x = gp[x]
        return x

    for (a, b), n in cross.items():
        if n > f_merge * n0[a] or n > f_merge * n0[b]:
            ra, rb = gfind(a), gfind(b)
            gp[max(ra, rb)] = min(ra, rb)
    mins = {}
    for i in range(nh):
        if grown[i] >= 0:
            r = gfind(grown[i])
            mins[r] = min(mins.get(r, 1 << 40), int(members[i]))
    return np.array([mins[gfind(grown[i])] if grown[i] >= 0 else -1 for i in range(nh)], np.int32)


def _halo(seed, nh=500):
    rng = np.random.default_rng(seed)
    upos = rng.integers(0, 40000, size=(nh, 3)).astype(np.int64)
    vel = rng.normal(0, 100, size=(nh, 3)).astype(np.float32)
    # two cold clumps
    for c, (cx, vx) in enumerate(((10000, 150.0), (26000, -120.0))):
        s = slice(40 * c, 40 * c + 60)
        upos[s] = rng.normal(cx, 1200, size=(60, 3)).astype(np.int64)
        vel[s] = (np.array([vx, 30, 0]) + rng.normal(0, 10, size=(60, 3))).astype(np.float32)
    members = np.arange(nh, dtype=np.int32) * 3 + 7
    vel_all = np.zeros((members.max() + 1, 3), np.float32)
    vel_all[members] = vel
    ell = 2.5 + rng.exponential(0.6, size=nh) - (rng.random(nh) < 0.5) * 1.0
    return upos, vel_all, members, ell


def _stage1(upos, vel_all, members, ell, prm):
    cand = (ell >= 2.5).astype(np.uint8)
    return oracle.fof6d_halo(upos, vel_all, members, cand, prm)


def test_identity_at_gamma_one():
    upos, vel, members, ell = _halo(3)
    prm = np.array([2500.0 ** 2, 80.0 ** 2, 5.0, -3.0, 1.0])
    lab1 = _stage1(upos, vel, members, ell, prm)
    assert (lab1 >= 0).sum() > 0
    got = oracle.grow_halo(upos, vel, members, ell, lab1, prm, gam=GAM1)
    assert np.array_equal(got, lab1)


def test_matches_brute_force():
    for seed in (4, 5, 6):
        upos, vel, members, ell = _halo(seed)
        prm = np.array([2500.0 ** 2, 80.0 ** 2, 5.0, -3.0, 1.0])
        lab1 = _stage1(upos, vel, members, ell, prm)
        for gam, fm in (((1.0, 2.0, 1.0, 1.0), 0.25), ((1.3, 1.5, 1.5, 1.5), 0.1),
                        ((1.0, 2.0, 1.0, 1.0), 0.0)):
            got = oracle.grow_halo(upos, vel, members, ell, lab1, prm, gam=gam, f_merge=fm)
            exp = _brute(upos, vel, members, ell, lab1, prm, 2.5, 2.0, 0.1 * math.pi, 1, 1, gam, fm)
            assert np.array_equal(got, exp), (seed, gam, fm)
            assert (got >= 0).sum() >= (lab1 >= 0).sum()  # growth never loses a member


def _line(xs):
    upos = np.zeros((len(xs), 3), np.int64)
    upos[:, 0] = xs
    return upos


def test_trail_joins_group():
    """A 25-member group on a line of spacing 100 (lx = 150 links it in stage 1), then a
    trail of 10 untagged candidates at spacing 250 from the group's end: only the relaxed
    length 300 links them, as one component touching the group: all join it."""
    xs = np.r_[np.arange(25) * 100, 2400 + 250 * np.arange(1, 11)]
    upos = _line(xs)
    n = len(xs)
    members = np.arange(n, dtype=np.int32)
    vel = np.zeros((n, 3), np.float32)
    ell = np.full(n, 3.0)
    prm = np.array([150.0 ** 2, 1.0, 0, 0, 0])
    lab1 = oracle.fof6d_halo(upos, vel, members, np.ones(n, np.uint8), prm, use_lv=0, use_vt=0)
    assert (lab1[:25] == 0).all() and (lab1[25:] == -1).all()
    got = oracle.grow_halo(upos, vel, members, ell, lab1, prm, use_lv=0, use_vt=0)
    assert (got == 0).all()
    # below the relaxed ell threshold the trail cannot grow
    ell2 = ell.copy()
    ell2[25:] = 2.0
    got = oracle.grow_halo(upos, vel, members, ell2, lab1, prm, use_lv=0, use_vt=0)
    assert np.array_equal(got, lab1)


def test_merge_threshold():
    """Groups A (x = 0..2400, 25 members) and B (x = 2650..5050, 25 members), spacing
    100: stage-1 length 150 keeps them apart; the relaxed length 300 links the last
    members of A to the first of B. Links across the gap of 250: pairs at distance
    < 300, i.e. (2400, 2650) only at 250, (2300, 2650) at 350 no, (2400, 2750) no -> 1
    link. 1 > f N_o = f 25 iff f < 0.04."""
    xs = np.r_[np.arange(25) * 100, 2650 + np.arange(25) * 100]
    upos = _line(xs)
    n = len(xs)
    members = np.arange(n, dtype=np.int32)
    vel = np.zeros((n, 3), np.float32)
    ell = np.full(n, 3.0)
    prm = np.array([150.0 ** 2, 1.0, 0, 0, 0])
    lab1 = oracle.fof6d_halo(upos, vel, members, np.ones(n, np.uint8), prm, use_lv=0, use_vt=0)
    assert (lab1[:25] == 0).all() and (lab1[25:] == 25).all()
    kw = dict(use_lv=0, use_vt=0)
    assert np.array_equal(oracle.grow_halo(upos, vel, members, ell, lab1, prm, f_merge=0.25, **kw), lab1)
    assert (oracle.grow_halo(upos, vel, members, ell, lab1, prm, f_merge=0.039, **kw) == 0).all()
    assert np.array_equal(oracle.grow_halo(upos, vel, members, ell, lab1, prm, f_merge=0.04, **kw), lab1)


def test_component_joins_group_with_most_links():
    """An untagged linked pair (indices 25, 26; relaxed length 300, strict) between groups A
    (indices 0-24, x = 0..2400)
    and B (25 members from x = b0, spacing 100), counted by hand:
      pair (2650, 2850), b0 = 3100: 2650-2400 = 250 -> 1 link to A; 2850-3100 = 250 -> 1
        link to B: a tie, so the pair joins the smaller label, A;
      pair (2650, 2900), b0 = 3050: 1 link to A; 2900-3050 = 150, 2900-3150 = 250 -> 2 to
        B: it joins B;
      pair (2750, 2950), b0 = 3100: none to A (350); 2950-3100, 2950-3200 -> 2 to B.
    No join of A and B: at most 2 cross links against f N_o = 6.25."""
    a = np.arange(25) * 100
    for pair, b0, to_b in (((2650, 2850), 3100, False), ((2650, 2900), 3050, True),
                           ((2750, 2950), 3100, True)):
        xs = np.r_[a, pair, b0 + np.arange(25) * 100]
        n = len(xs)
        members = np.arange(n, dtype=np.int32)
        vel = np.zeros((n, 3), np.float32)
        ell = np.full(n, 3.0)
        prm = np.array([150.0 ** 2, 1.0, 0, 0, 0])
        lab1 = np.r_[np.zeros(25), [-1, -1], np.full(25, 27)].astype(np.int32)
        got = oracle.grow_halo(_line(xs), vel, members, ell, lab1, prm, use_lv=0, use_vt=0)
        assert (got[:25] == 0).all(), (pair, b0)
        if to_b:  # B with the pair is labelled by its minimum index, the pair's 25
            assert (got[25:] == 25).all(), (pair, b0)
        else:
            assert (got[25:27] == 0).all() and (got[27:] == 27).all(), (pair, b0)
        exp = _brute(_line(xs), vel, members, ell, lab1, prm, 2.5, 2.0, 0.1 * math.pi, 0, 0,
                     oracle.GROW_DEFAULTS, 0.25)
        assert np.array_equal(got, exp)
