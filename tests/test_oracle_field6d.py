"""Pins for the oracle's field 6DFOF (Sec. 2.1, Eq. fof6d; Table 1 alpha_v = 1.25).

Inside each 3DFOF halo, members are linked iff dx^2/lx^2 + dv^2/lv^2 < 1 with
lv = alpha_v |Sigma_k|^(1/6). The pins tie the oracle to:
  - the alpha_v -> infinity limit, where Eq. fof6d becomes Eq. fof3d and the field 6D
    groups must be the 3DFOF halos;
  - an independent brute-force route (numpy determinant, pairwise predicate, a small
    union-find written here) on small boxes;
  - planted configurations: two blobs touching in space but moving apart, which 3DFOF
    joins and 6DFOF must separate; a halo with identical velocities (sigma = 0, no links).
"""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _table1():
    out = {}
    with open(os.path.join(HERE, "golden", "table1_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


ALPHA_V = _table1()["alpha_v"]


def _brute_field6d(pos, vel, label3, lx, alpha_v, nmin):
    """Independent route: per 3D group, sigma from numpy's determinant, every pair tested
    with dv2 = (dvx^2 + dvy^2) + dvz^2 and q = dx2/lx2 + dv2/lv2 in float64."""
    n = len(pos)
    out = np.full(n, -1, np.int32)
    L = 1 << 21
    for lab in np.unique(label3):
        m = np.flatnonzero(label3 == lab)
        if len(m) < nmin:
            continue
        p = pos[m].astype(np.int64)
        d = p - p[0]
        d = np.where(d >= L // 2, d - L, np.where(d < -L // 2, d + L, d))
        up = p[0] + d
        v = vel[m].astype(np.float64)
        det = np.linalg.det(np.cov(v.T, bias=True))
        sig = det ** (1.0 / 6.0) if det > 0 else 0.0
        lx2, lv2 = lx * lx, (alpha_v * sig) ** 2
        parent = list(range(len(m)))

        def find(x):
            while parent[x] != x:
                x = parent[x]
            return x

        with np.errstate(divide="ignore", invalid="ignore"):
            for i in range(len(m)):
                dx = up[i + 1:] - up[i]
                dx2 = (dx * dx).sum(1)
                dvv = v[i + 1:] - v[i]
                dv2 = (dvv[:, 0] * dvv[:, 0] + dvv[:, 1] * dvv[:, 1]) + dvv[:, 2] * dvv[:, 2]
                q = dx2 / lx2 + dv2 / lv2
                for j in np.flatnonzero(q < 1.0) + i + 1:
                    a, b = find(i), find(int(j))
                    if a != b:
                        parent[max(a, b)] = min(a, b)
        roots = np.array([find(k) for k in range(len(m))])
        for r in np.unique(roots):
            g = np.flatnonzero(roots == r)
            if len(g) >= nmin:
                out[m[g]] = m[g].min()
    return out


def test_alpha_v_infinite_gives_3dfof_halos():
    box = synth.named("c32")
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    assert int(np.floor(lx * lx)) + 1 == box.link_d2  # the same strict 3D link
    l6, rows = oracle.field6d(box.pos, box.vel, lab3, lx, alpha_v=1e30)
    cnt = np.bincount(lab3, minlength=box.n)
    in_halo = cnt[lab3] >= 20
    assert np.array_equal(l6[in_halo], lab3[in_halo])
    assert (l6[~in_halo] == -1).all()
    assert len(rows) == (cnt >= 20).sum()


def test_matches_brute_force_small_box():
    box = synth.small_clustered(4096, seed=synth.SEED0 + 77)
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    got, rows = oracle.field6d(box.pos, box.vel, lab3, lx, ALPHA_V, 20)
    exp = _brute_field6d(box.pos, box.vel, lab3, lx, ALPHA_V, 20)
    assert np.array_equal(got, exp)
    assert len(rows) > 0 and (got >= 0).sum() > 0


def test_bridged_blobs_are_split():
    """Two 7^3 grids of spacing 500 side by side (3DFOF with lx = 700 joins them into one
    halo), moving apart at +-200 km/s with 1 km/s internal dispersion. sigma_v =
    |Sigma|^(1/6) ~ (200 * 1 * 1)^(1/3) ~ 5.8, lv ~ 7.3: grid neighbours link (q ~ 0.51 +
    0.1), pairs across the blobs (|dv| ~ 400) never do, so 6DFOF returns the two grids."""
    rng = np.random.default_rng(8)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3) * 500
    a = g + 100000
    b = g + 100000 + [3500, 0, 0]
    nb = len(g)
    pos = np.vstack([a, b]).astype(np.int32)
    va = rng.normal(0, 1, size=(nb, 3)) + [200, 0, 0]
    vb = rng.normal(0, 1, size=(nb, 3)) - [200, 0, 0]
    vel = np.vstack([va, vb]).astype(np.float32)
    lx = 700.0
    lab3 = oracle.fof3d(pos, int(np.floor(lx * lx)) + 1)
    assert (lab3 == 0).all()  # one 3D halo
    l6, rows = oracle.field6d(pos, vel, lab3, lx, ALPHA_V, 20)
    assert 4.0 < rows[0, 2] < 8.0
    assert (l6[:nb] == 0).all()
    assert (l6[nb:] == nb).all()
    assert np.array_equal(l6, _brute_field6d(pos, vel, lab3, lx, ALPHA_V, 20))


def test_zero_dispersion_links_nothing():
    rng = np.random.default_rng(9)
    pos = np.round(rng.normal(0, 300, size=(200, 3)) + 50000).astype(np.int32)
    vel = np.tile(np.array([[5.0, 6.0, 7.0]], np.float32), (200, 1))
    lab3 = np.zeros(200, np.int32)
    l6, rows = oracle.field6d(pos, vel, lab3, 500.0, ALPHA_V, 20)
    assert rows[0, 2] == 0.0 and rows[0, 4] == 0.0
    assert (l6 == -1).all()


def test_rows_and_small_groups():
    box = synth.small_clustered(4096, seed=synth.SEED0 + 78)
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    l6, rows = oracle.field6d(box.pos, box.vel, lab3, lx, ALPHA_V, 20)
    cnt3 = np.bincount(lab3, minlength=box.n)
    assert np.array_equal(rows[:, 0], np.flatnonzero(cnt3 >= 20))
    assert np.array_equal(rows[:, 1], cnt3[cnt3 >= 20])
    np.testing.assert_allclose(rows[:, 3], lx * lx, rtol=0, atol=0)
    np.testing.assert_allclose(rows[:, 4], (ALPHA_V * rows[:, 2]) ** 2, rtol=1e-15)
    g = l6[l6 >= 0]
    c6 = np.bincount(g)
    assert (c6[c6 > 0] >= 20).all()
    # every 6D group lies inside one 3D halo and is labelled by its minimum index
    for lab in np.unique(g):
        mem = np.flatnonzero(l6 == lab)
        assert mem.min() == lab and len(np.unique(lab3[mem])) == 1
