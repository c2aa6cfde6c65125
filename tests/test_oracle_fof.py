"""Pins for the oracle's 3D friends-of-friends (Sec. 2.1, Eq. fof3d) and halo set-up.

The oracle's grid FOF is checked against (a) its own O(N^2) brute force, (b) an
independent route: scipy's periodic k-d tree for candidate pairs plus scipy's
connected components, and (c) invariants of the definition.
"""
import numpy as np
import pytest

import oracle
import synth

L = 1 << 21


def _pairs_scipy(pos, link_d2):
    from scipy.spatial import cKDTree

    t = cKDTree(pos.astype(np.float64), boxsize=float(L))
    pr = t.query_pairs(np.sqrt(float(link_d2)) + 1.0, output_type="ndarray")
    if len(pr) == 0:
        return pr.reshape(0, 2)
    d = pos[pr[:, 0]].astype(np.int64) - pos[pr[:, 1]].astype(np.int64)
    d = (d + L // 2) % L - L // 2
    d2 = (d * d).sum(1)
    return pr[d2 < link_d2]


def _components(n, pairs):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    m = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n)) if len(pairs) \
        else coo_matrix((n, n))
    _, comp = connected_components(m, directed=False)
    # canonical: minimum index of each component
    mins = np.full(comp.max() + 1, n, np.int64)
    np.minimum.at(mins, comp, np.arange(n))
    return mins[comp].astype(np.int32)


def _random_clustered(n, seed, nclump=6, spread=3000):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, L, size=(nclump, 3))
    which = rng.integers(0, nclump + 1, size=n)
    pos = rng.integers(0, L, size=(n, 3))
    inclump = which < nclump
    pos[inclump] = ctr[which[inclump]] + rng.normal(0, spread, size=(inclump.sum(), 3)).astype(np.int64)
    return (pos % L).astype(np.int32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_grid_equals_brute_clustered(seed):
    pos = _random_clustered(1500, seed)
    T = 1200 ** 2
    a = oracle.fof3d(pos, T)
    b = oracle.fof3d(pos, T, brute=True)
    assert np.array_equal(a, b)
    assert len(np.unique(a)) < len(a)  # something linked


def test_grid_equals_brute_wrap():
    # clumps straddling every face, edge and corner of the periodic box
    rng = np.random.default_rng(7)
    pts = []
    for cx in (0, L // 2):
        for cy in (0, L // 2):
            for cz in (0, L // 2):
                c = np.array([cx, cy, cz])
                pts.append(c + rng.normal(0, 300, size=(80, 3)).astype(np.int64))
    pos = (np.concatenate(pts) % L).astype(np.int32)
    T = 900 ** 2
    a = oracle.fof3d(pos, T)
    b = oracle.fof3d(pos, T, brute=True)
    assert np.array_equal(a, b)
    # the clump at the origin is split across the box corners; it must be one group
    g = a[:80]
    assert len(np.unique(g)) == 1 and g[0] == 0


def test_matches_independent_scipy_route():
    box = synth.named("c32")
    a = oracle.fof3d(box.pos, box.link_d2)
    pairs = _pairs_scipy(box.pos, box.link_d2)
    b = _components(box.n, pairs)
    assert np.array_equal(a, b)


def test_strict_inequality_and_exact_threshold():
    # two points at squared distance exactly T are not linked; at T-1 they are
    T = 5 ** 2 + 12 ** 2  # 169: separation (5, 12, 0) has d^2 = 169
    pos = np.array([[100, 100, 100], [105, 112, 100]], np.int32)
    assert list(oracle.fof3d(pos, T)) == [0, 1]
    assert list(oracle.fof3d(pos, T + 1)) == [0, 0]
    # across the periodic boundary
    pos = np.array([[L - 2, 0, 0], [3, 0, 0]], np.int32)  # minimum-image separation 5
    assert list(oracle.fof3d(pos, 26)) == [0, 0]
    assert list(oracle.fof3d(pos, 25)) == [0, 1]


def test_invariants_and_permutation():
    pos = _random_clustered(3000, 11)
    T = 1000 ** 2
    lab = oracle.fof3d(pos, T)
    n = len(lab)
    idx = np.arange(n)
    # canonical: label is the minimum index of its group
    assert np.all(lab <= idx)
    assert np.all(lab[lab] == lab)
    mins = np.full(n, n)
    np.minimum.at(mins, lab, idx)
    assert np.all(mins[lab] == lab)
    # every linked pair shares a label
    pairs = _pairs_scipy(pos, T)
    assert np.all(lab[pairs[:, 0]] == lab[pairs[:, 1]])
    # permutation invariance of the partition
    perm = np.random.default_rng(3).permutation(n)
    lab2 = oracle.fof3d(pos[perm], T)
    # map back: groups of perm[i] must coincide
    back = np.empty(n, np.int64)
    back[perm] = np.arange(n)
    g1 = lab[perm]          # label (original numbering) of permuted particle i
    # same partition <=> bijection between labels
    pairs_ = np.unique(np.stack([g1, lab2], 1), axis=0)
    assert len(np.unique(pairs_[:, 0])) == len(pairs_) == len(np.unique(pairs_[:, 1]))


def test_empty_and_singletons():
    assert oracle.fof3d(np.zeros((0, 3), np.int32), 100).shape == (0,)
    pos = np.array([[0, 0, 0], [0, 0, 0], [L // 2, 0, 0]], np.int32)
    assert list(oracle.fof3d(pos, 1)) == [0, 0, 2]  # coincident points: d^2 = 0 < 1


def test_halos_and_unwrap():
    lab = np.array([0, 0, 2, 0, 2, 5], np.int32)
    off, mem = oracle.halos(lab, 2)
    assert list(off) == [0, 3, 5]
    assert list(mem) == [0, 1, 3, 2, 4]
    off, mem = oracle.halos(lab, 3)
    assert list(off) == [0, 3] and list(mem) == [0, 1, 3]
    pos = np.array([[L - 1, 5, 0], [2, 5, L - 3], [L - 5, 0, 2]], np.int32)
    up = oracle.unwrap(pos, np.array([0, 1, 2], np.int32))
    assert up.tolist() == [[L - 1, 5, 0], [L + 2, 5, -3], [L - 5, 0, 2]]
