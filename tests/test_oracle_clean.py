"""Pins for the oracle's significance cleaning of outlier groups (Sec. 2.2, "Cleaning
the catalogue", Eq. ellsig; beta_ell = 1 and N_min = 20 from Table 1).

A group of N particles needs <ell> >= ell_bar(ell_th) (1 + beta/sqrt(N)); otherwise its
smallest-ell particles go, one at a time, until it passes; fewer than N_min left removes
the group. Pinned by hand-built groups with values worked out here, by the closed-form
ell_bar(2.5) = 2.822744797663897, and by an independent brute-force route.
"""
import math

import numpy as np
import pytest

import oracle

LBAR = 2.822744797663897  # Eq. ellsig at ell_th = 2.5 (closed form, pinned elsewhere)


def _brute(ell, lab, ell_th=2.5, beta=1.0, nmin=20):
    lbar = math.sqrt(2 / math.pi) * math.exp(-ell_th ** 2 / 2) / math.erfc(ell_th / math.sqrt(2))
    out = np.full(len(lab), -1, np.int32)
    for g in np.unique(lab[lab >= 0]):
        mem = sorted(np.flatnonzero(lab == g), key=lambda i: (ell[i], i))
        for k in range(len(mem)):
            rest = mem[k:]
            if math.fsum(ell[rest]) / len(rest) >= lbar * (1 + beta / math.sqrt(len(rest))):
                if len(rest) >= nmin:
                    out[rest] = min(rest)
                break
    return out


def test_significant_group_unchanged():
    ell = np.full(30, 5.0)
    lab = np.full(30, 3, np.int32)
    lab[:3] = -1
    got, kept = oracle.clean_groups(ell, lab)
    assert kept == 1 and (got[3:] == 3).all() and (got[:3] == -1).all()


def test_never_significant_group_removed():
    # every member at 2.6 < ell_bar: no subset's mean reaches the threshold
    ell = np.full(50, 2.6)
    got, kept = oracle.clean_groups(ell, np.zeros(50, np.int32))
    assert kept == 0 and (got == -1).all()


def test_worked_cut():
    """20 members at 3.0 and 30 at 5.0 (labels 0..49, lows first). N = 50: mean 4.2 >=
    2.8227 (1 + 1/sqrt 50) = 3.2219 -> kept whole. With 45 lows at 2.5 instead: mean
    (112.5 + 150)/75 = 3.5 vs 2.8227 (1 + 1/sqrt 75) = 3.1487 -> kept whole as well. With
    60 lows at 2.5 and 20 highs at 3.5: N = 80, mean 2.75 < 3.1383; each removal of a 2.5
    raises the mean; the first k with (150 - 2.5 k + 70)/(80 - k) >= 2.8227 (1 +
    1/sqrt(80 - k)) is worked out below and must be the cut."""
    ell = np.r_[np.full(20, 3.0), np.full(30, 5.0)]
    got, kept = oracle.clean_groups(ell, np.zeros(50, np.int32))
    assert kept == 1 and (got == 0).all()
    ell = np.r_[np.full(60, 2.5), np.full(20, 3.5)]
    k = next(k for k in range(80)
             if (150 - 2.5 * k + 70) / (80 - k) >= LBAR * (1 + 1 / math.sqrt(80 - k)))
    got, kept = oracle.clean_groups(ell, np.zeros(80, np.int32))
    assert kept == 1
    assert (got[:k] == -1).all() and (got[k:] == k).all()  # relabelled to the smallest kept


def test_drop_below_nmin():
    # 40 at 2.5 and 16 at 3.6: the first significant subset has fewer than 20 members
    ell = np.r_[np.full(40, 2.5), np.full(16, 3.6)]
    m = next(56 - k for k in range(56)
             if (40 * 2.5 + 16 * 3.6 - 2.5 * min(k, 40) - 3.6 * max(0, k - 40)) / (56 - k)
             >= LBAR * (1 + 1 / math.sqrt(56 - k)))
    assert m < 20
    got, kept = oracle.clean_groups(ell, np.zeros(56, np.int32))
    assert kept == 0 and (got == -1).all()
    assert (_brute(ell, np.zeros(56, np.int32)) == -1).all()


def test_ties_remove_smaller_index_first():
    ell = np.r_[np.full(10, 2.5), np.full(25, 4.0)]
    ell = ell[::-1].copy()  # the ties at 2.5 now sit at the highest indices
    lab = np.zeros(35, np.int32)
    got, _ = oracle.clean_groups(ell, lab)
    exp = _brute(ell, lab)
    assert np.array_equal(got, exp)


def test_infinite_ell_keeps_group():
    ell = np.r_[np.full(25, 2.5), [np.inf]]
    got, kept = oracle.clean_groups(ell, np.zeros(26, np.int32))
    assert kept == 1 and (got == 0).all()


def test_matches_brute_force_random_groups():
    rng = np.random.default_rng(12)
    n = 4000
    lab = np.full(n, -1, np.int32)
    ell = 2.5 + rng.exponential(0.35, size=n)
    start = 0
    for size in rng.integers(10, 200, size=25):
        if start + size > n:
            break
        idx = rng.choice(np.arange(start, start + 2 * size), size=size, replace=False)
        idx = idx[idx < n]
        lab[idx] = idx.min()
        start += 2 * size
    ell = ell.astype(np.float32).astype(np.float64)
    got, kept = oracle.clean_groups(ell, lab)
    exp = _brute(ell, lab)
    assert np.array_equal(got, exp)
    assert 0 < kept < len(np.unique(lab[lab >= 0]))
