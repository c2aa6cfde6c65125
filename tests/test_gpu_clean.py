"""Significance cleaning of outlier groups (Sec. 2.2, Eq. ellsig) on the GPU vs the
oracle, bit-exact: both take FP64 sums of the same FP32 ell values, which are exact and
so independent of the order of additions, and the same rounded threshold."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1902_01010_gb300 import Context

    return Context(0)


def _gpu(ctx, ell, lab, beta=1.0, **kw):
    from paper_1902_01010_gb300 import Params

    e = torch.from_numpy(np.ascontiguousarray(ell, np.float32)).cuda()
    l6 = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).cuda()
    kept = ctx.clean_groups(e, l6, Params.default(**kw), beta)
    return l6.cpu().numpy(), kept


def _random_groups(seed, n=20000, ngroups=120):
    rng = np.random.default_rng(seed)
    lab = np.full(n, -1, np.int32)
    perm = rng.permutation(n)
    ell = (2.5 + rng.exponential(0.3, size=n)).astype(np.float32)
    start = 0
    for size in rng.integers(5, 400, size=ngroups):
        idx = perm[start:start + size]
        start += size
        if start > n:
            break
        lab[idx] = idx.min()
        # each group its own tail: some pass whole, some after removals, some never
        ell[idx] = (2.5 + rng.exponential(rng.uniform(0.1, 1.5), size=len(idx))).astype(np.float32)
    return ell, lab


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_groups_match_oracle(ctx, seed):
    ell, lab = _random_groups(seed)
    got, kept = _gpu(ctx, ell, lab)
    exp, kexp = oracle.clean_groups(ell.astype(np.float64), lab)
    assert np.array_equal(got, exp) and kept == kexp
    assert 0 < kept < len(np.unique(lab[lab >= 0]))


def test_parameters_and_edges(ctx):
    ell, lab = _random_groups(4)
    for beta, nmin in ((0.0, 20), (3.0, 20), (1.0, 5), (1.0, 100)):
        got, kept = _gpu(ctx, ell, lab, beta, nmin=nmin)
        exp, kexp = oracle.clean_groups(ell.astype(np.float64), lab, 2.5, beta, nmin)
        assert np.array_equal(got, exp) and kept == kexp, (beta, nmin)
    # no groups at all
    got, kept = _gpu(ctx, ell, np.full(len(ell), -1, np.int32))
    assert kept == 0 and (got == -1).all()
    # a group holding an infinite ell is kept whole; one big group over many chunks
    n = 5000
    e = np.full(n, 2.5, np.float32)
    e[-1] = np.inf
    got, kept = _gpu(ctx, e, np.zeros(n, np.int32))
    assert kept == 1 and (got == 0).all()
    e = np.r_[np.full(4000, 2.5), np.full(1000, 4.5)].astype(np.float32)
    got, kept = _gpu(ctx, e, np.zeros(n, np.int32))
    exp, kexp = oracle.clean_groups(e.astype(np.float64), np.zeros(n, np.int32))
    assert np.array_equal(got, exp) and kept == kexp


def test_after_substructure_search(ctx):
    """The 64^3 box through vr_find_substructure, then cleaning of its 6D groups; the
    oracle cleans the same groups with the same FP32 ell."""
    box = synth.named("m64")
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    ell = out["ell"].cpu().numpy()
    l6 = out["label6"].cpu().numpy()
    assert (l6 >= 0).sum() > 0
    exp, kexp = oracle.clean_groups(ell.astype(np.float64), l6)
    kept = ctx.clean_groups(out["ell"], out["label6"])
    assert np.array_equal(out["label6"].cpu().numpy(), exp) and kept == kexp
