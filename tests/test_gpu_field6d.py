"""Field 6DFOF of 3DFOF halos (Sec. 2.1, Eq. fof6d) on the GPU vs the oracle.

Labels are compared bit-exactly twice: against the oracle's own field 6DFOF, and against
the oracle's linker fed the GPU's per-halo lengths (so a last-bit difference in sigma_v
could not hide or cause a flip). sigma_v = |Sigma|^(1/6) agrees to 1e-12 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
ALPHA_V = 1.25  # Table 1


@pytest.fixture(scope="module")
def ctx():
    from paper_1902_01010_gb300 import Context

    return Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu(ctx, pos, vel, lab3, lx, alpha_v=ALPHA_V):
    l6, hs = ctx.fof6d_field(_dev(pos), _dev(vel), _dev(lab3.astype(np.int32)), lx, alpha_v)
    ctx.sync()
    return l6.cpu().numpy(), hs.cpu().numpy()


@pytest.mark.parametrize("name", ["c32", "m64"])
def test_matches_oracle(ctx, name):
    from paper_1902_01010_gb300.vr import H_LABEL, H_NH, H_SIGMA, H_LX2, H_LV2, H_SEARCHED

    box = synth.named(name)
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    got, hs = _gpu(ctx, box.pos, box.vel, lab3, lx)
    exp, rows = oracle.field6d(box.pos, box.vel, lab3, lx, ALPHA_V, 20)
    assert len(hs) == len(rows) > 0
    assert np.array_equal(hs[:, H_LABEL], rows[:, 0]) and np.array_equal(hs[:, H_NH], rows[:, 1])
    np.testing.assert_allclose(hs[:, H_SIGMA], rows[:, 2], rtol=1e-12)
    assert (hs[:, H_LX2] == lx * lx).all() and (hs[:, H_SEARCHED] == 1).all()
    np.testing.assert_allclose(hs[:, H_LV2], rows[:, 4], rtol=1e-12)
    assert np.array_equal(got, exp)
    assert (got >= 0).sum() > 1000
    # the oracle's linker fed the GPU's lengths and frame
    off, mem = oracle.halos(lab3, 20)
    vel_all = box.vel
    for h in range(len(off) - 1):
        m = mem[off[h]:off[h + 1]]
        up = oracle.unwrap(box.pos, m)
        prm = np.array([hs[h, H_LX2], hs[h, H_LV2], 0.0, 0.0, 0.0])
        l6 = oracle.fof6d_halo(up, vel_all, m, np.ones(len(m), np.uint8), prm, use_lv=1, use_vt=0)
        assert np.array_equal(got[m], l6), h


def test_alpha_v_infinite_gives_3d_halos(ctx):
    box = synth.named("c32")
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    got, _ = _gpu(ctx, box.pos, box.vel, lab3, 0.2 * synth.mean_spacing(box.n), alpha_v=1e30)
    cnt = np.bincount(lab3, minlength=box.n)
    inh = cnt[lab3] >= 20
    assert np.array_equal(got[inh], lab3[inh]) and (got[~inh] == -1).all()


def test_bridged_blobs_and_zero_dispersion(ctx):
    rng = np.random.default_rng(8)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3) * 500
    nb = len(g)
    pos = np.vstack([g + 100000, g + 100000 + [3500, 0, 0]]).astype(np.int32)
    vel = np.vstack([rng.normal(0, 1, size=(nb, 3)) + [200, 0, 0],
                     rng.normal(0, 1, size=(nb, 3)) - [200, 0, 0]]).astype(np.float32)
    lab3 = np.zeros(2 * nb, np.int32)
    got, _ = _gpu(ctx, pos, vel, lab3, 700.0)
    assert (got[:nb] == 0).all() and (got[nb:] == nb).all()
    vel0 = np.tile(np.array([[5.0, 6.0, 7.0]], np.float32), (2 * nb, 1))
    got0, hs0 = _gpu(ctx, pos, vel0, lab3, 700.0)
    assert (got0 == -1).all() and hs0[0, 8] == 0.0


def test_large_box_sampled_halos(ctx):
    """256^3 mass-function box at full size through the C ABI: the 6D labels of a sample
    of halos (the largest ones and a spread of small ones) match the oracle's linker fed
    the GPU's lengths."""
    from paper_1902_01010_gb300.vr import H_LX2, H_LV2

    box = synth.named("c256")
    pos, vel = _dev(box.pos), _dev(box.vel)
    lab = ctx.fof3d(pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    l6, hs = ctx.fof6d_field(pos, vel, lab, lx, ALPHA_V)
    ctx.sync()
    got, hs, lab3 = l6.cpu().numpy(), hs.cpu().numpy(), lab.cpu().numpy()
    off, mem = oracle.halos(lab3, 20)
    sizes = np.diff(off)
    order = np.argsort(-sizes)
    pick = list(order[1:3]) + list(order[:: max(1, len(order) // 12)])
    for h in pick:
        m = mem[off[h]:off[h + 1]]
        if len(m) > 60000:
            continue  # the O(N_H^2) oracle linker takes minutes on the largest halos
        up = oracle.unwrap(box.pos, m)
        prm = np.array([hs[h, H_LX2], hs[h, H_LV2], 0.0, 0.0, 0.0])
        l6o = oracle.fof6d_halo(up, box.vel, m, np.ones(len(m), np.uint8), prm, use_lv=1, use_vt=0)
        assert np.array_equal(got[m], l6o), (h, len(m))
