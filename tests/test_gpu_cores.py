"""Core search (Sec. 2.3, Eq. coreloop) on the GPU vs the oracle, bit-exact: per halo the
oracle runs the same loop with the GPU's sigma_v (the lengths are inputs of the loop), so
the cores, their labels and levels must agree."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
SIGMA = 8  # VR_H_SIGMA


@pytest.fixture(scope="module")
def ctx():
    from paper_1902_01010_gb300 import Context

    return Context(0)


def _check(ctx, pos_np, vel_np, lab3_np, lab6_np, lx, nsearch_min=160, **kw):
    from paper_1902_01010_gb300 import CoreParams, Params

    P = Params.default(nsearch_min=nsearch_min)
    cp = CoreParams.default(**kw)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = ctx.core_search(dev(pos_np), dev(vel_np), dev(lab3_np.astype(np.int32)),
                          None if lab6_np is None else dev(lab6_np.astype(np.int32)), lx, 1.25,
                          P, cp)
    ctx.sync()
    core, lev = out["core"].cpu().numpy(), out["level"].cpu().numpy()
    hs = out["halos"][: out["nhalo"]].cpu().numpy()
    ecore = np.full(len(pos_np), -1, np.int32)
    elev = np.full(len(pos_np), -1, np.int32)
    off, mem = oracle.halos(lab3_np, 20)
    ncores = 0
    okw = dict(ax=cp.alpha_x, av=cp.alpha_v, n_loop=cp.n_loop, f_c=cp.f_c, an=cp.alpha_n)
    for h in range(len(off) - 1):
        m = mem[off[h]:off[h + 1]]
        if len(m) < nsearch_min:
            continue
        c, l, nc = oracle.core_search_halo(oracle.unwrap(pos_np, m), vel_np, m,
                                           None if lab6_np is None else lab6_np[m], lx,
                                           1.25 * hs[h, SIGMA], **okw)
        ecore[m], elev[m] = c, l
        ncores += nc
    assert np.array_equal(core, ecore) and np.array_equal(lev, elev)
    assert out["ncores"] == ncores
    return core, lev, out["ncores"]


@pytest.mark.parametrize("name", ["c32", "m64"])
def test_boxes_match_oracle(ctx, name):
    box = synth.named(name)
    lab3 = oracle.fof3d(box.pos, box.link_d2)
    lx = 0.2 * synth.mean_spacing(box.n)
    core, lev, nc = _check(ctx, box.pos, box.vel, lab3, None, lx)
    assert nc > 0 and (core >= 0).sum() > 0


def test_with_substructure_and_factors(ctx):
    box = synth.named("c32")
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    lab3, l6 = lab.cpu().numpy(), out["label6"].cpu().numpy()
    lx = 0.2 * synth.mean_spacing(box.n)
    _check(ctx, box.pos, box.vel, lab3, l6, lx)
    _check(ctx, box.pos, box.vel, lab3, l6, lx, alpha_x=0.7, alpha_v=0.9, n_loop=8, f_c=0.01,
           alpha_n=1.1)
    core, lev, nc = _check(ctx, box.pos, box.vel, lab3, l6, lx, n_loop=0)
    assert nc == 0 and (core == -1).all()


def test_two_blobs(ctx):
    rng = np.random.default_rng(8)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3) * 500
    nb = len(g)
    pos = np.vstack([g + 100000, g + 100000 + [3500, 0, 0]]).astype(np.int32)
    vel = np.vstack([rng.normal(0, 0.3, size=(nb, 3)) + [200, 0, 0],
                     rng.normal(0, 0.3, size=(nb, 3)) - [200, 0, 0]]).astype(np.float32)
    core, lev, nc = _check(ctx, pos, vel, np.zeros(2 * nb, np.int32), None, 700.0)
    assert nc == 2 and (core[:nb] == 0).all() and (lev[:nb] == 1).all()
    assert (core[nb:] == nb).all() and (lev[nb:] == 0).all()
