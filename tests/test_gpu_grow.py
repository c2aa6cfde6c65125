"""Two-stage linking (Sec. 2.2) on the GPU vs the oracle, bit-exact: the oracle grows
the GPU's stage-1 groups with the GPU's ell and per-halo parameters (the inputs of
vr_grow_groups), so the relaxed links, the attachments and the joins must agree."""
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


BOXES = {}


def _stage1(ctx, name):
    if name not in BOXES:
        box = synth.named(name)
        pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
        lab = ctx.fof3d(pos, box.link_d2)
        out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
        ctx.sync()
        BOXES[name] = (box, pos, vel, lab, out)
    return BOXES[name]


def _grow(ctx, name, **kw):
    from paper_1902_01010_gb300 import GrowParams

    box, pos, vel, lab, out = _stage1(ctx, name)
    hs = out["halos"][: out["nhalo"]].contiguous()
    l6 = out["label6"].clone()
    ctx.grow_groups(pos, vel, out["ell"], lab, hs, l6, grow=GrowParams.default(**kw))
    ctx.sync()
    return box, lab.cpu().numpy(), out, hs.cpu().numpy(), l6.cpu().numpy()


@pytest.mark.parametrize("name", ["c32", "m64"])
def test_defaults_match_oracle(ctx, name):
    box, lab3, out, hs, got = _grow(ctx, name)
    l6 = out["label6"].cpu().numpy()
    exp = oracle.two_stage(box.pos, box.vel, lab3, out["ell"].cpu().numpy(), l6, hs)
    assert np.array_equal(got, exp)
    assert (got >= 0).sum() > (l6 >= 0).sum()  # the relaxed pass grows the groups


@pytest.mark.parametrize("kw", [dict(gamma_ell=1.2, gamma_x=1.5, gamma_vr=1.5, gamma_theta=2.0),
                                dict(f_merge=0.0), dict(f_merge=10.0), dict(gamma_x=3.0)])
def test_factors_match_oracle(ctx, kw):
    box, lab3, out, hs, got = _grow(ctx, "c32", **kw)
    g = tuple(kw.get(k, d) for k, d in (("gamma_ell", 1.0), ("gamma_x", 2.0), ("gamma_vr", 1.0),
                                        ("gamma_theta", 1.0)))
    exp = oracle.two_stage(box.pos, box.vel, lab3, out["ell"].cpu().numpy(),
                           out["label6"].cpu().numpy(), hs, gam=g, f_merge=kw.get("f_merge", 0.25))
    assert np.array_equal(got, exp), kw


def test_gamma_one_is_identity(ctx):
    _, _, out, _, got = _grow(ctx, "m64", gamma_ell=1.0, gamma_x=1.0, gamma_vr=1.0, gamma_theta=1.0)
    assert np.array_equal(got, out["label6"].cpu().numpy())


def test_bad_factors_rejected(ctx):
    from paper_1902_01010_gb300 import GrowParams, VrError

    box, pos, vel, lab, out = _stage1(ctx, "c32")
    hs = out["halos"][: out["nhalo"]].contiguous()
    for kw in (dict(gamma_x=0.0), dict(f_merge=-1.0), dict(gamma_theta=6.0)):
        with pytest.raises(VrError) as e:
            ctx.grow_groups(pos, vel, out["ell"], lab, hs, out["label6"].clone(),
                            grow=GrowParams.default(**kw))
        assert e.value.code == 1
