"""Launch shapes of the batched form (vr_autotune, vr_tuning_force): every f_l and 6D
linker shape gives bit-identical outputs, and the tuner measures each halo-size bin once
on the caller's data and keeps the fastest shape."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def box_and_labels():
    from paper_1902_01010_gb300 import Context

    ctx = Context(0)
    box = synth.named("m64")
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    ctx.sync()
    return box, pos, vel, lab


def _run(ctx, box, pos, vel, lab):
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    return {k: (v[: out["nhalo"]] if k == "halos" else v).cpu().numpy()
            for k, v in out.items() if k != "nhalo"}


def test_every_shape_gives_identical_outputs(box_and_labels):
    from paper_1902_01010_gb300 import Context

    box, pos, vel, lab = box_and_labels
    ctx = Context(0)
    nv = len(ctx.tuning_report()["f_l"]["shapes"])
    nl = len(ctx.tuning_report()["link6"]["warps"])
    ref = _run(ctx, box, pos, vel, lab)
    assert (ref["label6"] >= 0).any() and np.isfinite(ref["f_l"]).any()
    for vs in range(nv):
        for ls in range(nl):
            ctx.tuning_force(vs, ls)
            got = _run(ctx, box, pos, vel, lab)
            for k in ("f_l", "R", "ell", "halos", "label6"):
                assert np.array_equal(got[k], ref[k], equal_nan=True), (vs, ls, k)
    ctx.tuning_force(-1, -1)


def test_autotune_measures_once_and_keeps_the_fastest(box_and_labels):
    from paper_1902_01010_gb300 import Context

    box, pos, vel, lab = box_and_labels
    ctx = Context(0)
    ref = _run(ctx, box, pos, vel, lab)
    rep0 = ctx.tuning_report()
    assert rep0["f_l"]["chosen"] == [0, 0, 0] and rep0["link6"]["chosen"] == 0
    ctx.autotune(True)
    got = _run(ctx, box, pos, vel, lab)  # measures every shape, same outputs
    for k in ref:
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    rep = ctx.tuning_report()
    sizes = ref["halos"][:, 1]
    meas = rep["f_l"]["measured"]
    # exactly the bins that hold halos are measured
    for k, (lo, hi) in enumerate(((65536, 1 << 31), (4096, 65536), (256, 4096))):
        has = bool(((sizes > lo) & (sizes <= hi)).any())
        assert (min(meas[k]) > 0) == has, (k, meas[k])
        if has:
            assert meas[k][rep["f_l"]["chosen"][k]] == min(meas[k])
    assert min(rep["link6"]["measured"]) > 0
    assert rep["link6"]["measured"][rep["link6"]["chosen"]] == min(rep["link6"]["measured"])
    again = _run(ctx, box, pos, vel, lab)  # tuned: no new measurement, same outputs
    assert ctx.tuning_report()["f_l"]["measured"] == meas
    for k in ref:
        assert np.array_equal(again[k], ref[k], equal_nan=True), k
    ctx.autotune(False)
    assert ctx.tuning_report()["f_l"]["chosen"] == [0, 0, 0]
