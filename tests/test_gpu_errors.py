"""Error paths that the host observes, each followed by a normal call on the same context
(include/vr.h conventions): an undersized workspace is refused before any launch; a halo
that spans half the box or more, a halo of more than 2^22 members and a two-stage-linking
count table that fills up are reported as VR_ERR_UNSUPPORTED. No case faults the GPU: the
kernels record a status word and return."""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

VR_ERR_WORKSPACE_TOO_SMALL = 3
VR_ERR_UNSUPPORTED = 6


@pytest.fixture(scope="module")
def ctx():
    from paper_1902_01010_gb300 import Context

    return Context(0)


@pytest.fixture(scope="module")
def reference(ctx):
    """The 32^3 box through 3D FOF and the substructure search before any error."""
    import synth

    box = synth.named("c32")
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    return box, lab.cpu().numpy(), out["label6"].cpu().numpy(), out["f_l"].cpu().numpy()


def _still_works(ctx, reference):
    box, lab0, l60, fl0 = reference
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    assert np.array_equal(lab.cpu().numpy(), lab0)
    assert np.array_equal(out["label6"].cpu().numpy(), l60)
    assert np.array_equal(out["f_l"].cpu().numpy(), fl0, equal_nan=True)


def test_workspace_too_small_is_refused_before_any_launch(ctx, reference):
    from paper_1902_01010_gb300 import Params, lib
    from paper_1902_01010_gb300.vr import _ptr, _stream, alloc_outputs

    box = reference[0]
    L = lib()
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = torch.full((box.n,), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    launches = L.vr_launch_count
    launches.restype = ctypes.c_int64
    n0 = launches()
    st = L.vr_fof3d(ctx.h, _ptr(pos), box.n, int(box.link_d2), _ptr(lab), _ptr(ws), 1024,
                    _stream(None))
    assert st == VR_ERR_WORKSPACE_TOO_SMALL
    assert launches() == n0  # refused before any kernel
    assert (lab.cpu().numpy() == -7).all()
    P = Params.default()
    out = alloc_outputs(box.n, P, pos.device)
    nh = ctypes.c_int64()
    lab0 = torch.from_numpy(reference[1]).cuda()
    st = L.vr_find_substructure(ctx.h, _ptr(pos), _ptr(vel), box.n, _ptr(lab0), float(box.lx_sub),
                                1.0, ctypes.byref(P), 1, _ptr(out["f_l"]), _ptr(out["R"]),
                                _ptr(out["ell"]), _ptr(out["label6"]), _ptr(out["halos"]),
                                ctypes.byref(nh), _ptr(ws), 1024, _stream(None))
    assert st == VR_ERR_WORKSPACE_TOO_SMALL
    assert launches() == n0
    assert b"workspace" in L.vr_last_error(ctx.h)
    _still_works(ctx, reference)


def test_halo_spanning_half_the_box(ctx, reference):
    """A chain of 40 particles 2^15 apart along x, linked by a linking length just above
    the step: one group spanning 39 * 2^15 > 2^20 lattice units, more than half the box,
    so no single periodic image of it exists."""
    from paper_1902_01010_gb300 import VrError

    n = 40
    pos = np.zeros((n, 3), np.int32)
    pos[:, 0] = np.arange(n) * (1 << 15)
    pos[:, 1:] = 5000
    vel = np.random.default_rng(0).normal(0, 50, (n, 3)).astype(np.float32)
    p, v = torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda()
    lab = ctx.fof3d(p, (1 << 30) + 1)
    ctx.sync()
    assert (lab.cpu().numpy() == 0).all()  # one group
    with pytest.raises(VrError) as e:
        ctx.find_substructure(p, v, lab, 1000.0, 1.0)
        ctx.sync()
    assert e.value.code == VR_ERR_UNSUPPORTED and "half the box" in str(e.value)
    _still_works(ctx, reference)


def test_halo_above_2_pow_22_members(ctx, reference):
    """2^22 + 1 particles with one 3D label: the halo table refuses it (the local index of a
    member has 22 bits in the f_l keys)."""
    from paper_1902_01010_gb300 import VrError

    n = (1 << 22) + 1
    g = torch.Generator(device="cuda").manual_seed(5)
    pos = torch.randint(0, 1 << 18, (n, 3), dtype=torch.int32, device="cuda", generator=g)
    vel = torch.randn((n, 3), dtype=torch.float32, device="cuda", generator=g)
    lab = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(VrError) as e:
        ctx.velden(pos, vel, lab)
        ctx.sync()
    assert e.value.code == VR_ERR_UNSUPPORTED and "2^22" in str(e.value)
    del pos, vel, lab
    torch.cuda.empty_cache()
    _still_works(ctx, reference)


def _link(ui, uj, vr2, cos2):
    """The relaxed speed-ratio and opening-angle criteria (Eq. linkingcriteria c, d) in the
    halo frame; positions coincide and the velocity length is unbounded here."""
    si, sj = ui @ ui, uj @ uj
    dot = ui @ uj
    return si > 0 and sj > 0 and si <= vr2 * sj and sj <= vr2 * si and dot >= 0 and \
        dot * dot >= (cos2 * si) * sj


def test_two_stage_link_table_full(ctx, reference):
    """Ten untagged outliers that do not link one another, each linked to all of 128
    tagged particles in 128 different groups: 1280 distinct (component, group) link counts
    for a table of 1024 entries (twice the 138 candidates, rounded up to the minimum)."""
    from paper_1902_01010_gb300 import GrowParams, Params, VrError
    from paper_1902_01010_gb300.vr import HALO_COLS

    P = Params.default()
    vr2 = P.v_ratio ** 2
    cos2 = math.cos(P.theta_op) ** 2
    nt, dirs = 128, []
    c17, s17 = math.cos(math.radians(17)), math.sin(math.radians(17))
    for k in range(5):  # five directions 17 degrees off x, about 20 degrees apart
        a = 2 * math.pi * k / 5
        dirs.append(np.array([c17, s17 * math.cos(a), s17 * math.sin(a)]))
    unt = [d * m for d in dirs for m in (50.5, 101.5)]  # speeds more than a factor 2 apart
    ut = np.array([100.0, 0.0, 0.0])
    for i in range(len(unt)):
        assert _link(unt[i], ut, vr2, cos2)
        for j in range(i + 1, len(unt)):
            assert not _link(unt[i], unt[j], vr2, cos2)
    nu = len(unt)
    n = nu + nt
    vel = np.array(unt + [ut] * nt, np.float32)
    pos = np.full((n, 3), 7000, np.int32)
    ell = np.full(n, 3.0, np.float32)
    label6 = np.array([-1] * nu + list(range(nu, n)), np.int32)  # tagged: one group each
    hs = np.zeros((1, HALO_COLS), np.float64)
    hs[0, :3] = (0, n, 1)
    hs[0, 9], hs[0, 10] = 1.0e6, 1.0e12  # lx2, lv2: every pair passes the 6D distance term
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lab3 = torch.zeros(n, dtype=torch.int32, device="cuda")
    l6 = t(label6)
    with pytest.raises(VrError) as e:
        ctx.grow_groups(t(pos), t(vel), t(ell), lab3, t(hs), l6, P, GrowParams.default())
        ctx.sync()
    assert e.value.code == VR_ERR_UNSUPPORTED and "link-count table" in str(e.value)
    _still_works(ctx, reference)


def test_log_levels(ctx, reference, capfd):
    """vr_set_log_level: level 2 prints one line per 3D FOF / substructure call, level 1
    prints an error as it is recorded, level 0 prints nothing; results are unchanged."""
    box = reference[0]
    pos = torch.from_numpy(box.pos).cuda()
    capfd.readouterr()
    ctx.log_level(2)
    lab = ctx.fof3d(pos, box.link_d2)
    ctx.sync()
    err = capfd.readouterr().err
    assert f"vr: vr_fof3d n={box.n} status 0" in err
    assert np.array_equal(lab.cpu().numpy(), reference[1])
    ctx.log_level(1)
    with pytest.raises(Exception):
        ctx.fof3d(pos, 0)  # link_d2 below 1
    err = capfd.readouterr().err
    assert "vr: link_d2 must be in" in err and "vr_fof3d n=" not in err
    ctx.log_level(0)
    with pytest.raises(Exception):
        ctx.fof3d(pos, 0)
    assert capfd.readouterr().err == ""
    from paper_1902_01010_gb300 import VrError

    with pytest.raises(VrError):
        ctx.log_level(3)
    _still_works(ctx, reference)
