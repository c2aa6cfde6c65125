"""The allocation-free 3D FOF entry point (vr_fof3d_noalloc) against vr_fof3d.

vr_fof3d_noalloc exists for callers that cannot allocate device memory (it takes no
context and no workspace; its scratch is a static device array inside the library).
Called through the C ABI on the current device, it must return exactly the labels of
vr_fof3d, on two calls in a row (the second call reuses the static array as the first
left it). This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

MAX_N = 131072


def _entry():
    from paper_1902_01010_gb300 import lib

    L = lib()
    f = L.vr_fof3d_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _call(f, pos, link_d2):
    n = pos.shape[0]
    out = torch.full((n,), -7, dtype=torch.int32, device=pos.device)
    st = f(ctypes.c_void_p(pos.data_ptr()), n, int(link_d2), ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, out.cpu().numpy()


def test_noalloc_matches_fof3d_twice():
    from paper_1902_01010_gb300 import Context

    f = _entry()
    ctx = Context(0)
    for name, box in (("c32", synth.named("c32")), ("m48", synth.named("m48"))):
        assert box.n <= MAX_N
        pos = torch.from_numpy(box.pos).cuda()
        ref = ctx.fof3d(pos, box.link_d2)
        ctx.sync()
        ref = ref.cpu().numpy()
        for call in range(2):
            st, got = _call(f, pos, box.link_d2)
            assert st == 0, (name, call, st)
            assert np.array_equal(got, ref), (name, call)


def test_noalloc_alternating_inputs_and_limits():
    f = _entry()
    a = synth.named("c32")
    b = synth.named("m40")
    pa, pb = torch.from_numpy(a.pos).cuda(), torch.from_numpy(b.pos).cuda()
    sa1 = _call(f, pa, a.link_d2)
    sb = _call(f, pb, b.link_d2)
    sa2 = _call(f, pa, a.link_d2)
    assert sa1[0] == sb[0] == sa2[0] == 0
    assert np.array_equal(sa1[1], sa2[1])
    # sizes above the stated maximum are rejected before any work
    big = torch.zeros((MAX_N + 1, 3), dtype=torch.int32, device="cuda")
    st, out = _call(f, big, 100)
    assert st == 1 and (out == -7).all()


def test_noalloc_at_the_stated_maximum():
    """n exactly VR_FOF3D_NOALLOC_MAX_N: the FOF scratch for that size fits the static array,
    and the labels equal vr_fof3d's, twice in a row."""
    from paper_1902_01010_gb300 import Context

    f = _entry()
    ctx = Context(0)
    box = synth.mass_function_box(MAX_N, synth.SEED0 + 77)
    assert box.n == MAX_N
    pos = torch.from_numpy(box.pos).cuda()
    ref = ctx.fof3d(pos, box.link_d2)
    ctx.sync()
    ref = ref.cpu().numpy()
    assert len(np.unique(ref)) < MAX_N  # some groups formed
    for call in range(2):
        st, got = _call(f, pos, box.link_d2)
        assert st == 0, (call, st)
        assert np.array_equal(got, ref), call

