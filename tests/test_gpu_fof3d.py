"""3D FOF (Sec. 2.1, Eq. fof3d) on the GPU vs the oracle: labels must be bit-identical."""
import numpy as np
import pytest
import torch

import oracle
from helpers import named_box, oracle_labels
import synth

pytestmark = pytest.mark.gpu

L = 1 << 21


@pytest.fixture(scope="module")
def ctx():
    from paper_1902_01010_gb300 import Context

    return Context(0)


def _run(ctx, pos, T):
    p = torch.from_numpy(np.ascontiguousarray(pos, np.int32)).cuda()
    lab = ctx.fof3d(p, T)
    ctx.sync()
    return lab.cpu().numpy()


def _clustered(n, seed, nclump=6, spread=3000):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, L, size=(nclump, 3))
    which = rng.integers(0, nclump + 1, size=n)
    pos = rng.integers(0, L, size=(n, 3))
    inc = which < nclump
    pos[inc] = ctr[which[inc]] + rng.normal(0, spread, size=(inc.sum(), 3)).astype(np.int64)
    return (pos % L).astype(np.int32)


def test_small_box_bit_exact(ctx):
    box = synth.named("c32")
    assert np.array_equal(_run(ctx, box.pos, box.link_d2), oracle.fof3d(box.pos, box.link_d2))


@pytest.mark.parametrize("seed,T", [(1, 1200 ** 2), (2, 3000 ** 2), (3, 20000 ** 2), (4, 1)])
def test_clustered_sets(ctx, seed, T):
    pos = _clustered(20000, seed)
    assert np.array_equal(_run(ctx, pos, T), oracle.fof3d(pos, T))


def test_wrap_and_degenerate(ctx):
    rng = np.random.default_rng(7)
    pts = [np.array([cx, cy, cz]) + rng.normal(0, 300, size=(500, 3)).astype(np.int64)
           for cx in (0, L // 2) for cy in (0, L // 2) for cz in (0, L // 2)]
    pos = (np.concatenate(pts) % L).astype(np.int32)
    pos[:50] = pos[0]  # coincident particles
    for T in (900 ** 2, 1, 2, (1 << 19) ** 2):
        assert np.array_equal(_run(ctx, pos, T), oracle.fof3d(pos, T)), T


def test_tiny_and_empty(ctx):
    assert _run(ctx, np.array([[5, 5, 5]], np.int32), 10).tolist() == [0]
    pos = np.array([[L - 2, 0, 0], [3, 0, 0], [100, 100, 100]], np.int32)
    assert _run(ctx, pos, 26).tolist() == [0, 0, 2]
    assert _run(ctx, pos, 25).tolist() == [0, 1, 2]
    from paper_1902_01010_gb300 import Context  # n = 0 is a no-op
    c = Context(0)
    out = c.fof3d(torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 100)
    assert out.numel() == 0


def test_bad_arguments(ctx):
    from paper_1902_01010_gb300 import VrError

    p = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(VrError):
        ctx.fof3d(p, 0)
    with pytest.raises(VrError):
        ctx.fof3d(p, (1 << 38) + 1)


def test_mass_function_box_64cubed(ctx):
    box = synth.named("m64")
    assert np.array_equal(_run(ctx, box.pos, box.link_d2), oracle.fof3d(box.pos, box.link_d2))


@pytest.mark.slow
def test_256cubed_bit_exact(ctx):
    box = named_box("c256")
    got = _run(ctx, box.pos, box.link_d2)
    ref = oracle_labels("c256")
    assert np.array_equal(got, ref)
