"""Shared test helpers: run the oracle per halo and compare with tolerances."""
import functools

import numpy as np

import oracle
import synth


@functools.lru_cache(maxsize=2)
def named_box(name):
    """synth.named(name), drawn once per test process."""
    return synth.named(name)


@functools.lru_cache(maxsize=2)
def oracle_labels(name):
    """Oracle 3D FOF labels of a named box, computed once per test process (the 256^3
    box takes minutes)."""
    box = named_box(name)
    lab = oracle.fof3d(box.pos, box.link_d2)
    lab.setflags(write=False)
    return lab


def oracle_fl(pos, vel, label, nse=256, nv=32, nmin=20):
    """Oracle f_l for every halo member (NaN elsewhere)."""
    n = len(label)
    out = np.full(n, np.nan)
    off, mem = oracle.halos(label, nmin)
    for h in range(len(off) - 1):
        m = mem[off[h]:off[h + 1]]
        up = oracle.unwrap(pos, m)
        out[m] = oracle.velden_halo(up, vel, m, nse, nv)
    return out


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def assert_close_nan(got, ref, rtol, floor=0.0, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(ref)), f"{what}: NaN pattern differs"
    fin = np.isfinite(ref)
    e = rel_err(got[fin], ref[fin], floor)
    bad = np.flatnonzero(e > rtol)
    assert len(bad) == 0, f"{what}: {len(bad)} of {fin.sum()} beyond {rtol}; worst {e.max():.3e}"
    return e.max() if len(e) else 0.0
