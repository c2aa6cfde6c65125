"""Seeded synthetic particle boxes (inputs only; none of the halo finder's arithmetic).

The boxes stand in for the N-body snapshots the paper analyses (its Table 2 runs are
not available): periodic boxes on a 2^21 integer lattice per axis, NFW hosts with
Plummer subhalos, Gaussian velocities and a uniform background. ``synth.c`` holds the
recipe; this module compiles it on first use and returns numpy arrays.

Both the CUDA library's tests/bench and the oracle consume these arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

LATTICE = 1 << 21
SEED0 = 1902010100


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (OpenMP; portable flags, no -march)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
            )
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_box.restype = ctypes.c_int64
        lib.synth_box.argtypes = [
            ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_void_p,
        ]
        lib.synth_hosts_total.restype = ctypes.c_int64
        lib.synth_hosts_total.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double]
        _lib = lib
    return _lib


@dataclass
class Box:
    """One synthetic box: particle data plus the linking parameters that go with it."""

    name: str
    n: int
    pos: np.ndarray       # int32 [n,3], lattice units in [0, 2^21)
    vel: np.ndarray       # float32 [n,3], km/s
    host_id: np.ndarray   # int32 [n], generating host (-1 = background)
    sub_id: np.ndarray    # int32 [n], generating subhalo (-1 = none)
    nhost: int
    link_d2: int          # 3D FOF: link iff d^2 < link_d2 (b = 0.2 of the mean spacing)
    lx_sub: float         # substructure spatial linking length, 0.1 mean spacing (lattice units)


def link_d2_for(n: int, b_num: int = 1, b_den: int = 5) -> int:
    """Smallest integer T with d^2 < T  <=>  d < b * 2^21 / N^(1/3), for N = m^3.

    (b * 2^21 / m)^2 = b_num^2 2^42 / (b_den^2 m^2) is never an integer for the
    configurations used (b = 1/5), so T = floor(.) + 1 exactly.
    """
    m = round(n ** (1.0 / 3.0))
    if m ** 3 != n:
        # non-cubic N: use the real mean spacing
        ell = (b_num / b_den) * LATTICE / n ** (1.0 / 3.0)
        return int(np.floor(ell * ell)) + 1
    num = b_num * b_num * (1 << 42)
    den = b_den * b_den * m * m
    return num // den + 1


def mean_spacing(n: int) -> float:
    return LATTICE / n ** (1.0 / 3.0)


def make_box(kind: int, n: int, seed: int, *, nhost: int = 8, frac_halo: float = 0.4,
             size_lo: float = 20.0, size_hi: float = 1e6, conc_lo: float = 4.0,
             conc_hi: float = 15.0, sigma_host: float = 100.0, sigma_bg: float = 30.0,
             name: str = "custom") -> Box:
    lib = _load()
    pos = np.empty((n, 3), np.int32)
    vel = np.empty((n, 3), np.float32)
    hid = np.empty(n, np.int32)
    sid = np.empty(n, np.int32)
    nh = lib.synth_box(n, kind, seed, nhost, frac_halo, size_lo, size_hi, conc_lo, conc_hi,
                       sigma_host, sigma_bg, pos.ctypes.data, vel.ctypes.data, hid.ctypes.data,
                       sid.ctypes.data)
    if nh < 0:
        raise ValueError("synth_box rejected its arguments")
    return Box(name, n, pos, vel, hid, sid, int(nh), link_d2_for(n), 0.1 * mean_spacing(n))


def small_clustered(n: int = 32768, seed: int = SEED0) -> Box:
    """32^3 particles, 10 Mpc/h: 8 NFW hosts (c = 8, 500-5000 particles), two Plummer
    subhalos of 5% host mass each at a 2 sigma_host bulk offset, sigma_host 100 km/s,
    uniform background at 30 km/s."""
    return make_box(0, n, seed, nhost=8, size_lo=500, size_hi=5000, conc_lo=8.0, conc_hi=8.0,
                    sigma_host=100.0, sigma_bg=30.0, name=f"clustered_{n}")


def mass_function_box(n: int, seed: int) -> Box:
    """40% of the particles in NFW hosts with dN/dM ~ M^-1.9 on [20, 1e6], c in [4, 15],
    sigma_host = 100 km/s (n_h/1000)^(1/3), power-law Plummer subhalos (~10% of host mass),
    uniform background at 30 km/s."""
    return make_box(1, n, seed, frac_halo=0.4, size_lo=20, size_hi=1e6, conc_lo=4.0,
                    conc_hi=15.0, sigma_host=100.0, sigma_bg=30.0, name=f"massfn_{n}")


def prelabelled_halos(nhost: int, seed: int, size_hi: float = 4e6):
    """`nhost` pre-labelled halos and no background: NFW hosts with dN/dM ~ M^-1.9 on
    [20, size_hi], c in [4, 15], sigma_host = 100 km/s (n_h/1000)^(1/3), power-law
    Plummer subhalos, placed at random in the 2^21 lattice box (they may overlap: the
    labels, not the positions, say which halo a particle belongs to). Returns (box,
    label) with label = the minimum particle index of each particle's halo, the form of
    the 3D FOF labels."""
    n = int(_load().synth_hosts_total(seed, nhost, 20.0, size_hi))
    lib = _load()
    pos = np.empty((n, 3), np.int32)
    vel = np.empty((n, 3), np.float32)
    hid = np.empty(n, np.int32)
    sid = np.empty(n, np.int32)
    nh = lib.synth_box(n, 2, seed, nhost, 1.0, 20.0, size_hi, 4.0, 15.0, 100.0, 30.0,
                       pos.ctypes.data, vel.ctypes.data, hid.ctypes.data, sid.ctypes.data)
    if nh != nhost:
        raise ValueError("synth_box rejected its arguments")
    first = np.full(nhost, n, np.int64)
    np.minimum.at(first, hid, np.arange(n, dtype=np.int64))
    label = first[hid].astype(np.int32)
    box = Box(f"prelabelled_{nhost}", n, pos, vel, hid, sid, nhost, link_d2_for(n),
              0.1 * mean_spacing(n))
    return box, label


def named(name: str, replica: int = 0) -> Box:
    """The standard workloads: 32^3 clustered, 256^3 / 512^3 / 1024^3 mass-function boxes,
    and m<k> = a k^3 mass-function box. `replica` > 0 draws an independent box of the same
    kind (another seed)."""
    r = 100000 * replica
    if name == "c32":
        return small_clustered(32 ** 3, SEED0 + 0 + r)
    if name == "c256":
        return mass_function_box(256 ** 3, SEED0 + 1 + r)
    if name == "c512":
        return mass_function_box(512 ** 3, SEED0 + 2 + r)
    if name == "c1024":
        return mass_function_box(1024 ** 3, SEED0 + 4 + r)
    if name.startswith("m") and name[1:].isdigit():
        m = int(name[1:])
        return mass_function_box(m ** 3, SEED0 + 10 + m + r)
    raise KeyError(name)
