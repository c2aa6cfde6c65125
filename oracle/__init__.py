"""ORACLE — test infrastructure only.

Plain single-threaded FP64 C restatement of the VELOCIraptor substructure hot path
(Elahi et al. 2019, Sec. 2.1-2.2), used to check the CUDA library. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may load it. It shares
no code with the CUDA library; both consume the arrays written by ``synth``.

The C source is ``oracle.c`` (compiled with -O2 -ffp-contract=off, so no fused
multiply-add changes its rounding). This module compiles it on first use and wraps
each entry point for numpy arrays.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_HS = 12  # per-halo row of pipeline(): see HALO_COLS
HALO_COLS = ("label", "nh", "searched", "Rbar", "sigR", "vfx", "vfy", "vfz", "sigma_host",
             "lx2", "lv2", "ncells")


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                                   "-shared", "-std=gnu11", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Search parameters with the paper's defaults (Table 1; Table A1)."""

    _fields_ = [
        ("nse", ctypes.c_int32), ("nv", ctypes.c_int32), ("f_cell", ctypes.c_double),
        ("ncell_min", ctypes.c_int32), ("nmin", ctypes.c_int32), ("nsearch_min", ctypes.c_int32),
        ("ell_th", ctypes.c_double), ("v_ratio", ctypes.c_double), ("theta_op", ctypes.c_double),
        ("use_lv", ctypes.c_int32), ("use_vr_theta", ctypes.c_int32),
        ("split_rule", ctypes.c_int32), ("fit_nbins_min", ctypes.c_int32),
        ("fit_nbins_max", ctypes.c_int32), ("fit_iters", ctypes.c_int32),
    ]

    @classmethod
    def default(cls, **kw) -> "Params":
        p = cls(nse=256, nv=32, f_cell=0.01, ncell_min=100, nmin=20, nsearch_min=160,
                ell_th=2.5, v_ratio=2.0, theta_op=0.1 * math.pi, use_lv=1, use_vr_theta=1,
                split_rule=0, fit_nbins_min=10, fit_nbins_max=200, fit_iters=100)
        for k, v in kw.items():
            setattr(p, k, v)
        return p


def _lib_():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        sig = {
            "or_fof3d": (ctypes.c_int, [vp, i64, i64, vp]),
            "or_fof3d_brute": (ctypes.c_int, [vp, i64, i64, vp]),
            "or_halos": (i64, [vp, i64, i32, vp, vp]),
            "or_unwrap": (None, [vp, vp, i64, vp]),
            "or_velden_halo": (ctypes.c_int, [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp]),
            "or_velden_one": (dbl, [vp, vp, vp, i64, i64, ctypes.c_int, ctypes.c_int]),
            "or_knn_one": (i64, [vp, vp, i64, i64, ctypes.c_int, vp]),
            "or_ncell": (i64, [i64, dbl, i32]),
            "or_ln_fbg": (dbl, [vp, vp, vp]),
            "or_background_halo": (i64, [vp, vp, vp, i64, vp, dbl, i32, ctypes.c_int, vp, vp, vp,
                                          vp]),
            "or_ell_bins": (ctypes.c_int, [vp, i64, ctypes.c_int, ctypes.c_int, vp, vp]),
            "or_sg_fit": (None, [vp, i64, dbl, dbl, dbl, ctypes.c_int, vp]),
            "or_ell_fit": (ctypes.c_int, [vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]),
            "or_fof6d_halo": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, dbl, dbl, ctypes.c_int,
                                             ctypes.c_int, i32, vp]),
            "or_halo_frame": (None, [vp, vp, i64, vp]),
            "or_pipeline": (i64, [vp, vp, i64, i64, dbl, dbl, ctypes.POINTER(Params), vp, vp, vp,
                                  vp, vp, vp]),
            "or_ell_bar": (dbl, [dbl]),
            "or_field6d": (i64, [vp, vp, i64, vp, dbl, dbl, i32, vp, vp]),
            "or_clean_groups": (i64, [vp, vp, i64, dbl, dbl, i32]),
            "or_grow_halo": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp, dbl, dbl, dbl,
                                            ctypes.c_int, ctypes.c_int, vp, dbl, vp]),
            "or_core_search": (i64, [vp, vp, vp, i64, vp, dbl, dbl, dbl, dbl, ctypes.c_int,
                                     dbl, dbl, i32, vp, vp]),
            "or_core_assign": (ctypes.c_int, [vp, i64, vp, ctypes.c_int, ctypes.c_int, vp]),
            "or_core_grow": (i64, [vp, vp, vp, i64, vp, dbl, dbl, dbl, dbl, ctypes.c_int,
                                   dbl, dbl, i32, dbl, ctypes.c_int, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ------------------------------------------------------------------- wrappers

def fof3d(pos, link_d2: int, brute: bool = False) -> np.ndarray:
    """3D FOF labels (minimum index per group), Eq. fof3d."""
    pos = _c(pos, np.int32)
    n = pos.shape[0]
    lab = np.empty(n, np.int32)
    f = _lib_().or_fof3d_brute if brute else _lib_().or_fof3d
    rc = f(_p(pos), n, int(link_d2), _p(lab))
    if rc != 0:
        raise RuntimeError(f"oracle fof3d failed ({rc})")
    return lab


def halos(label, nmin: int):
    """(offsets[H+1], members) of groups with >= nmin members, members increasing."""
    label = _c(label, np.int32)
    n = label.shape[0]
    L = _lib_()
    H = L.or_halos(_p(label), n, nmin, None, None)
    if H < 0:
        raise ValueError("bad labels")
    off = np.empty(H + 1, np.int64)
    mem = np.empty(max(n, 1), np.int32)
    L.or_halos(_p(label), n, nmin, _p(off), _p(mem))
    return off, mem[: off[-1]].copy()


def unwrap(pos, members) -> np.ndarray:
    pos = _c(pos, np.int32)
    members = _c(members, np.int32)
    up = np.empty((members.shape[0], 3), np.int64)
    _lib_().or_unwrap(_p(pos), _p(members), members.shape[0], _p(up))
    return up


def velden_halo(upos, vel, members, nse=256, nv=32) -> np.ndarray:
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    out = np.empty(members.shape[0], np.float64)
    rc = _lib_().or_velden_halo(_p(upos), _p(vel), _p(members), members.shape[0], nse, nv, _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle velden failed ({rc})")
    return out


def velden_one(upos, vel, members, k: int, nse=256, nv=32) -> float:
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    return _lib_().or_velden_one(_p(upos), _p(vel), _p(members), members.shape[0], k, nse, nv)


def knn_one(upos, members, k: int, nse=256) -> np.ndarray:
    upos = _c(upos, np.int64)
    members = _c(members, np.int32)
    out = np.empty(min(nse, members.shape[0]), np.int32)
    m = _lib_().or_knn_one(_p(upos), _p(members), members.shape[0], k, nse, _p(out))
    return out[:m]


def ncell(nh: int, f_cell=0.01, ncell_min=100) -> int:
    return int(_lib_().or_ncell(nh, f_cell, ncell_min))


def ln_fbg(v, vbar, sig6) -> float:
    v = _c(v, np.float64)
    vbar = _c(vbar, np.float64)
    sig6 = _c(sig6, np.float64)
    return _lib_().or_ln_fbg(_p(v), _p(vbar), _p(sig6))


def background_halo(upos, vel, members, f_l, f_cell=0.01, ncell_min=100, split_rule=0,
                    boxes=False):
    """Returns (R [nh], leaf_of [nh], cell_stats [nleaves, 13]), plus the leaves'
    half-open regions [nleaves, 6] (lo[3], hi[3]) when boxes is set."""
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    f_l = _c(f_l, np.float64)
    nh = members.shape[0]
    R = np.empty(nh, np.float64)
    leaf = np.empty(nh, np.int32)
    cs = np.empty((max(nh, 1), 13), np.float64)
    lb = np.empty((max(nh, 1), 6), np.int64) if boxes else None
    nl = _lib_().or_background_halo(_p(upos), _p(vel), _p(members), nh, _p(f_l), f_cell,
                                    ncell_min, split_rule, _p(R), _p(leaf), _p(cs), _p(lb))
    if nl < 0:
        raise RuntimeError("oracle background failed")
    if boxes:
        return R, leaf, cs[:nl].copy(), lb[:nl].copy()
    return R, leaf, cs[:nl].copy()


def ell_bins(R, nbins_min=10, nbins_max=200):
    """(counts [nbins], (median, MAD', lo, width, nbins)); counts is empty when the
    values are degenerate."""
    R = _c(R, np.float64)
    cnt = np.zeros(max(nbins_max, 1), np.float64)
    meta = np.empty(5, np.float64)
    _lib_().or_ell_bins(_p(R), R.shape[0], nbins_min, nbins_max, _p(cnt), _p(meta))
    return cnt[: int(meta[4])].copy(), meta


def sg_fit(counts, lo: float, width: float, sigma0: float, iters=100) -> np.ndarray:
    """Fit of A f_SG to binned counts (bin b centred at lo + (b + 1/2) width):
    (Rbar, sigma_R, s, A)."""
    counts = _c(counts, np.float64)
    out = np.empty(4, np.float64)
    _lib_().or_sg_fit(_p(counts), counts.shape[0], float(lo), float(width), float(sigma0),
                      iters, _p(out))
    return out


def ell_fit(R, nbins_min=10, nbins_max=200, iters=100) -> np.ndarray:
    """(Rbar, sigma_R, s, A, lo, width, nbins, MAD')."""
    R = _c(R, np.float64)
    out = np.empty(8, np.float64)
    _lib_().or_ell_fit(_p(R), R.shape[0], nbins_min, nbins_max, iters, _p(out))
    return out


def fof6d_halo(upos, vel, members, cand, prm, v_ratio=2.0, theta_op=0.1 * math.pi, use_lv=1,
               use_vt=1, nmin=20) -> np.ndarray:
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    cand = _c(cand, np.uint8)
    prm = _c(prm, np.float64)
    out = np.empty(members.shape[0], np.int32)
    _lib_().or_fof6d_halo(_p(upos), _p(vel), _p(members), members.shape[0], _p(cand), _p(prm),
                          v_ratio, theta_op, use_lv, use_vt, nmin, _p(out))
    return out


def halo_frame(vel, members) -> np.ndarray:
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    out = np.empty(4, np.float64)
    _lib_().or_halo_frame(_p(vel), _p(members), members.shape[0], _p(out))
    return out


def field6d(pos, vel, label3, lx: float, alpha_v: float = 1.25, nmin: int = 20):
    """Field 6DFOF of the 3DFOF groups (Sec. 2.1, Eq. fof6d). Returns (label6, rows) with
    rows[h] = (label3, N_H, sigma_v, lx^2, lv^2) per group of >= nmin members."""
    pos = _c(pos, np.int32)
    vel = _c(vel, np.float32)
    label3 = _c(label3, np.int32)
    n = pos.shape[0]
    lab6 = np.empty(n, np.int32)
    rows = np.empty((n // max(nmin, 1) + 1, 5), np.float64)
    H = _lib_().or_field6d(_p(pos), _p(vel), n, _p(label3), float(lx), float(alpha_v), nmin,
                           _p(lab6), _p(rows))
    if H < 0:
        raise ValueError("bad labels")
    return lab6, rows[:H].copy()


def clean_groups(ell, label6, ell_th: float = 2.5, beta: float = 1.0, nmin: int = 20):
    """Significance cleaning of groups (Sec. 2.2, Eq. ellsig). Returns (label6, kept)."""
    ell = _c(ell, np.float64)
    lab = _c(label6, np.int32).copy()
    kept = _lib_().or_clean_groups(_p(ell), _p(lab), lab.shape[0], float(ell_th), float(beta),
                                   nmin)
    return lab, int(kept)


GROW_DEFAULTS = (1.0, 2.0, 1.0, 1.0)  # gamma_ell, gamma_x, gamma_vr, gamma_theta (Table A1)
F_MERGE = 0.25  # f_merge,th (Sec. 2.2)


def grow_halo(upos, vel, members, ell, lab1, prm, ell_th=2.5, v_ratio=2.0,
              theta_op=0.1 * math.pi, use_lv=1, use_vt=1, gam=GROW_DEFAULTS,
              f_merge=F_MERGE) -> np.ndarray:
    """Two-stage linking inside one halo (Sec. 2.2): relaxed growth of the stage-1
    groups lab1 and the merge threshold. ell, lab1 per member; members ascending."""
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    ell = _c(ell, np.float64)
    lab1 = _c(lab1, np.int32)
    prm = _c(prm, np.float64)
    g = _c(gam, np.float64)
    out = np.empty(members.shape[0], np.int32)
    _lib_().or_grow_halo(_p(upos), _p(vel), _p(members), members.shape[0], _p(ell), _p(lab1),
                         _p(prm), ell_th, v_ratio, theta_op, use_lv, use_vt, _p(g), f_merge,
                         _p(out))
    return out


def two_stage(pos, vel, label3, ell, label6, halo_rows, nmin=20, **kw) -> np.ndarray:
    """grow_halo over every searched halo of a box (rows as the halo table: label, N_H,
    searched, ..., vframe at 5-7, lx2 at 9, lv2 at 10). Returns the final labels."""
    out = np.asarray(label6, np.int32).copy()
    off, mem = halos(label3, nmin)
    for h in range(len(off) - 1):
        r = halo_rows[h]
        if r[2] == 0:
            continue
        m = mem[off[h]:off[h + 1]]
        prm = np.array([r[9], r[10], r[5], r[6], r[7]])
        out[m] = grow_halo(unwrap(pos, m), vel, m, np.asarray(ell, np.float64)[m],
                           np.asarray(label6, np.int32)[m], prm, **kw)
    return out


CORE_DEFAULTS = dict(ax=0.8, av=1.0, n_loop=5, f_c=0.02, an=1.2)  # Table 1, core search


def core_search_halo(upos, vel, members, lab6, lx, lv, ax=0.8, av=1.0, n_loop=5, f_c=0.02,
                     an=1.2, nmin=20):
    """Core search inside one halo (Sec. 2.3, Eq. coreloop). lab6 per member (None: no
    substructure). Returns (core label per member, level per member, number of cores)."""
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    nh = members.shape[0]
    l6 = None if lab6 is None else _c(lab6, np.int32)
    core = np.empty(nh, np.int32)
    lev = np.empty(nh, np.int32)
    nc = _lib_().or_core_search(_p(upos), _p(vel), _p(members), nh, _p(l6), float(lx), float(lv),
                                ax, av, n_loop, f_c, an, nmin, _p(core), _p(lev))
    return core, lev, int(nc)


def core_search(pos, vel, label3, label6, lx, alpha_v=1.25, nsearch_min=160, nmin=20, **kw):
    """core_search_halo over every halo with N_H >= nsearch_min, lv = alpha_v sigma_v
    (halo_frame). Returns (core, level) per particle."""
    n = len(pos)
    core = np.full(n, -1, np.int32)
    lev = np.full(n, -1, np.int32)
    off, mem = halos(label3, nmin)
    for h in range(len(off) - 1):
        m = mem[off[h]:off[h + 1]]
        if len(m) < nsearch_min:
            continue
        lv = alpha_v * halo_frame(vel, m)[3]
        c, l, _ = core_search_halo(unwrap(pos, m), vel, m,
                                   None if label6 is None else np.asarray(label6, np.int32)[m],
                                   lx, lv, nmin=nmin, **kw)
        core[m] = c
        lev[m] = l
    return core, lev


CORE_GROW_DEFAULTS = dict(beta_c=1.0, mode=2)  # Table 1 beta_C; Table A1 core growth mode


def core_assign(X, init, ncore, mode=2):
    """One core-growth assignment step (Eq. coredist; mode 0: scalar dispersions) of the
    phase-space rows X [n][6]: init[i] is the core seeded by row i or -1. Returns (core per
    row, number of cores with a positive-definite tensor)."""
    X = _c(X, np.float64)
    init = _c(init, np.int32)
    out = np.empty(len(init), np.int32)
    npd = _lib_().or_core_assign(_p(X), len(init), _p(init), int(ncore), int(mode), _p(out))
    return out, int(npd)


def core_grow_halo(upos, vel, members, lab6, lx, lv, ax=0.8, av=1.0, n_loop=5, f_c=0.02,
                   an=1.2, nmin=20, beta_c=1.0, mode=2):
    """Core search, core cleaning (Eq. coresig) and core growth (Eqs. coremeanphase,
    coredispphase, coredist) inside one halo (Sec. 2.3). Returns (core, level, grown, gap)
    per member and the number of cores kept; gap is the second smallest D^2 minus the
    smallest for members assigned by distance, NaN otherwise."""
    upos = _c(upos, np.int64)
    vel = _c(vel, np.float32)
    members = _c(members, np.int32)
    nh = members.shape[0]
    l6 = None if lab6 is None else _c(lab6, np.int32)
    core = np.empty(nh, np.int32)
    lev = np.empty(nh, np.int32)
    grown = np.empty(nh, np.int32)
    gap = np.empty(nh, np.float64)
    nk = _lib_().or_core_grow(_p(upos), _p(vel), _p(members), nh, _p(l6), float(lx), float(lv),
                              ax, av, n_loop, f_c, an, nmin, float(beta_c), int(mode), _p(core),
                              _p(lev), _p(grown), _p(gap))
    return core, lev, grown, gap, int(nk)


def core_grow(pos, vel, label3, label6, lx, alpha_v=1.25, nsearch_min=160, nmin=20, **kw):
    """core_grow_halo over every halo with N_H >= nsearch_min, lv = alpha_v sigma_v.
    Returns (core, level, grown, gap) per particle."""
    n = len(pos)
    core = np.full(n, -1, np.int32)
    lev = np.full(n, -1, np.int32)
    grown = np.full(n, -1, np.int32)
    gap = np.full(n, np.nan)
    off, mem = halos(label3, nmin)
    for h in range(len(off) - 1):
        m = mem[off[h]:off[h + 1]]
        if len(m) < nsearch_min:
            continue
        lv = alpha_v * halo_frame(vel, m)[3]
        c, l, g, d, _ = core_grow_halo(unwrap(pos, m), vel, m,
                                       None if label6 is None else np.asarray(label6, np.int32)[m],
                                       lx, lv, nmin=nmin, **kw)
        core[m], lev[m], grown[m], gap[m] = c, l, g, d
    return core, lev, grown, gap


def ell_bar(ell_th: float) -> float:
    return _lib_().or_ell_bar(ell_th)


def pipeline(pos, vel, link_d2: int, lx_sub: float, alpha_lv: float = 1.0, params=None):
    """Full oracle pass. Returns dict of per-particle arrays and the per-halo table."""
    pos = _c(pos, np.int32)
    vel = _c(vel, np.float32)
    n = pos.shape[0]
    P = params or Params.default()
    lab3 = np.empty(n, np.int32)
    fl = np.empty(n, np.float64)
    R = np.empty(n, np.float64)
    ell = np.empty(n, np.float64)
    lab6 = np.empty(n, np.int32)
    hs = np.empty((n // max(P.nmin, 1) + 1, OR_HS), np.float64)
    H = _lib_().or_pipeline(_p(pos), _p(vel), n, int(link_d2), lx_sub, alpha_lv, ctypes.byref(P),
                            _p(lab3), _p(fl), _p(R), _p(ell), _p(lab6), _p(hs))
    if H < 0:
        raise RuntimeError("oracle pipeline failed")
    return dict(label3=lab3, f_l=fl, R=R, ell=ell, label6=lab6, halos=hs[:H].copy())
