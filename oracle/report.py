"""Oracle-side sampling, timing and comparison -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and bench.py's CPU-baseline and reference legs use this
module. It runs the FP64 oracle (oracle.c) on bounded samples of a box, times each
stage, extrapolates the oracle's whole-box rate from those timings, and compares the
oracle's outputs with another pipeline's outputs on the same particles:

  - per halo, both pipelines independent (Sec. 2.2: f_l, R, the fit of Eq. skewgaus,
    ell of Eq. ell, the links of Eq. linkingcriteria): the largest f_l and R errors, the
    errors of the fitted R-bar and sigma_R, every particle whose outlier flag
    (ell >= ell_th) differs between the two, with both ells, and the band of ell inside
    which such a flip is explained by the measured R, R-bar and sigma_R differences;
  - the 6D predicates (Eq. linkingcriteria b-d with the term of Eq. fof6d) within a
    relative 1e-12 of their thresholds among a halo's link candidates.

Nothing here feeds a product path: the CUDA library never imports it.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import (background_halo, ell_fit, fof3d, fof6d_halo, halo_frame, unwrap,
               velden_halo, velden_one)

LATTICE = 1 << 21


def stratified(sizes, rng, bins=((20, 160, 6), (160, 1000, 6), (1000, 5000, 4),
                                  (5000, 12000, 2))):
    """Indices of a size-stratified sample: k halos drawn (seeded) from each size bin
    [lo, hi) of `sizes`."""
    pick = []
    for lo, hi, k in bins:
        idx = np.flatnonzero((sizes >= lo) & (sizes < hi))
        if len(idx):
            pick += [int(i) for i in rng.choice(idx, size=min(k, len(idx)), replace=False)]
    return sorted(set(pick))


def run_halo(pos, vel, m, lx_sub, alpha_lv=1.0, nse=256, nv=32, nsearch_min=160,
             ell_th=2.5, f_cell=0.01, ncell_min=100):
    """The oracle pipeline on one halo (members m, increasing particle index), stage by
    stage as or_pipeline runs it. Returns outputs in member order and stage seconds."""
    t = {}
    t0 = time.perf_counter()
    up = unwrap(pos, m)
    fl = velden_halo(up, vel, m, nse, nv)
    t1 = time.perf_counter()
    t["velden"] = t1 - t0
    fr = halo_frame(vel, m)
    out = dict(f_l=fl, R=np.full(len(m), np.nan), ell=np.full(len(m), np.nan),
               label6=np.full(len(m), -1, np.int32), rbar=math.nan, sig=math.nan,
               frame=fr, prm=None)
    if len(m) >= nsearch_min:
        R, _, _ = background_halo(up, vel, m, fl, f_cell, ncell_min)
        t2 = time.perf_counter()
        fit = ell_fit(R)
        e = (R - fit[0]) / fit[1]
        cand = (e >= ell_th).astype(np.uint8)
        prm = np.array([lx_sub * lx_sub, (alpha_lv * fr[3]) ** 2, fr[0], fr[1], fr[2]])
        l6 = fof6d_halo(up, vel, m, cand, prm)
        t3 = time.perf_counter()
        t["background"] = t2 - t1
        t["fit_link"] = t3 - t2
        out.update(R=R, ell=e, label6=l6, rbar=fit[0], sig=fit[1], prm=prm)
    else:
        t["background"] = t["fit_link"] = 0.0
    out["t"] = t
    return out


def fof_subcube(pos, link_d2, side_div=8, corner=0):
    """The oracle's 3D FOF on the particles of one sub-cube of side 2^21 / side_div
    (corner index `corner` along each axis). Returns (particle indices, labels in those
    indices' numbering, seconds)."""
    w = LATTICE // side_div
    lo = corner * w
    sel = np.flatnonzero(np.all((pos >= lo) & (pos < lo + w), axis=1))
    t0 = time.perf_counter()
    lab = fof3d(pos[sel], link_d2)
    return sel, lab, time.perf_counter() - t0


def extrapolate(n_box, sizes, samples, fof_s_per_particle, nsearch_min=160):
    """Whole-box oracle seconds from sampled stage times: f_l costs a N_H^2 (every member
    ranks every other member), the other stages b N_H (searched halos) and the 3D FOF
    c per particle of the box. a and b are medians over the sampled halos of >= 1000
    and >= nsearch_min members (all sampled halos when none qualify)."""
    ns = np.array([s["n"] for s in samples], np.float64)
    tv = np.array([s["t"]["velden"] for s in samples])
    tb = np.array([s["t"]["background"] + s["t"]["fit_link"] for s in samples])
    big = ns >= 1000
    a = float(np.median((tv / ns ** 2)[big if big.any() else slice(None)]))
    srch = ns >= nsearch_min
    b = float(np.median((tb / ns)[srch])) if srch.any() else 0.0
    sizes = np.asarray(sizes, np.float64)
    t_fl = a * float((sizes ** 2).sum())
    t_rest = b * float(sizes[sizes >= nsearch_min].sum())
    t_fof = fof_s_per_particle * n_box
    total = t_fl + t_fof + t_rest
    return dict(seconds=total, particles_per_s=n_box / total, a_fl=a, b_rest=b,
                c_fof=fof_s_per_particle, seconds_fl=t_fl, seconds_fof=t_fof,
                seconds_rest=t_rest)


def _rel(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    fin = np.isfinite(a) & np.isfinite(b)
    if not fin.any():
        return 0.0
    return float((np.abs(a[fin] - b[fin]) / np.maximum(np.abs(b[fin]), floor)).max())


def compare_halo(m, gpu, orc, ell_th=2.5):
    """Independent-pipeline comparison of one searched halo. gpu: dict of per-member
    arrays f_l, R, ell, label6 and scalars rbar, sig; orc: run_halo's output.

    The flip band: ell = (R - R-bar) / sigma_R, so to first order a particle's ell moves
    by at most (max |dR| + |dR-bar|) / sigma_R + ell_th |d sigma_R| / sigma_R near the
    threshold; a flag may flip only for particles whose oracle ell lies within that band
    of ell_th (times 1.01 for the second-order terms, plus 1e-6 for ell stored in FP32)."""
    fin = np.isfinite(orc["R"]) & np.isfinite(gpu["R"])
    dR = float(np.abs(gpu["R"][fin] - orc["R"][fin]).max()) if fin.any() else 0.0
    drb = abs(gpu["rbar"] - orc["rbar"])
    dsg = abs(gpu["sig"] - orc["sig"])
    band = 1.01 * ((dR + drb) / orc["sig"] + ell_th * dsg / orc["sig"]) + 1e-6
    fg = gpu["ell"] >= ell_th
    fo = orc["ell"] >= ell_th
    flips = []
    for k in np.flatnonzero(fg != fo):
        flips.append(dict(particle=int(m[k]), ell_oracle=float(orc["ell"][k]),
                          ell_gpu=float(gpu["ell"][k]), R_oracle=float(orc["R"][k]),
                          R_gpu=float(gpu["R"][k]),
                          within_band=bool(abs(orc["ell"][k] - ell_th) <= band)))
    return dict(
        n=int(len(m)),
        f_l_max_rel=_rel(gpu["f_l"], orc["f_l"]),
        R_max_rel=_rel(gpu["R"], orc["R"], 1.0),
        rbar_abs=float(drb), sigma_abs=float(dsg),
        sigma_rel=float(dsg / orc["sig"]) if orc["sig"] else math.nan,
        band=float(band), flips=flips,
        label6_membership_differs=int(((gpu["label6"] >= 0) != (orc["label6"] >= 0)).sum()),
        label6_differs=int((gpu["label6"] != orc["label6"]).sum()),
    )


def near_threshold_pairs(up, vel, m, cand, prm, v_ratio=2.0, theta_op=0.1 * math.pi,
                         tol=1e-12, cap=50, max_cand=6000):
    """Candidate pairs of one halo whose 6D predicates sit within a relative `tol` of
    their thresholds, evaluated in FP64 in the predicate's fixed order (Eq.
    linkingcriteria b-d, the dv term of Eq. fof6d): q = dx2/lx2 + dv2/lv2 against 1,
    s_i against V_r^2 s_j, dot^2 against cos^2 Theta_op s_i s_j. Returns counts and the
    first `cap` such pairs (particle indices). Halos with more than max_cand candidates
    are checked on the first max_cand candidates."""
    c = np.flatnonzero(cand)[:max_cand]
    res = dict(candidates=int(len(c)), q=0, v_ratio=0, theta=0, pairs=[])
    if len(c) < 2:
        return res
    x = up[c].astype(np.int64)
    v = vel[m[c]].astype(np.float64)
    u = v - np.asarray(prm[2:5], np.float64)
    s = (u[:, 0] * u[:, 0] + u[:, 1] * u[:, 1]) + u[:, 2] * u[:, 2]
    vr2 = v_ratio * v_ratio
    cos2 = math.cos(theta_op) ** 2
    for i0 in range(0, len(c), 512):
        i1 = min(len(c), i0 + 512)
        d = x[i0:i1, None, :] - x[None, :, :]
        dx2 = (d * d).sum(-1).astype(np.float64)
        dv = v[i0:i1, None, :] - v[None, :, :]
        dv2 = (dv[..., 0] * dv[..., 0] + dv[..., 1] * dv[..., 1]) + dv[..., 2] * dv[..., 2]
        q = dx2 / prm[0] + dv2 / prm[1]
        si, sj = s[i0:i1, None], s[None, :]
        r_vr = si / (vr2 * sj)
        dot = (u[i0:i1, None, 0] * u[None, :, 0] + u[i0:i1, None, 1] * u[None, :, 1]) \
            + u[i0:i1, None, 2] * u[None, :, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            r_th = (dot * dot) / ((cos2 * si) * sj)
        upper = np.arange(i0, i1)[:, None] < np.arange(len(c))[None, :]
        for name, val in (("q", q), ("v_ratio", r_vr), ("theta", r_th)):
            near = upper & np.isfinite(val) & (np.abs(val - 1.0) <= tol)
            if name == "theta":
                near &= dot >= 0
            ii, jj = np.nonzero(near)
            res[name] += int(len(ii))
            for a, b in zip(ii[:cap], jj[:cap]):
                if len(res["pairs"]) < cap:
                    res["pairs"].append(dict(kind=name, i=int(m[c[i0 + a]]), j=int(m[c[b]]),
                                             value=float(val[a, b])))
    return res


def sampled_members_fl(up, vel, m, ks, nse=256, nv=32):
    """Oracle f_l of sampled members ks of one halo (each one on its own)."""
    return np.array([velden_one(up, vel, m, int(k), nse, nv) for k in ks])
