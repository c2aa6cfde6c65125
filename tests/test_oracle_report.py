"""Host logic of the oracle-side report used by the benchmark's CPU-baseline leg:
stratified sampling, the whole-box extrapolation, the flip band and the search for 6D
predicates near their thresholds (no GPU)."""
import math

import numpy as np

import oracle
import synth
from oracle import report


def test_stratified_sample_draws_per_bin():
    rng = np.random.default_rng(0)
    sizes = np.concatenate([np.full(50, 30), np.full(10, 500), np.full(3, 2000)])
    pick = report.stratified(sizes, rng, ((20, 160, 6), (160, 1000, 6), (1000, 5000, 4),
                                          (5000, 12000, 2)))
    s = sizes[pick]
    assert (s == 30).sum() == 6 and (s == 500).sum() == 6 and (s == 2000).sum() == 3


def test_extrapolation_model():
    samples = [{"n": n, "t": {"velden": 2e-8 * n * n, "background": 1e-6 * n,
                              "fit_link": 1e-6 * n if n >= 160 else 0.0}} for n in
               (50, 400, 2000, 9000)]
    samples[0]["t"]["background"] = 0.0
    sizes = np.array([50, 400, 2000, 9000, 100000])
    ext = report.extrapolate(10 ** 6, sizes, samples, 5e-6)
    assert math.isclose(ext["a_fl"], 2e-8, rel_tol=1e-12)
    assert math.isclose(ext["b_rest"], 2e-6, rel_tol=1e-12)
    want = 2e-8 * (sizes.astype(float) ** 2).sum() + 2e-6 * sizes[1:].sum() + 5.0
    assert math.isclose(ext["seconds"], want, rel_tol=1e-12)
    assert math.isclose(ext["particles_per_s"], 1e6 / want, rel_tol=1e-12)


def _halo():
    box = synth.named("c32")
    lab = oracle.fof3d(box.pos, box.link_d2)
    off, mem = oracle.halos(lab, 20)
    sizes = np.diff(off)
    h = int(np.argmax(sizes))
    return box, mem[off[h]:off[h + 1]]


def test_compare_halo_identical_and_perturbed():
    box, m = _halo()
    o = report.run_halo(box.pos, box.vel, m, box.lx_sub)
    same = report.compare_halo(m, dict(o), o)
    assert same["f_l_max_rel"] == 0 and same["R_max_rel"] == 0 and same["flips"] == []
    assert same["label6_differs"] == 0
    # move R by 1e-4 and sigma_R by 1e-5 relative: flags flip only inside the band
    g = dict(o)
    g["R"] = o["R"] + 1e-4
    g["sig"] = o["sig"] * (1 + 1e-5)
    g["ell"] = (g["R"] - g["rbar"]) / g["sig"]
    r = report.compare_halo(m, g, o)
    want_band = 1.01 * (1e-4 / o["sig"] + 2.5 * o["sig"] * 1e-5 / o["sig"]) + 1e-6
    assert math.isclose(r["band"], want_band, rel_tol=1e-6)
    assert all(f["within_band"] for f in r["flips"])
    # a planted flip far from the threshold is reported outside the band
    k = int(np.nanargmax(o["ell"]))
    g["ell"] = g["ell"].copy()
    g["ell"][k] = 0.0
    r = report.compare_halo(m, g, o)
    far = [f for f in r["flips"] if f["particle"] == int(m[k])]
    assert far and not far[0]["within_band"]


def test_near_threshold_pairs_finds_exact_boundary():
    # two candidates with dx2/lx2 = 0.5 and dv2/lv2 = 0.5 exactly: q = 1
    up = np.array([[0, 0, 0], [4, 0, 0], [1000, 0, 0]], np.int64)
    vel = np.array([[10, 0, 0], [10, 2, 0], [10, 50, 0]], np.float32)
    m = np.arange(3, dtype=np.int32)
    prm = np.array([32.0, 8.0, 0.0, 0.0, 0.0])
    r = report.near_threshold_pairs(up, vel, m, np.ones(3, np.uint8), prm)
    assert r["q"] == 1 and r["pairs"][0]["kind"] == "q"
    assert (r["pairs"][0]["i"], r["pairs"][0]["j"]) == (0, 1)
    prm2 = prm.copy()
    prm2[0] = 32.0 * (1 + 1e-9)
    assert report.near_threshold_pairs(up, vel, m, np.ones(3, np.uint8), prm2)["q"] == 0


def test_fof_subcube_labels_are_the_oracle_fof_of_the_subset():
    box = synth.named("c32")
    sel, lab, t = report.fof_subcube(box.pos, box.link_d2, side_div=2)
    assert np.all(box.pos[sel] < (1 << 20))
    assert np.array_equal(lab, oracle.fof3d(box.pos[sel], box.link_d2)) and t >= 0
