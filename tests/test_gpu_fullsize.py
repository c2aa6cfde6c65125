"""The 512^3 clustered box (134M particles, the benchmark's workload) and the 1024^3 box
(1.07B particles) through the benchmark's calls and launch form: vr_fof3d, then
vr_find_substructure batched, default parameters. The oracle cannot run a whole box, so
it checks sampled outputs one by one (group members are gathered on the GPU):

  - 3D groups. A sampled group G is recomputed by the oracle's FOF over every particle
    within the linking length of G's bounding box (periodic). That set holds every
    particle linked to a member of G, so G is the true group iff the oracle's component
    of G's minimum member inside the set is exactly G; its label must be that minimum.
    Sampled: halos of several sizes and the groups of random particles.
  - f_l of sampled members of sampled halos (oracle.velden_one): 1e-4 relative.
  - R of sampled searched halos, the oracle's background fed the GPU f_l:
    |dR| <= 1e-4 max(1, |R|); the fit fed the GPU R: R-bar, sigma_R to 1e-7; ell.
  - 6D labels of those halos, the oracle's linker fed the GPU outlier mask and rows:
    bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import named_box

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

L = 1 << 21


@pytest.fixture(scope="module", params=["c512", "c1024"])
def run(request):
    from paper_1902_01010_gb300 import Context

    ctx = Context(0)
    box = named_box(request.param)
    pos, vel = torch.from_numpy(box.pos).cuda(), torch.from_numpy(box.vel).cuda()
    lab = ctx.fof3d(pos, box.link_d2)
    out = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0)
    ctx.sync()
    res = dict(box=box, pos_t=pos, lab_t=lab, label=lab.cpu().numpy(), nhalo=out["nhalo"])
    for k in ("f_l", "R", "ell", "label6"):
        res[k] = out[k].cpu().numpy()
    res["hs"] = out["halos"][: out["nhalo"]].cpu().numpy()
    del out, lab, vel
    yield res
    res.clear()
    del ctx, pos
    torch.cuda.empty_cache()


def _members(r, label):
    """Particles with 3D label `label`, in increasing index order."""
    return torch.nonzero(r["lab_t"] == int(label)).squeeze(1).cpu().numpy().astype(np.int32)


def _neighbourhood(pos_t, members, pos_np, link_d2):
    """Indices of every particle within sqrt(link_d2) of the bounding box of `members`
    (minimum image per axis), selected on the GPU."""
    a = pos_np[members[0]].astype(np.int64)
    up = a + (((pos_np[members].astype(np.int64) - a) + L // 2) % L - L // 2)
    lo, hi = up.min(0), up.max(0)
    c = (lo + hi) // 2
    w = (hi - lo) // 2 + int(np.ceil(np.sqrt(link_d2))) + 2
    keep = torch.ones(pos_t.shape[0], dtype=torch.bool, device=pos_t.device)
    for ax in range(3):
        d = (pos_t[:, ax].to(torch.int64) - int(c[ax]) + L // 2) % L - L // 2
        keep &= d.abs() <= int(w[ax])
    return torch.nonzero(keep).squeeze(1).cpu().numpy()


def _check_group(r, g_members):
    box = r["box"]
    nb = _neighbourhood(r["pos_t"], g_members, box.pos, box.link_d2)
    assert np.isin(g_members, nb).all()
    sub = oracle.fof3d(box.pos[nb], box.link_d2)
    m0 = np.flatnonzero(nb == g_members.min())[0]
    comp = nb[sub == sub[m0]]
    assert np.array_equal(np.sort(comp), np.sort(g_members)), (len(comp), len(g_members))
    assert (r["label"][g_members] == g_members.min()).all()


def test_3d_groups_sampled(run):
    hs = run["hs"]
    sizes = hs[:, 1]
    rng = np.random.default_rng(3)
    labels = []
    # halos of every size class up to ~60k members (the oracle FOF of a neighbourhood
    # costs about 10 us per particle), and the groups of 20 random particles
    for lo_s, hi_s, k in ((20, 160, 6), (160, 5000, 6), (5000, 60000, 3)):
        idx = np.flatnonzero((sizes >= lo_s) & (sizes < hi_s))
        labels += [int(hs[h, 0]) for h in rng.choice(idx, size=min(k, len(idx)), replace=False)]
    labels += [int(run["label"][i]) for i in rng.choice(len(run["label"]), 20, replace=False)]
    big = 0
    for lab in sorted(set(labels)):
        g = _members(run, lab)
        _check_group(run, g)
        big = max(big, len(g))
    assert big >= 5000
    # the halo table lists exactly the groups of >= 20 members, in label order
    cnt = torch.bincount(run["lab_t"].to(torch.int64), minlength=run["lab_t"].shape[0])
    big_labels = torch.nonzero(cnt >= 20).squeeze(1).cpu().numpy()
    assert np.array_equal(big_labels, hs[:, 0].astype(np.int64))
    assert np.array_equal(cnt[big_labels].cpu().numpy(), hs[:, 1].astype(np.int64))
    del cnt


def _sample_halos(r, rng, nmax):
    sizes = r["hs"][:, 1]
    searched = np.flatnonzero((r["hs"][:, 2] == 1) & (sizes <= nmax))
    pick = list(rng.choice(searched, size=min(10, len(searched)), replace=False))
    pick += list(searched[np.argsort(sizes[searched])[-2:]])
    return sorted(set(int(h) for h in pick))


def test_substructure_stages_sampled(run):
    box = run["box"]
    rng = np.random.default_rng(4)
    nflags = 0
    for h in _sample_halos(run, rng, 150000):
        hs = run["hs"][h]
        m = _members(run, hs[0])
        assert hs[0] == m[0] and hs[1] == len(m)
        up = oracle.unwrap(box.pos, m)
        # f_l, member by member
        for k in rng.choice(len(m), 8, replace=False):
            ref = oracle.velden_one(up, box.vel, m, int(k))
            assert abs(run["f_l"][m[k]] - ref) <= 1e-4 * ref, (h, k, run["f_l"][m[k]], ref)
        # R with the GPU f_l
        R_ref, _, _ = oracle.background_halo(up, box.vel, m, run["f_l"][m].astype(np.float64))
        Rg = run["R"][m].astype(np.float64)
        assert np.array_equal(np.isnan(Rg), np.isnan(R_ref))
        fin = np.isfinite(R_ref)
        assert (np.abs(Rg[fin] - R_ref[fin]) / np.maximum(1.0, np.abs(R_ref[fin]))).max() <= 1e-4
        # fit with the GPU R, then ell
        fit = oracle.ell_fit(Rg)
        assert abs(hs[3] - fit[0]) <= 1e-7 * max(1.0, abs(fit[0]))
        assert abs(hs[4] - fit[1]) <= 1e-7 * fit[1]
        e = (Rg - hs[3]) / hs[4]
        assert np.allclose(run["ell"][m], e, rtol=1e-6, atol=1e-6, equal_nan=True)
        # 6D labels with the GPU mask and rows
        cand = (run["ell"][m].astype(np.float64) >= 2.5).astype(np.uint8)
        prm = np.array([hs[9], hs[10], hs[5], hs[6], hs[7]])
        ref6 = oracle.fof6d_halo(up, box.vel, m, cand, prm)
        assert np.array_equal(run["label6"][m], ref6), h
        nflags += int((ref6 >= 0).sum())
    assert nflags > 0
