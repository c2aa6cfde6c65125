#!/usr/bin/env python3
"""Benchmark: particles/s of the VELOCIraptor hot path (3D FOF + f_l + background ratio
+ skew-Gaussian fit + 6D outlier linking) on a synthetic 512^3 clustered box, one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c512] [--form batched|plain] [--plain-steps P]
                    [--no-next-rows] [--no-cpu-baseline]

One step = vr_fof3d + vr_find_substructure over the whole box, inputs resident in HBM
(3.2 GB of positions and velocities, far above the 129 MB L2, so no flush is needed
between steps). Under torchrun (N > 1) every rank runs an independent replica on its own
box (weak scaling, no collective on the data path); `value` is all ranks' particles over
the slowest rank's time. Rank 0 prints one JSON line.

The headline runs the batched form (each stage one launch over all halos); the same
inputs are then timed in the plain form (each stage launched once per halo) and reported
under "plain_form". Field 6DFOF of the 3DFOF halos, the significance cleaning of the
step's outlier groups, their two-stage growth and the core search are timed afterwards on
the same box and reported under "next_rows" (outside the headline).

The CPU baseline (rank 0, after the timed region) runs the FP64 C oracle on one host core
over a bounded sample of the same box: its 3D FOF on one sub-cube (1/512 of the volume),
and its whole per-halo pipeline on a size-stratified sample of the GPU's halos. The
oracle's whole-box rate is extrapolated from those stage times (f_l costs a N_H^2 per
halo, the other stages b N_H, the FOF c per particle) and labelled as such. The same
sample gives the parity report: the oracle's outputs against the GPU's on those particles
(largest f_l and R errors, fit errors, every outlier flag that flips near ell_th with
the band that explains it, 6D predicates within 1e-12 of their thresholds, 3D groups of
the sub-cube), plus the whole 32^3 box through both pipelines.

--impl reference times the same oracle on the host cores: one step = its FOF on one
sub-cube plus its per-halo pipeline on a size-stratified sample of the generator's hosts,
and the line's value is the whole-box rate extrapolated from those stage times.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particles/s for 3DFOF+velden+6DFOF at 512^3, batched vs plain; % HBM roofline"
WORKLOADS = {
    "c512": "512^3 clustered box, 200 Mpc/h: 40% of particles in NFW hosts (dN/dM ~ M^-1.9 on "
            "[20, 1e6], c in [4, 15]) with power-law Plummer subhalos (~10% of host mass), "
            "uniform background; int32 2^21-lattice positions, FP32 Gaussian velocities; "
            "b = 0.2, N_se = 256, N_v = 32, f_cell = 0.01, ell_th = 2.5, l_x,S = 0.1 spacing, "
            "l_v = 1.0 sigma_host",
    "c256": "256^3 clustered box, 100 Mpc/h, same generator and parameters as the 512^3 box",
    "m160": "160^3 box (4.1M particles), same generator and parameters: small profiling case",
    "c1024": "1024^3 clustered box (1.07 B particles), 1 Gpc/h, same generator and parameters "
             "as the 512^3 box",
    "prelabelled": "batching form: 200,000 pre-labelled halos (NFW hosts with dN/dM ~ M^-1.9 on "
          "[20, 4e6], power-law Plummer subhalos, 92.7M particles, no background); "
          "substructure search only (f_l, background R, fit, 6D links; no 3D FOF), same "
          "search parameters",
}
CPU_SAMPLE_DESC = (
    "oracle (FP64 C, one host core) on a bounded sample of the same box: its 3D FOF on the "
    "sub-cube [0, 2^21/8)^3 (1/512 of the volume), and its per-halo pipeline (f_l, background "
    "R, fit, 6D links) on {nh} halos drawn per size bin ({bins}); whole-box rate EXTRAPOLATED "
    "from the measured stage times: f_l a N_H^2 per halo (every member ranks every other), the "
    "other stages b N_H, FOF c per particle, summed over the box's {nhalo} halos")
CPU_BINS = ((20, 160, 6), (160, 1000, 6), (1000, 5000, 4), (5000, 12000, 2))
REF_BINS = ((20, 160, 4), (160, 1000, 4), (1000, 5000, 3), (5000, 12000, 1))
TIMED_KERNELS = ("velden_big", "fof_link", "link6", "cells_build", "cells_build_big", "ell_fit", "ratio",
                 "halo_frame", "velden_small")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception as e:  # no nvidia-smi: report nothing
            log("clock sampling unavailable:", e)
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- peaks & roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic work of the dominant kernel (per query particle of a halo larger than N_se):
# N_se position distances (3 sub + 3 mul + 2 add) + N_se velocity differences (same) +
# selection of N_se out of the candidates and N_v out of N_se (one compare each) + the
# Epanechnikov sum over N_v (3 ops): 256*8 + 256*8 + 256 + 256 + 32*3 = 4,704 ALU ops.
VELDEN_OPS_PER_QUERY = 256 * 8 + 256 * 8 + 256 + 256 + 32 * 3
# DRAM bytes per query particle of k_velden_big from one ncu capture (dram__bytes_read.sum
# + dram__bytes_write.sum of one launch over its query particles); the kernel's traffic
# grows with its queries, so a full launch is this times its queries. None whenever the
# kernel has changed since the capture.
VELDEN_DRAM_BYTES_PER_QUERY = 3866411264 / 39635926
VELDEN_DRAM_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the three per-bin "
                      "k_velden_big launches of one 512^3 step (3.87 GB over 39,635,926 query "
                      "particles), times this step's query particles")
LANES_PER_SM = 128  # FP32/INT32 lanes per SM (4 partitions x 32)


def alu_peak_tops(sms, sm_mhz):
    """One 32-bit ALU operation per lane per clock: SMs x 128 lanes x SM clock."""
    return sms * LANES_PER_SM * sm_mhz * 1e6 / 1e12


def ncell_rule(nh, f_cell=0.01, ncell_min=100):
    nc = int(np.floor(f_cell * nh))
    if nc < ncell_min:
        nc = min(ncell_min, nh // 8)
    return max(nc, 1)


def algorithmic_bytes(n, sizes, nse=256, nsearch_min=160):
    """The method's minimum DRAM bytes per step by stage (per particle: 3D FOF 16 B,
    position + label; f_l 32 B per halo member, position, velocity, index, f_l; cells +
    moments 16 B per member per tree level + 24 B; R and ell 40 B and the 6D links 32 B
    per member of a searched halo), and the split of those bytes over the timed
    kernels."""
    sizes = np.asarray(sizes, np.int64)
    srch = sizes[sizes >= nsearch_min]
    levels = np.array([max(0, int(np.ceil(np.log2(h / ncell_rule(int(h)))))) for h in srch])
    cells = float(((16.0 * levels + 24.0) * srch).sum())
    big = sizes > nse
    nh, ns = float(sizes.sum()), float(srch.sum())
    stage = {"fof3d": 16.0 * n, "velden": 32.0 * nh, "cells": cells,
             "outlier_ratio": 40.0 * ns, "fof6d": 32.0 * ns}
    big_cells = srch >= 65536
    kern = {"fof_link": 16.0 * n, "velden_big": 32.0 * float(sizes[big].sum()),
            "velden_small": 32.0 * float(sizes[~big].sum()),
            "cells_build": float(((16.0 * levels + 24.0) * srch)[~big_cells].sum()),
            "cells_build_big": float(((16.0 * levels + 24.0) * srch)[big_cells].sum()),
            "ratio": 40.0 * ns, "ell_fit": 8.0 * ns, "link6": 32.0 * ns,
            "halo_frame": 12.0 * nh}
    return stage, kern


def reduce_over_ranks(ms, n_local, device=None):
    """(slowest rank's time, all ranks' particles) across the process group (identity
    without one). Replicas share nothing but this reduction."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(n_local)
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(n_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


# ------------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    import synth
    from paper_1902_01010_gb300 import Context, Params, lib

    L = lib()
    L.vr_timing_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.vr_timing_read.argtypes = [ctypes.c_void_p, ctypes.c_char_p,
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.vr_timing_reset.argtypes = [ctypes.c_void_p]
    L.vr_launch_count.restype = ctypes.c_int64

    t0 = time.time()
    prelab = args.workload == "prelabelled"  # pre-labelled halos: the step has no 3D FOF
    if prelab:
        box, lab_np = synth.prelabelled_halos(200000, synth.SEED0 + 3 + 100000 * rank)
    else:
        box = synth.named(args.workload, replica=rank)  # each rank: its own seeded box
    log(f"rank {rank}: generated {box.n} particles in {time.time() - t0:.1f}s")
    P = Params.default()
    ctx = Context(local)
    pos = torch.from_numpy(box.pos).to(dev)
    vel = torch.from_numpy(box.vel).to(dev)
    lab = torch.empty(box.n, dtype=torch.int32, device=dev)
    if prelab:
        lab.copy_(torch.from_numpy(lab_np))
    from paper_1902_01010_gb300.vr import alloc_outputs

    out = alloc_outputs(box.n, P, dev)
    batched = 1 if args.form == "batched" else 0
    stream = torch.cuda.current_stream(dev)

    def step():
        if not prelab:
            ctx.fof3d(pos, box.link_d2, label=lab)
        ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0, P, batched=batched, out=out)

    # launch shapes: the first warm-up step times every candidate shape per halo-size bin
    # on this machine and keeps the fastest (vr_autotune); the timed steps use the winners
    if args.autotune:
        ctx.autotune(True)
    for _ in range(args.warmup):
        step()
    ctx.sync()
    torch.cuda.synchronize(dev)
    tuning = ctx.tuning_report()

    # ---- timed region: device-resident inputs
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize(dev)
    L.vr_timing_enable(ctx.h, 1)
    L.vr_timing_reset(ctx.h)
    launches0 = L.vr_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = L.vr_launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    kern = {}
    for nm in TIMED_KERNELS:
        t = ctypes.c_double()
        c = ctypes.c_int64()
        L.vr_timing_read(ctx.h, nm.encode(), ctypes.byref(t), ctypes.byref(c))
        kern[nm] = (t.value, c.value)
    L.vr_timing_enable(ctx.h, 0)
    ctx.sync()
    ms_max, n_all = reduce_over_ranks(ms, box.n, dev)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    ms_per_step = ms_max / args.steps
    value = n_all / (ms_per_step / 1e3)

    # ---- end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hpos = torch.from_numpy(box.pos).pin_memory()
        hvel = torch.from_numpy(box.vel).pin_memory()
        hl3 = torch.empty(box.n, dtype=torch.int32).pin_memory()  # 3D labels: out, or in (pre-labelled)
        if prelab:
            hl3.copy_(torch.from_numpy(lab_np))
        hl6 = torch.empty(box.n, dtype=torch.int32).pin_memory()
        # the velocities (needed from the substructure search on) come in on a second
        # stream while the 3D FOF runs; the 3D labels go out on it during the search
        cs = torch.cuda.Stream(dev)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pos.copy_(hpos, non_blocking=True)
            if prelab:
                lab.copy_(hl3, non_blocking=True)
            with torch.cuda.stream(cs):
                vel.copy_(hvel, non_blocking=True)
                ev_vel = torch.cuda.Event()
                ev_vel.record(cs)
            if not prelab:
                ctx.fof3d(pos, box.link_d2, label=lab)
                ev_lab = torch.cuda.Event()
                ev_lab.record(stream)
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_lab)
                    hl3.copy_(lab, non_blocking=True)
            stream.wait_event(ev_vel)
            ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0, P, batched=batched, out=out)
            hl6.copy_(out["label6"], non_blocking=True)
            torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t1) / args.e2e_steps
        e2e = {"value": ws * box.n / dt, "unit": "particles/s",
               "h2d_bytes_per_step": int(hpos.numel() * 4 + hvel.numel() * 4
                                         + (hl3.numel() * 4 if prelab else 0)),
               "d2h_bytes_per_step": int(hl6.numel() * 4 + (0 if prelab else hl3.numel() * 4))}

    # ---- rows beyond the headline step, on the same box (timed separately, 3 calls each):
    #      field 6DFOF of the 3DFOF halos (Sec. 2.1), significance cleaning of the outlier
    #      groups the step produced (Sec. 2.2, Eq. ellsig), their two-stage growth with
    #      the merge threshold (Sec. 2.2), the core search (Sec. 2.3, Eq. coreloop) and the
    #      core search followed by core cleaning and growth (Sec. 2.3, Eqs. coresig, coredist)
    next_rows = None
    if args.next_rows and not prelab:
        lx = 0.2 * synth.mean_spacing(box.n)
        l6f = torch.empty(box.n, dtype=torch.int32, device=dev)
        halos_f = torch.empty((box.n // P.nmin + 1, 12), dtype=torch.float64, device=dev)
        l6c = out["label6"].clone()

        def field():
            ctx.fof6d_field(pos, vel, lab, lx, 1.25, P, label6=l6f, halos=halos_f)

        def clean():
            l6c.copy_(out["label6"])
            return ctx.clean_groups(out["ell"], l6c, P, 1.0)

        from paper_1902_01010_gb300 import GrowParams

        l6g = out["label6"].clone()
        hs_g = out["halos"][: out["nhalo"]].contiguous()
        gp = GrowParams.default()

        def grow():
            l6g.copy_(out["label6"])
            ctx.grow_groups(pos, vel, out["ell"], lab, hs_g, l6g, P, gp)

        core_out = {}

        def cores():
            core_out.update(ctx.core_search(pos, vel, lab, out["label6"], lx, 1.25, P,
                                            out=core_out or None))

        grow_out = {}

        def core_growth():
            grow_out.update(ctx.core_grow(pos, vel, lab, out["label6"], lx, 1.25, P,
                                          out=grow_out or None))

        field()
        clean()
        grow()
        cores()
        core_growth()
        ctx.sync()
        res = {}
        for name, f in (("field_6dfof", field), ("clean_groups", clean), ("two_stage_linking", grow),
                        ("core_search", cores), ("core_search_and_growth", core_growth)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(3):
                f()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            res[name] = {"ms": e0.elapsed_time(e1) / 3}
        ng = clean()
        a = l6f.cpu().numpy()
        res["field_6dfof"].update({"particles_per_s": box.n / (res["field_6dfof"]["ms"] / 1e3),
                                   "particles_in_6d_groups": int((a >= 0).sum()),
                                   "groups": int(len(np.unique(a[a >= 0]))),
                                   "alpha_v": 1.25, "l_x": "0.2 mean spacing"})
        res["clean_groups"].update({"groups_kept": int(ng),
                                    "groups_in": int(len(np.unique(
                                        out["label6"].cpu().numpy()[out["label6"].cpu().numpy() >= 0]))),
                                    "beta": 1.0})
        a6 = out["label6"].cpu().numpy()
        ag = l6g.cpu().numpy()
        res["two_stage_linking"].update({
            "particles_in_groups_before": int((a6 >= 0).sum()),
            "particles_in_groups_after": int((ag >= 0).sum()),
            "groups_before": int(len(np.unique(a6[a6 >= 0]))),
            "groups_after": int(len(np.unique(ag[ag >= 0]))),
            "gamma": [gp.gamma_ell, gp.gamma_x, gp.gamma_vr, gp.gamma_theta], "f_merge": gp.f_merge})
        cc = core_out["core"].cpu().numpy()
        res["core_search"].update({"cores": int(core_out["ncores"]),
                                   "particles_in_cores": int((cc >= 0).sum()),
                                   "params": "alpha_x,C 0.8, alpha_v,C 1.0, n_loop 5, f_C 0.02, "
                                             "alpha_N,C 1.2; l_x 0.2 spacing, l_v 1.25 sigma_v"})
        gg, gc = grow_out["grown"].cpu().numpy(), grow_out["core"].cpu().numpy()
        res["core_search_and_growth"].update({
            "cores_kept": int(grow_out["nkept"]), "particles_in_cores": int((gc >= 0).sum()),
            "particles_in_grown_cores": int((gg >= 0).sum()),
            "params": "core search as core_search; beta_C 1, growth mode 2 (tensors "
                      "recomputed per level)"})
        next_rows = res

    # ---- the other launch form on the same inputs: one launch per halo and stage
    plain = None
    if batched and args.plain_steps > 0:
        def step_plain():
            if not prelab:
                ctx.fof3d(pos, box.link_d2, label=lab)
            ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0, P, batched=0, out=out)

        # no separate warm-up: every kernel and buffer was already used by the batched steps
        ctx.sync()
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)
        l0 = L.vr_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.plain_steps):
            step_plain()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pl_launch = L.vr_launch_count() - l0
        pms, pn = reduce_over_ranks(e0.elapsed_time(e1), box.n, dev)
        pms /= args.plain_steps
        plain = {"value": pn / (pms / 1e3), "unit": "particles/s", "ms_per_step": pms,
                 "steps": args.plain_steps, "warmup": "the batched steps (same kernels and buffers)",
                 "gpu_launches_per_step": int(pl_launch // args.plain_steps),
                 "batched_speedup": pms / ms_per_step}

    if rank != 0:
        return
    # ---- roofline of the dominant kernel (device time inside the timed region)
    dom = max(kern, key=lambda k: kern[k][0])
    peaks, how = measured_peaks()
    hs_np = out["halos"][: out["nhalo"]].cpu().numpy()
    sizes = hs_np[:, 1].astype(np.int64)
    nq_big = float(sizes[sizes > P.nse].sum())
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    stage_b, kern_b = algorithmic_bytes(box.n, sizes, P.nse, P.nsearch_min)
    hbm = peaks["hbm_gbs"]
    roof = None
    if dom == "velden_big" and kern[dom][1] > 0:
        per_launch_ms = kern[dom][0] / kern[dom][1]
        ops = VELDEN_OPS_PER_QUERY * nq_big
        achieved = ops / (per_launch_ms / 1e3) / 1e12
        peak = alu_peak_tops(sms, sm_mhz)
        traffic = (VELDEN_DRAM_BYTES_PER_QUERY * nq_big if VELDEN_DRAM_BYTES_PER_QUERY else None)
        roof = {"kernel": "k_velden_big", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": VELDEN_DRAM_SOURCE,
                "peak_source": f"{sms} SMs (device) x {LANES_PER_SM} FP32/INT32 lanes x "
                               f"{sm_mhz:.0f} MHz (sm_max_mhz of {how} peaks): one 32-bit "
                               f"operation per lane per clock",
                "algorithmic": f"{VELDEN_OPS_PER_QUERY} ops x {int(nq_big)} query particles",
                "launch_ms": per_launch_ms,
                "hbm_achieved_gbs": kern_b["velden_big"] / (per_launch_ms / 1e3) / 1e9,
                "hbm_frac": kern_b["velden_big"] / (per_launch_ms / 1e3) / 1e9 / hbm}
    elif dom == "fof_link" and kern[dom][1] > 0:
        per_launch_ms = kern[dom][0] / kern[dom][1]
        achieved = 16.0 * box.n / (per_launch_ms / 1e3) / 1e9
        roof = {"kernel": "k_fof_link", "bound": "hbm", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "launch_ms": per_launch_ms}
    step_bytes = sum(stage_b.values())
    step_gbs = step_bytes / (ms_per_step / 1e3) / 1e9
    if roof is not None:
        roof["step_hbm"] = {"algorithmic_bytes": step_bytes, "by_stage": stage_b,
                            "achieved_gbs": step_gbs, "peak_gbs": hbm,
                            "hbm_frac": step_gbs / hbm, "peak_source": f"hbm_gbs of {how} peaks"}
    shares = {k: round(v[0] / max(ms, 1e-9), 4) for k, v in kern.items()}
    kernels = {}
    for k, (t_ms, nl) in kern.items():
        if nl <= 0:
            continue
        per = t_ms / nl
        gbs = kern_b.get(k, 0.0) / (per / 1e3) / 1e9
        kernels[k] = {"ms_per_launch": per, "share_of_step": shares[k],
                      "algorithmic_bytes": kern_b.get(k), "achieved_gbs": gbs,
                      "hbm_frac": gbs / hbm}

    cpu, parity = None, None
    if not args.no_cpu_baseline and not prelab:
        cpu, parity = cpu_leg(box, ctx, dev, lab, out, hs_np, P, args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64 and exact u32 distances, f32 f_l, f64 background/fit/links", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.workload, args.workload),
                   "n_particles": box.n, "halos": int(out["nhalo"]), "form": args.form,
                   "l2": "inputs 24 B/particle >> 129 MB L2; no flush between steps",
                   "parallelism": f"replicas x{ws}"},
        "hbm_frac": step_gbs / hbm,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "kernel_share_of_step": shares,
        "kernels": kernels,
        "plain_form": plain,
        "tuning": tuning,
        "next_rows": next_rows,
        "parity": parity,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- oracle arm
def _gpu_members(lab_t, label):
    """Particles with 3D label `label` (increasing index), selected on the GPU."""
    import torch

    return torch.nonzero(lab_t == int(label)).squeeze(1).cpu().numpy().astype(np.int32)


def _fof_subcube_parity(box, lab_t, sel, lab_o):
    """Groups of the oracle's FOF on a sub-cube whose members all lie more than one
    linking length inside it cannot link outside it, so each must be exactly a GPU 3D
    group: same members, labelled by their minimum index."""
    import torch

    L = 1 << 21
    w = L // 8
    reach = int(np.ceil(np.sqrt(box.link_d2))) + 1
    p = box.pos[sel].astype(np.int64)
    interior = np.all((p >= reach) & (p < w - reach), axis=1)
    gl = sel[lab_o]  # the oracle's labels as particle indices (its minimum member)
    comp_all_in = np.ones(len(sel), bool)
    # a component is checked when every member is interior
    bad_comp = np.unique(lab_o[~interior])
    comp_all_in[np.isin(lab_o, bad_comp)] = False
    idx = np.flatnonzero(comp_all_in)
    sel_t = torch.from_numpy(sel[idx].astype(np.int64)).to(lab_t.device)
    lg = lab_t[sel_t].cpu().numpy().astype(np.int64)
    cnt_t = torch.bincount(lab_t.to(torch.int64), minlength=lab_t.shape[0])
    sizes_g = cnt_t[torch.from_numpy(gl[idx].astype(np.int64)).to(lab_t.device)].cpu().numpy()
    del cnt_t
    sizes_o = np.bincount(lab_o[idx], minlength=len(sel))[lab_o[idx]]
    mism = int(((lg != gl[idx]) | (sizes_g != sizes_o)).sum())
    return {"particles": int(len(sel)), "particles_in_checked_groups": int(len(idx)),
            "groups_checked": int(len(np.unique(lab_o[idx]))), "mismatched_particles": mism}


def _halo_gpu(out, members_t, hs_row):
    g = {k: out[k][members_t].cpu().numpy() for k in ("f_l", "R", "ell", "label6")}
    for k in ("f_l", "R", "ell"):
        g[k] = g[k].astype(np.float64)
    g["rbar"], g["sig"] = float(hs_row[3]), float(hs_row[4])
    return g


def cpu_leg(box, ctx, dev, lab_t, out, hs_np, P, wname):
    """The oracle timed on a bounded sample of this box (rank 0, after the timed region),
    with the parity report of the same sample. Returns (cpu_baseline, parity)."""
    import torch

    import oracle
    from oracle import report

    t_start = time.perf_counter()
    rng = np.random.default_rng(20190201)
    sizes = hs_np[:, 1].astype(np.int64)
    th = P.ell_th
    # ---- 3D FOF on one sub-cube
    sel, lab_o, t_fof = report.fof_subcube(box.pos, box.link_d2, side_div=8)
    fof_par = _fof_subcube_parity(box, lab_t, sel, lab_o)
    # ---- per-halo pipeline, both sides independent
    pick = report.stratified(sizes, rng, CPU_BINS)
    samples, halos = [], []
    for h in pick:
        row = hs_np[h]
        m = _gpu_members(lab_t, row[0])
        mt = torch.from_numpy(m.astype(np.int64)).to(dev)
        o = report.run_halo(box.pos, box.vel, m, box.lx_sub, 1.0, P.nse, P.nv, P.nsearch_min, th)
        samples.append({"n": len(m), "t": o["t"]})
        g = _halo_gpu(out, mt, row)
        rec = {"label": int(row[0]), "n": int(len(m)),
               "f_l_max_rel": report._rel(g["f_l"], o["f_l"])}
        if row[2] == 1:
            rec.update(report.compare_halo(m, g, o, th))
            # stage by stage: the oracle fed the GPU's inputs (R from the GPU f_l, the fit
            # from the GPU R, the links from the GPU mask and halo row): labels must match
            up = oracle.unwrap(box.pos, m)
            Rs, _, _ = oracle.background_halo(up, box.vel, m, g["f_l"])
            rec["R_max_rel_gpu_fl"] = report._rel(g["R"], Rs, 1.0)
            fit = oracle.ell_fit(g["R"])
            rec["rbar_rel_gpu_R"] = abs(g["rbar"] - fit[0]) / max(1.0, abs(fit[0]))
            rec["sigma_rel_gpu_R"] = abs(g["sig"] - fit[1]) / fit[1]
            cand = (g["ell"] >= th).astype(np.uint8)
            prm = row[[9, 10, 5, 6, 7]]
            l6 = oracle.fof6d_halo(up, box.vel, m, cand, prm)
            rec["label6_mismatch_gpu_inputs"] = int((l6 != g["label6"]).sum())
            rec["near_threshold"] = report.near_threshold_pairs(up, box.vel, m, cand, prm,
                                                                P.v_ratio, P.theta_op)
        halos.append(rec)
    t_sample = time.perf_counter() - t_start
    ext = report.extrapolate(box.n, sizes, samples, t_fof / len(sel), P.nsearch_min)
    # ---- the two largest searched halos of <= 150,000 members: sampled f_l members, and
    #      the stage-by-stage checks (the oracle's own f_l of every member would take hours)
    big = []
    srch = np.flatnonzero((hs_np[:, 2] == 1) & (sizes <= 150000))
    for h in srch[np.argsort(sizes[srch])[-2:]]:
        row = hs_np[h]
        m = _gpu_members(lab_t, row[0])
        mt = torch.from_numpy(m.astype(np.int64)).to(dev)
        g = _halo_gpu(out, mt, row)
        up = oracle.unwrap(box.pos, m)
        ks = rng.choice(len(m), 16, replace=False)
        fo = report.sampled_members_fl(up, box.vel, m, ks, P.nse, P.nv)
        Rs, _, _ = oracle.background_halo(up, box.vel, m, g["f_l"])
        fit = oracle.ell_fit(g["R"])
        cand = (g["ell"] >= th).astype(np.uint8)
        prm = row[[9, 10, 5, 6, 7]]
        l6 = oracle.fof6d_halo(up, box.vel, m, cand, prm)
        big.append({"label": int(row[0]), "n": int(len(m)), "f_l_members_checked": 16,
                    "f_l_max_rel": report._rel(g["f_l"][ks], fo),
                    "R_max_rel_gpu_fl": report._rel(g["R"], Rs, 1.0),
                    "rbar_rel_gpu_R": abs(g["rbar"] - fit[0]) / max(1.0, abs(fit[0])),
                    "sigma_rel_gpu_R": abs(g["sig"] - fit[1]) / fit[1],
                    "label6_mismatch_gpu_inputs": int((l6 != g["label6"]).sum()),
                    "near_threshold": report.near_threshold_pairs(up, box.vel, m, cand, prm,
                                                                  P.v_ratio, P.theta_op)})
    small = _parity_c32(ctx, dev, P)
    srch_recs = [r for r in halos if "R_max_rel" in r]

    def mx(key, recs):
        v = [r[key] for r in recs if key in r]
        return float(max(v)) if v else None

    flips = [dict(f, halo=r["label"], band=r["band"]) for r in srch_recs for f in r["flips"]]
    near = [p for r in srch_recs + big for p in r["near_threshold"]["pairs"]]
    parity = {
        "sampled": {
            "box": wname, "halos": len(halos) + len(big), "searched_halos": len(srch_recs) + len(big),
            "independent": {
                "f_l_max_rel": mx("f_l_max_rel", halos + big),
                "R_max_rel": mx("R_max_rel", srch_recs),
                "rbar_max_abs": mx("rbar_abs", srch_recs),
                "sigma_max_rel": mx("sigma_rel", srch_recs),
                "ell_th_flips": flips,
                "flips_outside_band": sum(not f["within_band"] for f in flips),
                "label6_membership_differs": sum(r["label6_membership_differs"] for r in srch_recs),
            },
            "gpu_inputs": {
                "R_max_rel": mx("R_max_rel_gpu_fl", srch_recs + big),
                "rbar_max_rel": mx("rbar_rel_gpu_R", srch_recs + big),
                "sigma_max_rel": mx("sigma_rel_gpu_R", srch_recs + big),
                "label6_mismatches": sum(r["label6_mismatch_gpu_inputs"] for r in srch_recs + big),
            },
            "near_threshold_predicates": {
                "tol": 1e-12, "q": sum(r["near_threshold"]["q"] for r in srch_recs + big),
                "v_ratio": sum(r["near_threshold"]["v_ratio"] for r in srch_recs + big),
                "theta": sum(r["near_threshold"]["theta"] for r in srch_recs + big),
                "pairs": near[:50]},
            "fof3d_subcube": fof_par,
            "per_halo": halos + big,
        },
        "c32_whole_box": small,
        "tolerances": {"f_l": "1e-4 relative", "R": "1e-4 max(1,|R|)",
                       "labels": "bit-exact (3D; 6D with the same inputs)",
                       "flips": "only inside the band of ell_th that the measured R, R-bar "
                                "and sigma_R differences explain"},
    }
    nsamp = sum(k for _, _, k in CPU_BINS)
    cpu = {"value": ext["particles_per_s"], "unit": "particles/s", "cores": 1, "kind": "oracle",
           "sample": CPU_SAMPLE_DESC.format(nh=len(pick), bins=CPU_BINS, nhalo=len(sizes)),
           "extrapolated": True, "sample_seconds": t_sample, "fof_subcube_particles": int(len(sel)),
           "fof_seconds": t_fof, "model": ext, "halos_requested": nsamp}
    return cpu, parity


def _parity_c32(ctx, dev, P):
    """The 32^3 box through both pipelines, every particle: 3D labels, f_l, R, fit, ell
    flips with their bands, 6D membership."""
    import torch

    import oracle
    import synth
    from oracle import report

    box = synth.named("c32")
    pos = torch.from_numpy(box.pos).to(dev)
    vel = torch.from_numpy(box.vel).to(dev)
    lab = ctx.fof3d(pos, box.link_d2)
    o = ctx.find_substructure(pos, vel, lab, box.lx_sub, 1.0, P)
    ctx.sync()
    ref = oracle.pipeline(box.pos, box.vel, box.link_d2, box.lx_sub, 1.0)
    g = {k: o[k].cpu().numpy() for k in ("f_l", "R", "ell", "label6")}
    hs = o["halos"][: o["nhalo"]].cpu().numpy()
    l3 = lab.cpu().numpy()
    off, mem = oracle.halos(ref["label3"], P.nmin)
    recs = []
    for h in range(len(off) - 1):
        if hs[h, 2] != 1:
            continue
        m = mem[off[h]:off[h + 1]]
        gg = {k: g[k][m].astype(np.float64) if k != "label6" else g[k][m] for k in g}
        gg["rbar"], gg["sig"] = float(hs[h, 3]), float(hs[h, 4])
        oo = {"f_l": ref["f_l"][m], "R": ref["R"][m], "ell": ref["ell"][m],
              "label6": ref["label6"][m], "rbar": float(ref["halos"][h, 3]),
              "sig": float(ref["halos"][h, 4])}
        recs.append(report.compare_halo(m, gg, oo, P.ell_th))
    flips = [f for r in recs for f in r["flips"]]
    return {"particles": int(box.n), "label3_mismatches": int((l3 != ref["label3"]).sum()),
            "f_l_max_rel": report._rel(g["f_l"], ref["f_l"]),
            "R_max_rel": report._rel(g["R"], ref["R"], 1.0),
            "rbar_max_abs": max(r["rbar_abs"] for r in recs) if recs else None,
            "sigma_max_rel": max(r["sigma_rel"] for r in recs) if recs else None,
            "ell_th_flips": flips, "flips_outside_band": sum(not f["within_band"] for f in flips),
            "label6_membership_differs": int(((g["label6"] >= 0) != (ref["label6"] >= 0)).sum())}


def run_reference(args):
    """The oracle as it stands on the host cores: each step its 3D FOF on one sub-cube and
    its per-halo pipeline on a size-stratified sample of the generator's hosts (a host's
    particles stand in for a halo: the GPU path is not used here); the value is the
    whole-box rate extrapolated from the stage times over the generator's host sizes."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import report

    box = synth.named(args.workload if args.workload != "prelabelled" else "c512")
    hid = box.host_id
    order = np.argsort(hid, kind="stable")
    hs_sorted = hid[order]
    first = np.searchsorted(hs_sorted, 0)
    hosts, starts, counts = np.unique(hs_sorted[first:], return_index=True, return_counts=True)
    starts = starts + first
    keep = counts >= 20
    sizes = counts[keep]
    rng = np.random.default_rng(20190201)
    pick = report.stratified(sizes, rng, REF_BINS)
    members = []
    for i in pick:
        j = np.flatnonzero(keep)[i]
        members.append(np.sort(order[starts[j]:starts[j] + counts[j]]).astype(np.int32))

    def step():
        t0 = time.perf_counter()
        sel, _, t_fof = report.fof_subcube(box.pos, box.link_d2, side_div=8)
        samples = []
        for m in members:
            o = report.run_halo(box.pos, box.vel, m, box.lx_sub, 1.0)
            samples.append({"n": len(m), "t": o["t"]})
        return time.perf_counter() - t0, report.extrapolate(box.n, sizes, samples,
                                                           t_fof / len(sel))

    for _ in range(args.warmup):
        step()
    secs, exts = [], []
    for _ in range(args.steps):
        dt, ext = step()
        secs.append(dt)
        exts.append(ext)
    value = float(np.median([e["particles_per_s"] for e in exts]))
    desc = CPU_SAMPLE_DESC.format(nh=len(pick), bins=REF_BINS, nhalo=len(sizes)).replace(
        "the GPU's halos", "the generator's hosts") + (
        "; halos here are the generator's hosts (a host's particles, >= 20), sampled and "
        "summed over, since this arm runs no 3D FOF of the whole box")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(secs)) * 1e3,
        "value_basis": "whole-box rate extrapolated from each step's measured stage times; "
                       "ms_per_step is the wall time of one step's sample",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (int64 distances)", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.workload, args.workload),
                   "sample": desc, "parallelism": "single host core"},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": desc, "extrapolated": True, "model": exts[-1] if exts else None},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c512", choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="batched", choices=["plain", "batched"],
                    help="launch form of the headline number (batched: one launch per stage)")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed steps of the plain form (one launch per halo and stage) "
                         "reported beside a batched headline; 0 skips it")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-next-rows", dest="next_rows", action="store_false",
                    help="skip timing field 6DFOF and group cleaning after the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shapes instead of tuning them in the warm-up")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("note: warm-up raised to 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
