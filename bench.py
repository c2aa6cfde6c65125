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

--impl reference times the FP64 C oracle (the path's reference implementation) on the
host cores, one step = the oracle pipeline over a bounded sample of the workload (a 64^3
box drawn by the same generator with the same parameters).
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
SAMPLE_BOX = "m64"
SAMPLE_DESC = ("64^3 box (262,144 particles) drawn by the same generator with the same "
               "parameters; full oracle pipeline (3D FOF, f_l, background R, fit, 6D links)")
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
# DRAM bytes per query particle of k_velden_big from one ncu capture of the 160^3 box
# (41.9 MB over 1,183,473 queries; profiles/k_velden_big_160cubed.md). The kernel's DRAM
# traffic grows with the number of queries, so a full launch is this times its queries.
# Set to None whenever the kernel changes and the capture has not been redone.
VELDEN_DRAM_BYTES_PER_QUERY = 41.942784e6 / 1183473
SMS, LANES_PER_SM = 152, 128


def alu_peak_tops(sm_mhz):
    # one 32-bit ALU operation per lane per clock: 152 SMs x 128 lanes x SM clock
    return SMS * LANES_PER_SM * sm_mhz * 1e6 / 1e12


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

    for _ in range(args.warmup):
        step()
    ctx.sync()
    torch.cuda.synchronize(dev)

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
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pos.copy_(hpos, non_blocking=True)
            vel.copy_(hvel, non_blocking=True)
            if prelab:
                lab.copy_(hl3, non_blocking=True)
            step()
            if not prelab:
                hl3.copy_(lab, non_blocking=True)
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
    nh = out["halos"][: out["nhalo"]].cpu().numpy()
    nq_big = float(nh[nh[:, 1] > P.nse, 1].sum())
    roof = None
    if dom == "velden_big" and kern[dom][1] > 0:
        per_launch_ms = kern[dom][0] / kern[dom][1]
        ops = VELDEN_OPS_PER_QUERY * nq_big
        achieved = ops / (per_launch_ms / 1e3) / 1e12
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = alu_peak_tops(sm_mhz)
        traffic = (VELDEN_DRAM_BYTES_PER_QUERY * nq_big if VELDEN_DRAM_BYTES_PER_QUERY else None)
        roof = {"kernel": "k_velden_big", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "ncu dram bytes per query on the 160^3 box x queries of this launch",
                "peak_source": f"152 SMs x 128 lanes x {sm_mhz:.0f} MHz (sm_max_mhz of {how} peaks)",
                "algorithmic": f"{VELDEN_OPS_PER_QUERY} ops x {int(nq_big)} query particles",
                "launch_ms": per_launch_ms}
    elif dom == "fof_link" and kern[dom][1] > 0:
        per_launch_ms = kern[dom][0] / kern[dom][1]
        achieved = 16.0 * box.n / (per_launch_ms / 1e3) / 1e9
        roof = {"kernel": "k_fof_link", "bound": "hbm", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": None, "launch_ms": per_launch_ms}
    total_dev = sum(v[0] for v in kern.values())
    shares = {k: round(v[0] / max(ms, 1e-9), 4) for k, v in kern.items()}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_once()
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64 and exact u32 distances, f32 f_l, f64 background/fit/links", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.workload, args.workload),
                   "n_particles": box.n, "halos": int(out["nhalo"]), "form": args.form,
                   "l2": "inputs 24 B/particle >> 129 MB L2; no flush between steps",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "kernel_share_of_step": shares,
        "plain_form": plain,
        "next_rows": next_rows,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- oracle arm
def cpu_baseline_once():
    import oracle
    import synth

    box = synth.named(SAMPLE_BOX)
    t = time.perf_counter()
    oracle.pipeline(box.pos, box.vel, box.link_d2, box.lx_sub, 1.0)
    dt = time.perf_counter() - t
    return {"value": box.n / dt, "unit": "particles/s", "cores": 1, "kind": "oracle",
            "sample": SAMPLE_DESC, "seconds": dt}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    box = synth.named(SAMPLE_BOX)
    for _ in range(args.warmup):
        oracle.pipeline(box.pos, box.vel, box.link_d2, box.lx_sub, 1.0)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.pipeline(box.pos, box.vel, box.link_d2, box.lx_sub, 1.0)
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    value = box.n / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (int64 distances)", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.workload, args.workload),
                   "sample": SAMPLE_DESC, "parallelism": "single host core"},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": SAMPLE_DESC},
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
