#!/usr/bin/env python
"""Throughput benchmark of the 3D RTM hot path (SMIwiz, arXiv 2311.02293).

Workload: the 3D salt RTM stand-in -- 300^3 physical grid (340^3 with the 20
CPML layers), 10 m, order 8, nt = 2500, dt = 0.8 ms, 15 Hz Ricker, 8 shots,
150 x 150 receivers, FP32 compute, zero-lag cross-correlation image.  One
step = the whole hot path for one shot: forward modelling with boundary
saving, then the reverse loop (adjoint propagation, source-field
reconstruction, imaging), Algorithm 2.  Shots cycle over the 8 of the
workload.

Metric: grid-point updates per second over all three propagations
(forward, adjoint, reconstruction), counting the points each step actually
updates inside the computing box (Sec. 4.1).  `value` is timed with CUDA
events on device-resident inputs; `e2e` calls the C ABI with pinned host
buffers (host<->device copies inside the timed region).

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun, each rank processes its own shots (no collective on the data
path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D RTM grid-point updates/s (forward + adjoint + reconstruction, computing box)"
# DRAM bytes moved per algorithmic byte of each stencil class (forward,
# adjoint, reconstruction): ncu dram__bytes_read.sum + dram__bytes_write.sum
# over the kernels of one forward and one reverse step of the 340^3 salt
# case with the box off (`bench.py --profile rtm --nt 30 --no-box`).  A
# bench launch's traffic is this ratio times its algorithmic bytes.
TRAFFIC_PER_ALGO_BYTE = (1.525, 1.597, 1.441)
UNIT = "Gpt-updates/s"
WORKLOAD = "3d_rtm_salt_300^3_order8_nt2500_8shots_150x150rec"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shell", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--dr", type=int, default=1, help="boundary decimation ratio (Sec. 4.2; 1 = every step)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-other", action="store_true", help="skip the 3D forward and 2D gradient workloads")
    ap.add_argument("--other-nt3", type=int, default=3000, help="time steps of the 3D forward workload")
    ap.add_argument("--other-nt2", type=int, default=3000, help="time steps of the 2D gradient workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nt", type=int, default=2500, help="time steps (full workload: 2500)")
    ap.add_argument("--table", action="store_true",
                    help="results table instead: GPU and oracle rates of each workload (several minutes)")
    ap.add_argument("--serve", action="store_true",
                    help="serving mix instead: throughput and p50/p99 latency of the request server")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-scale", type=float, default=0.5,
                    help="grid sizes and nt of the serving mix relative to the full mix")
    ap.add_argument("--serve-slots", type=int, default=8, help="concurrent request slots of the server")
    ap.add_argument("--serve-rates", default="1.2,0.5",
                    help="Poisson arrival rates as multiples of the one-at-a-time rate (comma list)")
    ap.add_argument("--serve-mix", default="surveys", choices=["surveys", "independent"],
                    help="requests as shots of seeded surveys (shareable calls) or independent draws")
    ap.add_argument("--profile", choices=["fwd", "rtm", "family", "grad2d"],
                    help="profiling case instead: one untimed forward call (observed data), then one forward "
                         "or RTM call of a one-shot salt model, printing per-class times")
    ap.add_argument("--n", type=int, default=300, help="physical grid size of the profiling case (n^3)")
    ap.add_argument("--no-box", action="store_true", help="profiling case without the computing box")
    ap.add_argument("--freesurf", action="store_true", help="profiling case with the free surface (Sec. 2.1)")
    ap.add_argument("--kernels", default="auto", choices=["auto", "twopass", "fused", "inline", "generic"],
                    help="3D kernel family (auto = twopass: velocity and pressure passes, CPML band kernels; fused: "
                         "the single-pass step; inline: two passes with the CPML terms in band-tile classes)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_shots(nshot: int, world: int, rank: int, nsteps: int) -> list:
    """Shots of this rank, cycled over nsteps steps: rank r owns shots
    r, r+world, ... (replicas; no exchange on the data path)."""
    mine = list(range(rank % nshot, nshot, world)) or [rank % nshot]
    return [mine[k % len(mine)] for k in range(nsteps)]


def aggregate(t_ms: float, units: float, world: int, device):
    """(max time over ranks in ms, sum of units over ranks)."""
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
def shot_units(w) -> float:
    """Grid-point updates of one shot of the workload with the computing box
    (forward + adjoint on the extended grid, reconstruction on the physical
    grid), from the oracle's own box tables."""
    from oracle import oracle as O
    prob = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm)
    lo_s, hi_s = O.box_table(prob, w.vp, w.rho, w.srcs[0], 0, w.nt)
    lo_r, hi_r = O.box_table(prob, w.vp, w.rho, w.recs[0], 0, w.nt)
    L = np.full(3, w.nb)
    H = np.array(w.n) + w.nb - 1
    fwd = np.prod(np.maximum(hi_s - lo_s + 1, 0), axis=1).sum()
    adj = np.prod(np.maximum(hi_r - lo_r + 1, 0), axis=1).sum()
    rec = np.prod(np.maximum(np.minimum(hi_s, H) - np.maximum(lo_s, L) + 1, 0), axis=1).sum()
    return float(fwd + adj + rec)


def cpu_baseline_sample(w, nsteps: int = 3):
    """The FP64 oracle as it stands on this host's cores: one shot of the
    workload cut to `nsteps` time steps with the computing box off (every
    step updates the whole grid), RTM mode.  The oracle times its forward and
    reverse time loops itself, so set-up is excluded; the rate is point
    updates of those loops per second."""
    from oracle import oracle as O
    prob = O.Problem(w.n, w.d, nsteps, w.dt, order=w.order, nb=w.nb, fm=w.fm, use_box=False)
    dobs = np.zeros((nsteps, len(w.recs[0])))
    phase = np.zeros(4)
    t0 = time.perf_counter()
    O.gradient(prob, w.vp, w.rho, w.stf[:nsteps], w.srcs[0], w.recs[0], dobs, mode="rtm", phase_s=phase)
    wall = time.perf_counter() - t0
    ext = float(np.prod([n + 2 * w.nb for n in w.n]))
    phys = float(np.prod(w.n))
    k = nsteps - 1                    # timed steps of each loop (its first step touches fresh memory)
    fwd_pts, rev_pts = k * ext, k * (ext + phys)
    rate = (fwd_pts + rev_pts) / (phase[0] + phase[1]) / 1e9
    cores = O.max_threads()
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": float(phase[0] + phase[1]), "wall_seconds_incl_setup": wall,
            "per_phase_gpts": {"forward": fwd_pts / phase[0] / 1e9,
                               "reverse_adjoint_reconstruction_imaging": rev_pts / phase[1] / 1e9},
            "sample": f"one shot of the workload cut to {nsteps} of {w.nt} time steps, computing box off, "
                      f"FP64 C oracle on {cores} OpenMP threads (every phase, the adjoint scatter included); "
                      f"the last {k} steps of the forward loop ({phase[0]:.1f} s) and of the reverse loop "
                      f"({phase[1]:.1f} s) timed by the oracle; set-up and each loop's first step (which "
                      f"touches freshly allocated fields: {phase[2]:.1f} s + {phase[3]:.1f} s) excluded; "
                      f"{wall:.1f} s in all"}


def other_workloads(smi, synth, torch, dev, peak: float, args) -> dict:
    """The two other GPU workloads, each timed once with CUDA events after an
    untimed warm-up call, outside the main timed region:
      - 3D forward with the computing box: 400 x 400 x 200 + 20 CPML layers,
        order 8, nt 3000, corner source, 200 x 200 receivers;
      - 2D FWI gradient: 301 x 1001 + 20 layers, order 8, nt 3000, 40 shots
        in one batch, observed data from the true model.
    Each reports grid-point updates/s (box points) and the roofline of its
    dominant stencil class (algorithmic bytes / that class's event time)."""
    out = {}

    def roof(st):
        ms, by = np.array(st["ms"]), np.array(st["bytes"])
        dom = int(np.argmax(ms))
        ach = by[dom] / (ms[dom] / 1e3) / 1e9
        return {"class": ["forward", "adjoint", "reconstruction"][dom], "achieved_gbs": float(ach),
                "frac": float(ach / peak), "per_class_gbs": [float(b / (m / 1e3) / 1e9) if m > 0 else None
                                                              for b, m in zip(by, ms)]}

    def timed(f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    w = synth.random_smooth_3d(nt=args.other_nt3)
    vp, rho, stf = (torch.from_numpy(a).to(dev) for a in (w.vp, w.rho, w.stf))
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, profile=True)
    warm = smi.Problem(w.d, min(w.nt, 200), w.dt, w.fm, order=w.order, nb=w.nb)
    smi.smi_forward(vp, rho, warm, w.srcs, w.recs, stf[:warm.nt].contiguous())
    ms = timed(lambda: smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf))
    st = smi.smi_last_stats()
    out["forward_3d_random_400x400x200_nt%d" % w.nt] = {
        "gpts": st["point_updates"] / (ms * 1e6), "ms": ms, "roofline": roof(st),
        "effective_gpts": float(np.prod([n + 2 * w.nb for n in w.n]) * w.nt / (ms * 1e6))}
    del vp, rho, stf

    w = synth.layered_fault_2d(nt=args.other_nt2, nshot=40)
    vp, rho, stf, vpt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.vp, w.rho, w.stf, w.vp_true))
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, profile=True)
    dobs = smi.smi_forward(vpt, rho, prob, w.srcs, w.recs, stf, flat=True)
    smi.smi_fwi_gradient(vp, rho, prob, w.srcs[:2], w.recs[:2], stf, dobs[: 2 * w.nt * len(w.recs[0])])
    ms = timed(lambda: smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs))
    st = smi.smi_last_stats()
    out["gradient_2d_layered_301x1001_40shots_nt%d" % w.nt] = {
        "gpts": st["point_updates"] / (ms * 1e6), "ms": ms, "shots_per_s": 40 / (ms / 1e3), "roofline": roof(st)}
    torch.cuda.synchronize()
    return out


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2311_02293_gb300 import synth
    w = synth.salt_3d(nt=args.nt)
    from oracle import oracle as O
    O.build()
    small = synth.tiny_3d()
    for _ in range(args.warmup):       # warm-up: the oracle's code path on a tiny case
        p = O.Problem(small.n, small.d, small.nt, small.dt, order=small.order, nb=small.nb, fm=small.fm)
        O.gradient(p, small.vp, small.rho, small.stf, small.srcs[0], small.recs[0],
                   np.zeros((small.nt, len(small.recs[0]))), mode="rtm")
    units = shot_units(w)             # one step = one shot of the workload, as in our arm
    vals = []
    for _ in range(args.steps):
        cb = cpu_baseline_sample(w)
        vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": units / (v * 1e9) * 1e3,
            "ms_per_step_kind": "one shot's box point updates at the sampled per-step rate",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2311_02293_gb300 import build, synth
    if not os.path.exists(os.path.join(ROOT, "paper_2311_02293_gb300", "libsmi.so")):
        build.build()
    from paper_2311_02293_gb300 import smi

    w = synth.salt_3d(nt=args.nt)
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, shell_prec=args.shell,
                       profile=True, dr=args.dr, kernels=args.kernels)
    vp = torch.from_numpy(w.vp).to(dev)
    rho = torch.from_numpy(w.rho).to(dev)
    stf = torch.from_numpy(w.stf).to(dev)
    order = shard_shots(w.nshot, world, rank, args.warmup + args.steps)
    # observed data: forward modelling in the true model (untimed set-up)
    gen = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    dobs = {}
    for s in sorted(set(order)):
        dobs[s] = smi.smi_forward(torch.from_numpy(w.vp_true).to(dev), rho, gen, w.srcs[s:s + 1],
                                  w.recs[s:s + 1], stf)[0].contiguous()
    torch.cuda.synchronize()

    def step(s):
        img = smi.smi_rtm(vp, rho, prob, w.srcs[s:s + 1], w.recs[s:s + 1], stf, dobs[s])
        return img, smi.smi_last_stats()

    for k in range(args.warmup):
        step(order[k])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for k in range(args.steps):
        _, st = step(order[args.warmup + k])
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    units = sum(s["point_updates"] for s in stats)
    t_max, u_sum = aggregate(t_ms, units, world, dev)
    value = u_sum / (t_max / 1e3) / 1e9

    # roofline of the dominant stencil class (forward / adjoint / reconstruction)
    ms = np.sum([s["ms"] for s in stats], axis=0)
    by = np.sum([s["bytes"] for s in stats], axis=0)
    steps_cls = np.sum([s["steps"] for s in stats], axis=0)
    dom = int(np.argmax(ms))
    names = ["forward v+p stencil step", "adjoint v+p stencil step", "reconstruction + imaging step"]
    peak, peak_kind = measured_peaks()
    achieved = by[dom] / (ms[dom] / 1e3) / 1e9 if ms[dom] > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": float(TRAFFIC_PER_ALGO_BYTE[dom] * by[dom] / max(steps_cls[dom], 1)),
            "kernel": names[dom], "peak_source": peak_kind,
            "per_class_gbs": {names[c]: (by[c] / (ms[c] / 1e3) / 1e9 if ms[c] > 0 else None) for c in range(3)},
            "per_class_share": {names[c]: float(ms[c] / max(ms.sum(), 1e-9)) for c in range(3)},
            "bytes_per_launch": float(by[dom] / max(steps_cls[dom], 1))}

    # end to end: pinned host buffers through the C ABI, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        hvp = torch.from_numpy(w.vp).pin_memory()
        hrho = torch.from_numpy(w.rho).pin_memory()
        hstf = torch.from_numpy(w.stf).pin_memory()
        hd = {s: dobs[s].cpu().pin_memory() for s in dobs}
        himg = torch.empty(w.vp.shape, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        eunits = 0.0
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            s = order[args.warmup + k % max(args.steps, 1)]
            smi.smi_rtm(hvp, hrho, prob, w.srcs[s:s + 1], w.recs[s:s + 1], hstf, hd[s], out=himg)
            eunits += smi.smi_last_stats()["point_updates"]
        te = time.perf_counter() - t0
        h2d = hvp.numel() * 4 + hrho.numel() * 4 + hstf.numel() * 4 + next(iter(hd.values())).numel() * 4
        e2e = {"value": eunits / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(himg.numel() * 4), "steps": args.e2e_steps}

    others = None
    if rank == 0 and world == 1 and not args.no_other:
        others = other_workloads(smi, synth, torch, dev, measured_peaks()[0], args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(w)

    if rank == 0:
        ne = [n + 2 * w.nb for n in w.n]
        eff = args.steps * w.nt * (2 * np.prod(ne) + np.prod(w.n)) / (t_max / 1e3) / 1e9
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "shots_per_step": 1, "boundary_storage": args.shell,
                           "boundary_decimation": args.dr,
                           "nt": w.nt, "grid_extended": ne, "l2": "inputs larger than L2 (157 MB per field)",
                           "parallelism": f"replicas x{world} (shots sharded)"},
                "effective_gpts": float(eff),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
                "other_workloads": others}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """The case the ncu summaries under profiles/ capture: one shot of the
    salt model at n^3, one untimed forward call to make the observed data,
    then one forward (fwd) or RTM (rtm) call; prints per-class times and
    algorithmic bandwidths from the library's own CUDA events."""
    import torch
    from paper_2311_02293_gb300 import build, synth
    if not os.path.exists(os.path.join(ROOT, "paper_2311_02293_gb300", "libsmi.so")):
        build.build()
    from paper_2311_02293_gb300 import smi
    dev = torch.device("cuda:0")
    if args.profile == "grad2d":
        run_profile_grad2d(args, torch, synth, smi, dev)
        return
    w = synth.salt_3d(n=args.n, nt=args.nt, nshot=1)
    vp, rho, stf = (torch.from_numpy(a).to(dev) for a in (w.vp, w.rho, w.stf))
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, profile=True, use_box=not args.no_box,
                       freesurf=args.freesurf, kernels=args.kernels)
    seis = smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf)
    torch.cuda.synchronize()
    if args.profile == "family":
        # the FWI gradient of Vp alone against the (Vp, Ip) family gradient
        # (density part included): call times with CUDA events, warm calls
        dobs = (0.9 * seis[0]).contiguous()

        def timed(f):
            f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        t_vp = timed(lambda: smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs))
        t_fam = timed(lambda: smi.smi_fwi_gradient_family(vp, rho, prob, w.srcs, w.recs, stf, dobs, family=2))
        st = smi.smi_last_stats()
        print(json.dumps({"profile": "family", "n": args.n, "nt": args.nt, "box": not args.no_box,
                          "ms_gradient_vp": t_vp, "ms_gradient_family2": t_fam, "ratio": t_fam / t_vp,
                          "kernel_launches_family2": st["kernel_launches"]}), flush=True)
        return
    if args.profile == "fwd":
        smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf)
    else:
        img = smi.smi_rtm(vp, rho, prob, w.srcs, w.recs, stf, seis[0])
    torch.cuda.synchronize()
    st = smi.smi_last_stats()
    names = ["forward", "adjoint", "reconstruction"]
    line = {"profile": args.profile, "n": args.n, "nt": args.nt, "box": not args.no_box, "freesurf": args.freesurf,
            "kernels": args.kernels,
            "ms": dict(zip(names, st["ms"])),
            "algorithmic_gbs": {c: (b / (m * 1e6) if m else None) for c, b, m in zip(names, st["bytes"], st["ms"])},
            "kernel_launches": st["kernel_launches"]}
    if args.profile == "rtm" and (args.shell != "f32" or args.dr > 1):
        # the image with 16-bit and / or decimated boundary storage against
        # FP32 storage of every step, with the time and footprint of the call
        pq = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, use_box=not args.no_box,
                         shell_prec=args.shell, dr=args.dr, profile=True)
        iq = smi.smi_rtm(vp, rho, pq, w.srcs, w.recs, stf, seis[0])
        torch.cuda.synchronize()
        sq = smi.smi_last_stats()
        line["shell"] = args.shell
        line["dr"] = args.dr
        line["image_rel_l2_vs_f32_every_step"] = float(torch.linalg.norm(iq - img) / torch.linalg.norm(img))
        line["ms_with_options"] = dict(zip(names, sq["ms"]))
        line["device_bytes"] = {"f32_every_step": st["device_bytes"], "with_options": sq["device_bytes"]}
    print(json.dumps(line), flush=True)


def run_profile_grad2d(args, torch, synth, smi, dev):
    """The 2D FWI gradient workload (layered-fault stand-in, 301 x 1001 at
    12.5 m, order 8, 40 shots in one batch; --nt steps): observed data from
    the true model, one warm gradient call, then one timed call; prints the
    call time, the grid-point rate and the per-class CUDA-event times and
    algorithmic bandwidths of the timed call."""
    w = synth.layered_fault_2d(nt=args.nt, nshot=40)
    vp, rho, stf, vpt = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.vp, w.rho, w.stf, w.vp_true))
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, profile=True, use_box=not args.no_box)
    dobs = smi.smi_forward(vpt, rho, prob, w.srcs, w.recs, stf, flat=True)
    smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = smi.smi_last_stats()
    names = ["forward", "adjoint", "reconstruction"]
    print(json.dumps({"profile": "grad2d", "n": list(w.n), "nt": args.nt, "nshot": 40, "box": not args.no_box,
                      "ms_call": ms, "gpts": st["point_updates"] / (ms * 1e6), "ms": dict(zip(names, st["ms"])),
                      "algorithmic_gbs": {c: (b / (m * 1e6) if m else None)
                                          for c, b, m in zip(names, st["bytes"], st["ms"])},
                      "kernel_launches": st["kernel_launches"]}), flush=True)


def run_table(args):
    """One JSON line per workload for the results table: the GPU rate of the
    workload's call (CUDA events after a warm-up call; grid-point updates
    inside the computing box, and over the full grid) with the dominant
    stencil class's roofline fraction, and the FP64 oracle's per-step rate on
    all of this host's cores and on one core (a few time steps of one shot
    with the box off, set-up and each loop's first step excluded)."""
    import torch
    from oracle import oracle as O
    from paper_2311_02293_gb300 import build, synth
    if not os.path.exists(os.path.join(ROOT, "paper_2311_02293_gb300", "libsmi.so")):
        build.build()
    from paper_2311_02293_gb300 import smi
    dev = torch.device("cuda:0")
    peak = measured_peaks()[0]

    def oracle_rate(w, nsteps, nthreads):
        prob = O.Problem(w.n, w.d, nsteps, w.dt, order=w.order, nb=w.nb, fm=w.fm, use_box=False, nthreads=nthreads)
        phase = np.zeros(4)
        O.gradient(prob, w.vp, w.rho, w.stf[:nsteps], w.srcs[0], w.recs[0], np.zeros((nsteps, len(w.recs[0]))),
                   mode="rtm", phase_s=phase)
        ext, phys = float(np.prod([n + 2 * w.nb for n in w.n])), float(np.prod(w.n))
        k = nsteps - 1
        return {"gpts": k * (2 * ext + phys) / (phase[0] + phase[1]) / 1e9, "threads": nthreads or O.max_threads(),
                "steps_timed": k}

    def gpu(call, st_scale=1.0):
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = smi.smi_last_stats()
        cms, cby = np.array(st["ms"]), np.array(st["bytes"])
        dom = int(np.argmax(cms))
        return ms, st, {"class": ["forward", "adjoint", "reconstruction"][dom],
                        "frac": float(cby[dom] / (cms[dom] / 1e3) / 1e9 / peak)}

    rows = []
    cases = [("C1 2D forward 201x201 nt1000", synth.two_layer_2d(), "forward", 60, 20),
             ("C2 2D gradient 301x1001 40 shots nt3000", synth.layered_fault_2d(nt=3000, nshot=40), "gradient", 12, 4),
             ("C3 3D forward 400x400x200 nt3000", synth.random_smooth_3d(nt=3000), "forward", 3, 2),
             ("C4 3D RTM 300^3 one shot nt2500", synth.salt_3d(nt=2500).subset([0]), "rtm", 3, 2)]
    for name, w, kind, ns_all, ns_one in cases:
        vp, rho, stf = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.vp, w.rho, w.stf))
        line = {"table": name}
        for shell in (["f32", "f16"] if kind == "rtm" else ["f32"]):
            prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, profile=True, shell_prec=shell)
            if kind == "forward":
                call = lambda: smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf, flat=True)
                props = 1
            else:
                vpt = torch.from_numpy(np.ascontiguousarray(w.vp_true if w.vp_true is not None else w.vp)).to(dev)
                dobs = smi.smi_forward(vpt, rho, smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb),
                                       w.srcs, w.recs, stf, flat=True)
                if kind == "rtm":
                    call = lambda: smi.smi_rtm(vp, rho, prob, w.srcs, w.recs, stf, dobs)
                else:
                    call = lambda: smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs)
                props = 3
            ms, st, roof = gpu(call)
            ext = float(np.prod([n + 2 * w.nb for n in w.n]))
            phys = float(np.prod(w.n))
            full = (ext if props == 1 else 2 * ext + phys) * w.nt * len(w.srcs)
            line["gpu_" + shell] = {"ms": ms, "gpts": st["point_updates"] / (ms * 1e6), "effective_gpts": full / (ms * 1e6),
                                    "roofline": roof}
        line["oracle_all_cores"] = oracle_rate(w, ns_all, 0)
        line["oracle_one_core"] = oracle_rate(w, ns_one, 1)
        rows.append(line)
        print(json.dumps(line), flush=True)
        del vp, rho, stf
        torch.cuda.empty_cache()


def run_serve(args):
    """Serving mix: one-at-a-time plain FP32 calls vs the request server (FP16
    boundaries, --serve-slots slots) under Poisson arrivals at 1.2x and 0.5x
    the measured one-at-a-time service rate, and with every request queued at
    once; `value` is the served gradient shots/s of the saturated run.
    --serve-mix surveys draws the requests as shots of seeded surveys, which
    the server may merge into shot-batched calls; independent draws every
    request's own nt, so none can share a call."""
    import torch
    from paper_2311_02293_gb300 import build
    if not os.path.exists(os.path.join(ROOT, "paper_2311_02293_gb300", "libsmi.so")):
        build.build()
    from paper_2311_02293_gb300 import serve, smi
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    surveys = args.serve_mix == "surveys"
    reqs = serve.make_mix(args.serve_requests, scale=args.serve_scale, shell="f16", surveys=surveys)
    plain = serve.make_mix(args.serve_requests, scale=args.serve_scale, shell="f32", surveys=surveys)
    serve._prepare(reqs, dev)
    serve._prepare(plain, dev)
    serve.run_alone(plain[:4], dev)                        # warm-up
    clocks = Clocks(dev.index)
    clocks.start()
    _, t_alone = serve.run_alone(plain, dev)
    rate1 = len(plain) / t_alone
    out = {}
    # Poisson arrivals at 1.2x and 0.5x the one-at-a-time rate (latency under load; the arrival rate
    # bounds the throughput), then every request queued at once (the server's capacity)
    rates = [float(x) for x in args.serve_rates.split(",") if x.strip()]
    for name, factor in [(f"rate_{r:g}x", r) for r in rates] + [("saturated", None)]:
        m = serve.run_mix(reqs, dev, slots=args.serve_slots, rate=factor * rate1 if factor else None)
        out[name] = {"requests_per_s": m["requests_per_s"], "gradient_shots_per_s": m["gradient_shots_per_s"],
                     "p50_s": m["p50_s"], "p99_s": m["p99_s"], "failed": m["failed"], "seconds": m["seconds"],
                     "merged_calls": m["merged_calls"], "merged_requests": m["merged_requests"]}
    clk = clocks.stop()
    ngrad = sum(1 for r in plain if r.kind == "gradient")
    kinds = {k: sum(1 for r in reqs if r.kind == k) for k in ("gradient", "forward", "rtm")}
    line = {"metric": "served gradient shots/s (request server, FP16 boundaries)",
            "value": out["saturated"]["gradient_shots_per_s"], "unit": "gradient shots/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving_mix_{len(reqs)}req_scale{args.serve_scale}", "mix": args.serve_mix,
                       "kinds": kinds,
                       "slots": args.serve_slots, "arrivals": "poisson", "boundaries": "f16 served, f32 one at a time"},
            "clocks": clk,
            "one_at_a_time_fp32": {"requests_per_s": rate1, "gradient_shots_per_s": ngrad / t_alone,
                                   "seconds": t_alone},
            "served": out}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.profile:
        run_profile(a)
    elif a.table:
        run_table(a)
    elif a.serve:
        run_serve(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
