#!/usr/bin/env python
"""Benchmark of the Compton ring-localisation hot path on GB300.

One step = one burst through the whole path: 200,000 simulated 2-4-site
events -> rings (ordering, axis, eta, deta) -> ring x direction likelihood
sweep over a 49,152-direction HEALPix (nside 64, RING) grid -> block argmax ->
Gauss-Newton refinement of the best direction.  Inputs are resident in HBM
when the timed region starts; L2 is flushed (256 MiB write) before every timed
step.  The metric is ring x direction evaluations per second (rings x
directions per step / step time); per-step latency percentiles are reported
beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank localises its own burst
(replicas, weak scaling); the barrier and the max-over-ranks time come from
torch.distributed.  `--impl reference` times the CPU oracle instead (the
reference arm of this build), on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ring×direction evals/s; burst localization p50/p99 ms at ≤0.5° error vs oracle"
UNIT = "ring×direction evals/s"
N_SRC, N_BKG, NSIDE = 18182, 181818, 64
ALG_FP32_PER_PAIR, ALG_MUFU_SQRT, ALG_MUFU_EX2 = 16, 1, 1
FP32_PER_CLK_SM, SQRT_PER_CLK_SM, EX2_PER_CLK_SM = 128, 16, 32


def peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def alu_pairs_per_clk_sm():
    """Algorithmic pairs per clock per SM: the tighter of the FP32 pipe
    (16 FP32 ops per pair) and the MUFU pipe (one sqrt-class op at 16/clk and
    one ex2 at 32/clk per pair)."""
    fp32 = FP32_PER_CLK_SM / ALG_FP32_PER_PAIR
    mufu = 1.0 / (ALG_MUFU_SQRT / SQRT_PER_CLK_SM + ALG_MUFU_EX2 / EX2_PER_CLK_SM)
    return min(fp32, mufu)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=10)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 7]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        pw = [float(r[2]) for r in rows if re.match(r"^\s*[\d.]+\s*$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if "Active" in r[4 + k] and "Not" not in r[4 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# distributed plumbing (replicas)
# --------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v, dev=None):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# --------------------------------------------------------------------------
ORACLE_PARAMS = dict(sigma_e_frac=0.05, sigma_pos_cm=1.0, deta_min=math.radians(0.5),
                     deta_max=math.radians(20.0))


def event_config(world, n_events, n_valid, M):
    """The event workload's `config`, the same on both arms."""
    return {"workload": "events200k_healpix64", "events": n_events, "valid_rings": n_valid,
            "evals": "valid rings x directions", "directions": M,
            "grid": "HEALPix nside 64 RING", "sites": "2/3/4 at 0.5/0.3/0.2",
            "source_to_background": "1:10",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas x{world}"}


def oracle_path(ev, grid, threads):
    """The whole path on the oracle (C, FP64) for the events `ev`: rings of
    every event (1 thread), the map of every valid ring over every direction
    of `grid` (OpenMP, `threads`), its argmax and the refinement from it.
    Returns (seconds, valid rings, details)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.rings_from_events(ev, *ORACLE_PARAMS.values())
    t1 = time.perf_counter()
    m = oracle.likelihood_map(r, grid, nthreads=threads)
    t2 = time.perf_counter()
    j = oracle.argmax(m)
    d, obj, iters, st = oracle.refine(r, [grid[0][j], grid[1][j], grid[2][j]], tol_rad=1e-10)
    t3 = time.perf_counter()
    return t3 - t0, int(r["valid"].sum()), {
        "t_recon_s": t1 - t0, "t_map_s": t2 - t1, "t_refine_s": t3 - t2, "argmax": j,
        "dir": d, "status": st, "iters": iters}


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores.  Each
    step runs the whole path (rings, map over all 49,152 directions, argmax,
    refinement) on one slice of 5,000 events of the 200k-event burst, the
    slices taken in turn; the value is the ring x direction evaluations those
    steps made divided by the time they took, so the steps, ms_per_step and
    the timed region are what actually ran."""
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_2411_04785_gb300 import synth
    ev = synth.simulate_events(n_src=N_SRC, n_bkg=N_BKG, seed=2)
    N = ev["n"].size
    grid = oracle.grid_healpix_ring(NSIDE)
    M = grid[0].size
    threads = os.cpu_count() or 1
    slice_n = 5000
    n_slices = N // slice_n
    times, evals = [], 0
    for i in range(args.warmup + args.steps):
        a = (i % n_slices) * slice_n
        part = {"n": ev["n"][a:a + slice_n],
                **{k: np.ascontiguousarray(ev[k][:, a:a + slice_n]) for k in "xyze"}}
        t, n_valid, _ = oracle_path(part, grid, threads)
        if i >= args.warmup:
            times.append(t)
            evals += n_valid * M
    tot = float(np.sum(times))
    value = evals / tot
    n_valid_all = int(oracle.rings_from_events(ev, *ORACLE_PARAMS.values())["valid"].sum())
    sample = (f"each step: the whole path on one 5,000-event slice of the {N}-event burst "
              f"(slices in turn): oracle rings (1 thread), map of the slice's valid rings over "
              f"all {M} directions ({threads} threads), argmax, refinement; value = "
              f"evaluations made / time taken, no extrapolation")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": event_config(world, N, n_valid_all, M),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads,
                         "kind": "oracle", "sample": sample, "timed_s": tot,
                         "evals": evals, "extrapolated": False},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def ncu_traffic(summary, source):
    """DRAM bytes per launch (read + write) from a committed ncu summary under
    profiles/, if it was taken on the current kernel source (same sha256)."""
    try:
        txt = open(os.path.join(ROOT, "profiles", summary)).read()
        sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2411_04785_gb300", "csrc", source),
                                  "rb").read()).hexdigest()
    except OSError:
        return None
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != sha:
        return None
    return float(t.group(1))


def recon_pile(cc, synth, ev, params, dev, copies=80, warm=3, timed=5):
    """Reconstruction of the event workload tiled `copies` times (16M events,
    larger than L2): returns the HBM roofline record."""
    import torch
    pile = synth.tile_events(ev, copies)
    pn = torch.from_numpy(pile["n"]).to(dev)
    px, py, pz, pe = (torch.from_numpy(pile[k]).to(dev) for k in "xyze")
    rings = cc.empty_rings(pn.numel(), dev)
    for _ in range(warm):
        cc.rings_from_events(pn, px, py, pz, pe, params, rings)
    torch.cuda.synchronize()
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    for _ in range(timed):
        cc.rings_from_events(pn, px, py, pz, pe, params, rings)
    cc.trace_enable(False)
    rt = cc.trace_read(reset=True)["recon"]
    k = ev["n"].astype(np.int64)
    alg_bytes = copies * int((1 + 16 * k + 22).sum())
    ms = rt["ms"] / max(rt["launches"], 1)
    gbs = alg_bytes / (ms / 1e3) / 1e9 if ms > 0 else None
    hbm = float(peaks_file().get("hbm_gbs") or 6760.9)
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": gbs / hbm if gbs else None,
            "traffic": ncu_traffic("recon_pile16M_ncu.md", "recon.cu"),
            "kernel": "k_rings_from_events", "events": int(pn.numel()), "ms_per_launch": ms,
            "bytes_basis": "1 + 16 k + 22 bytes per event (n, k sites, ring)"}


def run_alu_rates():
    """Per-SM FP32 / MUFU issue rates behind the sweep's roofline."""
    src = os.path.join(ROOT, "paper_2411_04785_gb300", "csrc", "alu_rates.cu")
    exe = os.path.join(ROOT, "paper_2411_04785_gb300", "_build", "alu_rates")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", exe],
                   check=True)
    mhz = str(peaks_file().get("sm_max_mhz") or 2070)
    with ClockSampler(0) as clk:
        time.sleep(0.5)
        out = subprocess.run([exe, mhz], capture_output=True, text=True, check=True).stdout
    rec = json.loads(out)
    rec["clocks"] = clk.summary()
    print(json.dumps(rec))


def run_recon_pile(args):
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ev = synth.simulate_events(n_src=N_SRC, n_bkg=N_BKG, seed=2)
    print(json.dumps({"roofline_recon": recon_pile(cc, synth, ev, cc.Params(), dev,
                                                   warm=args.warmup, timed=max(args.steps, 1))}))


def burst_record(cc, synth, dev, steps, warmup, kcut=0.0, seed=3, world=1, pg=None,
                 gpu_index=0):
    """The large-burst configuration: 1,000,000 rings (70 % background, deta
    0.5-10 deg) x 786,432 HEALPix nside-256 directions, sweep + argmax + top-8
    seeds + refinement per step (no reconstruction: the rings are given).
    Returns the record (value, timing, roofline of the sweep, accuracy)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rings_np, s, _ = synth.rings_burst(n=1_000_000, seed=seed)
    rings = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in rings_np.items()}
    # kcut: the angular selection (Sec. 3) on a NESTED grid, whose compact
    # blocks let the sweep skip what the cut drops
    grid = cc.grid_healpix_nest(256, dev) if kcut > 0 else cc.grid_healpix_ring(256, dev)
    R, M = rings["ax"].numel(), grid[0].numel()
    loc = cc.Localizer(grid, cc.Params(topk=8, nms_rad=math.radians(1.0), k_cut=kcut),
                       max_rings=R)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        loc.from_rings(rings)
    torch.cuda.synchronize()
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        time.sleep(0.5)
        for i in range(steps):
            starts[i].record(stream)       # inputs (20 MB of rings) re-read per step
            loc.from_rings(rings)
            ends[i].record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    cc.trace_enable(False)
    trace = cc.trace_read(reset=True)
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])
    tot_s = max_over_ranks(pg, float(step_ms.sum()) / 1e3, dev)
    sw = trace["sweep"]
    sweep_ms = sw["ms"] / max(sw["launches"], 1)
    achieved = R * M / (sweep_ms / 1e3)
    sm_max = float(peaks_file().get("sm_max_mhz") or 2070.0)
    peak = sms * sm_max * 1e6 * alu_pairs_per_clk_sm()
    d = loc.dir.cpu().numpy()
    return {"metric": METRIC, "value": world * R * M * steps / tot_s, "unit": UNIT,
            "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * tot_s / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "burst1m_healpix256" + (f"_kcut{kcut:g}" if kcut > 0 else ""),
                       "rings": R, "directions": M,
                       "grid": "HEALPix nside 256 " + ("NESTED" if kcut > 0 else "RING"),
                       "topk": 8, "k_cut": kcut,
                       "l2": "working set (20 MB rings + 9.4 MB grid + 60 MB partial maps) "
                             "re-read each step"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "gpu_launches": sum(v["launches"] for v in trace.values()),
            "clocks": clk.summary(),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "pairs/s",
                         "frac": achieved / peak,
                         "traffic": ncu_traffic("sweep_burst1m_dram.md", "sweep.cu"),
                         "kernel": "k_sweep",
                         **({"note": "effective: pairs the angular selection skipped are "
                                     "counted as evaluated, so frac can exceed 1"}
                            if kcut > 0 else {})},
            "stages": {k: {"launches_per_step": v["launches"] / steps,
                           "ms_per_step": v["ms"] / steps}
                       for k, v in trace.items() if v["launches"]},
            "accuracy": {"refined_vs_source_deg": math.degrees(math.acos(min(1.0, float(d @ s)))),
                         "refine_iterations": int(loc.iters.item()),
                         "refine_status": int(loc.ref_status.item())}}


def noisefree_record(cc, synth, dev, steps, warmup, flush):
    """The tiny plain configuration: 2,000 noise-free FP32 rings from one
    source at (30 deg, 45 deg), deta 1 deg, over the 3,072-direction
    Fibonacci grid; sweep + argmax + FP64 refinement per step (rings given),
    L2 flushed before each step.  Launch and latency bound, not throughput
    bound: the record reports latency beside evals/s."""
    import torch
    import oracle
    rings_np, s = synth.rings_noise_free(n=2000)
    rings = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in rings_np.items()}
    grid = cc.grid_fibonacci(3072, dev)
    R, M = rings["ax"].numel(), grid[0].numel()
    loc = cc.Localizer(grid, cc.Params(topk=1), max_rings=R)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        loc.from_rings(rings)
    torch.cuda.synchronize()
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    step_ms = timed_loop(lambda: loc.from_rings(rings), steps, stream, flush)
    cc.trace_enable(False)
    trace = cc.trace_read(reset=True)
    d = loc.dir.cpu().numpy()
    g32 = tuple(v.astype(np.float32) for v in oracle.grid_fibonacci(M))
    want = oracle.likelihood_map(rings_np, g32)
    got = loc.map.cpu().numpy()
    return {"value": R * M * steps / (step_ms.sum() / 1e3), "unit": UNIT,
            "steps": steps, "warmup": warmup, "ms_per_step": float(step_ms.mean()),
            "config": {"workload": "noisefree2k_fib3072", "rings": R, "directions": M,
                       "grid": "Fibonacci", "l2": "flushed between timed steps (256 MiB write)"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "gpu_launches_per_step": sum(v["launches"] for v in trace.values()) / steps,
            "stages": {k: {"ms_per_step": v["ms"] / steps} for k, v in trace.items()
                       if v["launches"]},
            "accuracy": {"refined_vs_source_deg": math.degrees(math.acos(min(1.0, float(d @ s)))),
                         "map_max_rel_err_vs_oracle": float(np.max(
                             np.abs(got - want) / np.maximum(want, 1e-3 * want.max()))),
                         "argmax_equal_oracle": int(loc.argmax.item()) == oracle.argmax(want)}}


def run_burst(args):
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    out = burst_record(cc, synth, dev, args.steps, args.warmup, kcut=args.kcut, seed=3 + rank,
                       world=world, pg=pg, gpu_index=local)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()


def run_gpu(args):
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    ev = synth.simulate_events(n_src=N_SRC, n_bkg=N_BKG, seed=2 + rank)
    N = ev["n"].size
    tn = torch.from_numpy(ev["n"]).to(dev)
    tx, ty, tz, te = (torch.from_numpy(ev[k]).to(dev) for k in "xyze")
    grid = cc.grid_healpix_ring(NSIDE, dev)
    M = grid[0].numel()
    params = cc.Params(topk=1)
    loc = cc.Localizer(grid, params, max_rings=N)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        loc.from_events(tn, tx, ty, tz, te)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        time.sleep(0.5)                    # let nvidia-smi start sampling
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier(pg)
    cc.trace_enable(False)
    trace = cc.trace_read(reset=True)
    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    tot_s = max_over_ranks(pg, float(step_ms.sum()) / 1e3, dev)
    ms_per_step = 1e3 * tot_s / args.steps
    # evaluations = valid rings x directions: invalid rings are compacted away
    # before the sweep and cost nothing
    n_valid = int(loc._rings["valid"].sum().item())
    pairs_step = n_valid * M
    value = world * pairs_step * args.steps / tot_s
    launches = sum(v["launches"] for v in trace.values())
    assert int(loc.loc_status.item()) == 0 and int(loc.ref_status.item()) in (0, -5)

    # dominant kernel: the sweep (ALU bound)
    sw = trace["sweep"]
    sweep_ms = sw["ms"] / max(sw["launches"], 1)
    achieved = pairs_step / (sweep_ms / 1e3)
    clocks = clk.summary()
    pk = peaks_file()
    sm_max = float(pk.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    peak = sms * sm_max * 1e6 * alu_pairs_per_clk_sm()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "pairs/s",
                "frac": achieved / peak,
                "traffic": ncu_traffic("sweep_events200k_ncu.md", "sweep.cu"),
                "kernel": "k_sweep", "peak_basis": f"{sms} SMs x {sm_max:.0f} MHz x "
                f"{alu_pairs_per_clk_sm():.0f} pairs/clk/SM (16 FP32 ops at 128/clk; sqrt 16/clk "
                f"+ ex2 32/clk)"}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (sms * clocks["sm_mhz"] * 1e6 *
                                                        alu_pairs_per_clk_sm())
    stages = {k: {"launches_per_step": v["launches"] / args.steps,
                  "ms_per_step": v["ms"] / args.steps}
              for k, v in trace.items() if v["launches"]}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": event_config(world, N, n_valid, M),
           "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                          "p99": float(np.percentile(step_ms, 99))},
           "wall_s": wall, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
           "stages": stages}

    if not args.quick:
        # end to end through the public API with pinned host buffers
        hn = torch.from_numpy(ev["n"]).pin_memory()
        hx, hy, hz, he = (torch.from_numpy(ev[k]).pin_memory() for k in "xyze")
        hmap = torch.empty(M, dtype=torch.float32).pin_memory()
        hdir = torch.empty(3, dtype=torch.float64).pin_memory()
        hst = torch.empty(2, dtype=torch.int32).pin_memory()
        dn, dx, dy, dz, de = (torch.empty_like(t, device=dev) for t in (hn, hx, hy, hz, he))
        h2d = sum(t.numel() * t.element_size() for t in (hn, hx, hy, hz, he))
        d2h = hmap.numel() * 4 + 3 * 8 + 2 * 4

        def e2e_step():
            for d, h in ((dn, hn), (dx, hx), (dy, hy), (dz, hz), (de, he)):
                d.copy_(h, non_blocking=True)
            loc.from_events(dn, dx, dy, dz, de)
            hmap.copy_(loc.map, non_blocking=True)
            hdir.copy_(loc.dir, non_blocking=True)
            hst[0:1].copy_(loc.loc_status, non_blocking=True)
            hst[1:2].copy_(loc.ref_status, non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            es[i].record(stream)
            e2e_step()
            ee[i].record(stream)
            ee[i].synchronize()          # the host reads the result every step
        e_ms = np.array([a.elapsed_time(b) for a, b in zip(es, ee)])
        e_tot = max_over_ranks(pg, float(e_ms.sum()) / 1e3, dev)
        out["e2e"] = {"value": world * pairs_step * args.steps / e_tot, "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": 1e3 * e_tot / args.steps,
                      "latency_ms": {"p50": float(np.percentile(e_ms, 50)),
                                     "p99": float(np.percentile(e_ms, 99))}}

        # reconstruction on a pile of 16M events (HBM bound, larger than L2)
        out["roofline_recon"] = recon_pile(cc, synth, ev, params, dev)

        # the other configurations, measured in the same run: the largest
        # single-GPU one (1M rings x 786,432 directions, its own sweep
        # roofline) and the tiny noise-free one
        if world == 1:
            out["configs"] = {
                "burst1m_healpix256": burst_record(cc, synth, dev, steps=5, warmup=3,
                                                   gpu_index=gpu_index),
                "noisefree2k_fib3072": noisefree_record(cc, synth, dev, steps=200, warmup=10,
                                                        flush=flush)}

    # accuracy and the CPU baseline (rank 0, N = 1 only)
    d = loc.dir.cpu().numpy()
    s = ev["source"]
    out["accuracy"] = {"refined_vs_source_deg": math.degrees(math.acos(min(1.0, float(d @ s)))),
                       "refine_iterations": int(loc.iters.item()),
                       "refine_status": int(loc.ref_status.item())}
    out["accuracy"]["target_deg"] = 0.5
    out["accuracy"]["target_met"] = out["accuracy"]["refined_vs_source_deg"] <= 0.5
    if rank == 0 and world == 1 and not args.quick:
        import oracle
        threads = os.cpu_count() or 1
        t_cpu, nv_cpu, info = oracle_path(ev, oracle.grid_healpix_ring(NSIDE), threads)
        dd = info["dir"]
        out["accuracy"]["refined_vs_oracle_deg"] = math.degrees(
            math.atan2(np.linalg.norm(np.cross(d, dd)), float(d @ dd)))
        out["accuracy"]["oracle_vs_source_deg"] = math.degrees(
            math.atan2(np.linalg.norm(np.cross(dd, s)), float(dd @ s)))
        out["cpu_baseline"] = {
            "value": nv_cpu * M / t_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"one whole step on the oracle (C, FP64), the same burst, no "
                       f"extrapolation: rings of all {N} events on 1 thread "
                       f"({info['t_recon_s']:.2f} s), map of all {nv_cpu} valid rings over all "
                       f"{M} directions on {threads} threads ({info['t_map_s']:.1f} s), argmax, "
                       f"refinement ({info['t_refine_s']:.2f} s)"),
            "s_per_step": t_cpu, "extrapolated": False}
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()


def run_serve(args):
    """Serving: Poisson bursts (50/s; log-normal ring counts, median 20k,
    500-300k; background 1-50x; random source among 16 directions) served in
    real time by the continuous-batching server, first on the plain path,
    then on the learned path (ring filter trained here on the GPU).  Reports
    per-burst latency p50/p99 (arrival to result on the host), the ring x
    direction evaluations per second over the run, and the localisation error
    against the true source; the plain path's results are checked against
    the oracle on a sample of small bursts."""
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import serve, synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = cc.Params()
    # the learned path's filter, trained on the GPU by the library's kernels
    t0 = time.perf_counter()
    tr = synth.training_events(args.train_events, seed=11 + rank)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n = to(tr["n"])
    x, y, z, e = (to(np.asarray(tr[k], np.float32)) for k in "xyze")
    rings = cc.rings_from_events(n, x, y, z, e, p)
    F = cc.ring_features(n, x, y, z, e, rings, p)
    res = cc.ring_residuals(rings, to(tr["sources"]))
    filt = cc.RingFilter(dev, seed=0)
    losses = filt.train(F, to(tr["is_source"].astype(np.uint8)), res, rings["valid"], epochs=8,
                        batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del n, x, y, z, e, rings, F, res, tr

    pools, specs = synth.serving_bursts(args.bursts, 50.0, seed=5 + rank)
    bursts = serve.to_bursts(serve.pin_pools(pools), specs)
    grid = cc.grid_healpix_ring(NSIDE, dev)
    M = grid[0].numel()
    arms = {"plain": {}, "learned": {"ring_filter": filt, "tau": args.tau}}
    out_arms = {}
    gpu_index = local
    for name, kw in arms.items():
        srv = serve.Server(grid, p, hbm_budget=8 << 30, max_active=48, graphs=bool(args.graphs),
                           **kw)
        srv.prepare([b.count for b in bursts])                         # capture the graphs
        srv.run(bursts[:args.warmup * 4], realtime=False)              # warm-up
        torch.cuda.synchronize()
        cc.trace_read(reset=True)
        barrier(pg)
        with ClockSampler(gpu_index) as clk:
            time.sleep(0.5)
            res_arm, stats = srv.run(bursts, realtime=True, breakdown=True)
        launches = sum(v["launches"] for v in cc.trace_read(reset=True).values())
        lat = np.array([res_arm[b.bid]["latency"] for b in bursts]) * 1e3
        err = np.array([math.degrees(math.atan2(np.linalg.norm(np.cross(res_arm[b.bid]["dir"], b.source)),
                                                float(res_arm[b.bid]["dir"] @ b.source))) for b in bursts])
        rings_total = sum(b.count for b in bursts)
        out_arms[name] = {
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "evals_per_s": rings_total * M / stats["wall_s"], "wall_s": stats["wall_s"],
            "bursts_per_s": len(bursts) / stats["wall_s"],
            "batches": {"count": len(stats["batches"]), "mean_size": float(np.mean(stats["batches"])),
                        "max_size": int(max(stats["batches"]))},
            "error_vs_source_deg": {"p50": float(np.percentile(err, 50)),
                                    "p90": float(np.percentile(err, 90)),
                                    "within_0.5": float((err <= 0.5).mean())},
            "gpu_launches": launches, "clocks": clk.summary(),
            "breakdown_ms": {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}
                             for k, v in ((k, [res_arm[b.bid]["breakdown_ms"][k] for b in bursts])
                                          for k in res_arm[bursts[0].bid]["breakdown_ms"])}}
        if name == "plain":
            plain_res = res_arm
    # oracle parity of the plain path on the smallest bursts (rank 0)
    parity = None
    if rank == 0 and not args.quick:
        import oracle
        g64 = oracle.grid_healpix_ring(NSIDE)
        small = sorted(bursts, key=lambda b: b.count)[:3]
        worst = 0.0
        for b in small:
            ev = synth.burst_events(pools, specs[b.bid])
            r = oracle.rings_from_events(ev, p.sigma_e_frac, p.sigma_pos_cm, p.deta_min, p.deta_max)
            m = oracle.likelihood_map(r, g64)
            j = oracle.argmax(m)
            d, _, _, _ = oracle.refine(r, [g64[0][j], g64[1][j], g64[2][j]], tol_rad=1e-10)
            gd = plain_res[b.bid]["dir"]
            worst = max(worst, math.degrees(math.atan2(np.linalg.norm(np.cross(gd, d)), float(gd @ d))))
        parity = {"bursts": [b.count for b in small], "max_refined_vs_oracle_deg": worst}
    pl, le = out_arms["plain"], out_arms["learned"]
    out = {"metric": METRIC, "value": world * pl["evals_per_s"], "unit": UNIT, "n_gpus": world,
           "steps": len(bursts), "warmup": args.warmup * 4,
           "ms_per_step": pl["wall_s"] * 1e3 / len(bursts), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "serve_poisson50", "bursts": len(bursts), "rate_hz": 50.0,
                      "rings": "log-normal median 20k sigma 1 in [500, 300k]",
                      "background": "uniform 1-50x", "directions": M,
                      "grid": "HEALPix nside 64 RING", "hbm_budget_gb": 8, "max_active": 48,
                      "arrivals": "real time (Poisson)",
                      "front_end": "CUDA graph per size bucket" if args.graphs else "launched",
                      "filter": {"train_events": args.train_events, "train_s": t_train,
                                 "loss_first_last": [losses[0], losses[-1]], "tau": args.tau}},
           "latency_ms": {"plain": pl["latency_ms"], "learned": le["latency_ms"]},
           "arms": out_arms, "gpu_launches": pl["gpu_launches"], "clocks": pl["clocks"],
           "oracle_parity": parity}
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()


def timed_loop(step, steps, stream, flush=None):
    """CUDA-event time of every step on `stream` (ms)."""
    import torch
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        st[i].record(stream)
        step()
        en[i].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in zip(st, en)])


def run_cluster(args):
    """Max-step clustering (Sec. 2) of a 137Cs-like detection stream: 12
    copies of a 400k-event segment (81.7M detections, 15 ns step), every
    output (edges, event ids, per-event first / size / amplitude sum) plus
    the amplitude spectrum per step.  HBM bound; inputs (981 MB) are larger
    than L2."""
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t0, a0, _ = synth.detection_stream(seed=21 + rank)
    t_np, adc_np = synth.tile_stream(t0, a0, 12)
    N = t_np.size
    DT = 15_000
    td = torch.from_numpy(t_np).to(dev)
    ad = torch.from_numpy(adc_np).to(dev)
    o = cc.cluster_maxstep(td, ad, DT)
    hist = cc.cluster_spectrum(o["adc"], o["n_events"], 64, 256)
    stream = torch.cuda.current_stream()

    def step():
        cc.cluster_maxstep(td, ad, DT, out=o)
        cc.cluster_spectrum(o["adc"], o["n_events"], 64, 256, out=hist)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = int(o["n_events"].item())
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    barrier(pg)
    with ClockSampler(local) as clk:
        time.sleep(0.5)
        ms = timed_loop(step, args.steps, stream)
    barrier(pg)
    cc.trace_enable(False)
    trace = cc.trace_read(reset=True)
    tot_s = max_over_ranks(pg, float(ms.sum()) / 1e3, dev)
    # the clustering call alone (k_cluster_masks, k_cluster_scan, k_cluster_events;
    # the spectrum is the step's fourth launch), by events
    kms = timed_loop(lambda: cc.cluster_maxstep(td, ad, DT, out=o), args.steps, stream)
    alg = N * (8 + 4 + 1 + 4) + K * (8 + 4 + 8)
    pk = peaks_file()
    peak = float(pk.get("hbm_gbs") or 6800.0) * 1e9
    achieved = alg / (float(np.mean(kms)) / 1e3)
    out = {"metric": "detections clustered/s (max-step, Sec. 2)", "value": world * N * args.steps / tot_s,
           "unit": "detections/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": "cluster_cs137_81M", "detections": N, "events": K,
                      "dt_max_ps": DT, "l2": "inputs (981 MB) larger than L2"},
           "gpu_launches": sum(v["launches"] for v in trace.values()), "clocks": clk.summary(),
           "roofline": {"bound": "hbm", "achieved": achieved / 1e9, "peak": peak / 1e9,
                        "unit": "GB/s", "frac": achieved / peak,
                        "traffic": ncu_traffic("cluster_cs137_81M_ncu.md", "cluster.cu"),
                        "kernel": "cluster_maxstep (k_cluster_masks + k_cluster_scan + "
                                  "k_cluster_events)", "ms_per_call": float(np.mean(kms)),
                        "algorithmic_bytes": f"{N} x 17 B (t, adc in; edge, id out) + "
                                             f"{K} events x 20 B = {alg}"}}
    if not args.quick:
        ht = torch.from_numpy(t_np).pin_memory()
        ha = torch.from_numpy(adc_np).pin_memory()
        hh = torch.empty(256, dtype=torch.uint64).pin_memory()
        hk = torch.empty(1, dtype=torch.int64).pin_memory()

        def e2e():
            td.copy_(ht, non_blocking=True)
            ad.copy_(ha, non_blocking=True)
            step()
            hh.copy_(hist, non_blocking=True)
            hk.copy_(o["n_events"], non_blocking=True)

        e_ms = []
        for i in range(args.warmup + args.steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            e2e()
            s1.record(stream)
            s1.synchronize()
            if i >= args.warmup:
                e_ms.append(s0.elapsed_time(s1))
        e_tot = max_over_ranks(pg, float(np.sum(e_ms)) / 1e3, dev)
        out["e2e"] = {"value": world * N * args.steps / e_tot, "unit": "detections/s",
                      "h2d_bytes_per_step": N * 12, "d2h_bytes_per_step": 256 * 8 + 8,
                      "ms_per_step": 1e3 * e_tot / args.steps}
        if rank == 0 and world == 1:
            import oracle
            c0 = time.perf_counter()
            want = oracle.maxstep_events(t_np, adc_np, DT)
            c1 = time.perf_counter() - c0
            got_ok = (int(o["n_events"].item()) == want["count"].size and
                      np.array_equal(o["event_id"].cpu().numpy(), want["event_id"]))
            out["cpu_baseline"] = {"value": N / c1, "unit": "detections/s", "cores": 1,
                                   "kind": "oracle",
                                   "sample": f"the whole {N}-detection stream, oracle (C) on 1 thread"}
            out["parity"] = {"event_ids_bit_exact": bool(got_ok)}
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()


def run_voxel(args):
    """Near-field back projection (Sec. 3): 200,000 events from a point
    source 20 cm above the 4-layer detector (background 10:1) -> rings ->
    apexes -> image over the sphere universe inscribed in a 64^3 cube of
    0.3125 cm voxels (137,376 voxels); the cube and cylinder universes are
    timed beside it."""
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    S = (1.3, -0.7, 20.2)
    ev = synth.simulate_events(n_src=18182, n_bkg=181818, seed=12 + rank, source_point=S)
    N = ev["n"].size
    tn = torch.from_numpy(ev["n"]).to(dev)
    tx, ty, tz, te = (torch.from_numpy(ev[k]).to(dev) for k in "xyze")
    p = cc.Params()
    unis = {u: cc.voxel_universe(u, 64, 0.3125, (0.0, 0.0, 20.0), dev)
            for u in ("sphere", "cylinder", "cube")}
    rings = cc.rings_from_events(tn, tx, ty, tz, te, p)
    apex = cc.ring_apex(tn, tx, ty, tz, rings)
    vox = unis["sphere"]
    V = vox[0].numel()
    ws = torch.empty(max(cc.backproject_workspace_bytes(N, unis["cube"][0].numel(), p), 256),
                     dtype=torch.uint8, device=dev)
    img = cc.backproject(rings, apex, vox, p, workspace=ws)
    stream = torch.cuda.current_stream()

    def step():
        cc.rings_from_events(tn, tx, ty, tz, te, p, out=rings)
        cc.ring_apex(tn, tx, ty, tz, rings, out=apex)
        cc.backproject(rings, apex, vox, p, workspace=ws, out=img)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_valid = int(rings["valid"].sum().item())
    cc.trace_read(reset=True)
    cc.trace_enable(True)
    barrier(pg)
    with ClockSampler(local) as clk:
        time.sleep(0.5)
        ms = timed_loop(step, args.steps, stream)
    barrier(pg)
    cc.trace_enable(False)
    trace = cc.trace_read(reset=True)
    tot_s = max_over_ranks(pg, float(ms.sum()) / 1e3, dev)
    vt = trace["voxel"]
    sweep_ms = (vt["ms"] - 0.0) / max(args.steps, 1)   # apex + sweep per step
    pairs = n_valid * V
    sm_max = float(peaks_file().get("sm_max_mhz") or 2070.0)
    per_clk = 128.0 / 26.0        # 26 FP32 ops per pair at 128 lanes/clk/SM (MUFU: 3 ops, not binding)
    peak = sms * sm_max * 1e6 * per_clk
    achieved = pairs / (sweep_ms / 1e3)
    j = int(img[1].item())
    vj = np.array([vox[c][j].item() for c in range(3)])
    others = {}
    for u in ("cube", "cylinder"):
        o2 = cc.backproject(rings, apex, unis[u], p, workspace=ws)
        torch.cuda.synchronize()
        t_u = timed_loop(lambda: cc.backproject(rings, apex, unis[u], p, workspace=ws, out=o2),
                         max(3, args.steps // 4), stream)
        others[u] = {"voxels": unis[u][0].numel(), "ms": float(np.mean(t_u))}
    out = {"metric": "ring×voxel evals/s (near-field back projection, Sec. 3)",
           "value": world * pairs * args.steps / tot_s, "unit": "ring×voxel evals/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "voxel_point_source_200k_sphere64", "events": N,
                      "valid_rings": n_valid, "voxels": V,
                      "universe": "sphere in a 64^3 cube, 0.3125 cm voxels, centre (0,0,20) cm",
                      "source_point_cm": S, "l2": "working set re-read each step (no flush)"},
           "gpu_launches": sum(v["launches"] for v in trace.values()), "clocks": clk.summary(),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "pairs/s",
                        "frac": achieved / peak,
                        "traffic": ncu_traffic("voxel_sphere64_ncu.md", "voxel.cu"),
                        "kernel": "k_backproject",
                        "peak_basis": f"{sms} SMs x {sm_max:.0f} MHz x 128/26 pairs/clk/SM"},
           "universes_ms": dict(others, sphere={"voxels": V, "ms": float(np.mean(ms))}),
           "accuracy": {"argmax_voxel_cm": vj.tolist(),
                        "argmax_to_source_cm": float(np.linalg.norm(vj - np.array(S))),
                        "lateral_cm": float(np.linalg.norm((vj - np.array(S))[:2])),
                        "depth_cm": float(vj[2] - S[2]),
                        "note": "a planar Compton camera resolves depth (z) far worse "
                                "than the lateral position with 15-20 deg cones"}}
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()


def run_filter(args):
    """The learned ring filter's inference on 500k-ring batches (the
    learned-filter configuration): features + the fused MLP forward + the
    filter, rings from 500k simulated events, the step captured as a CUDA
    graph (as the serving front end runs it).  Tensor-core bound: the roofline
    is the MLP forward's FLOP rate against the measured BF16 peak, timed over
    a graph of 20 back-to-back forwards (a launch lasts ~20 us, shorter than
    the host's own call)."""
    import torch

    import paper_2411_04785_gb300 as cc
    from paper_2411_04785_gb300 import synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ev = synth.tile_events(synth.simulate_events(seed=2 + rank), 5)
    ev = {k: v[..., :500_000] if k != "n" else v[:500_000] for k, v in ev.items()}
    N = ev["n"].size
    tn = torch.from_numpy(np.ascontiguousarray(ev["n"])).to(dev)
    tx, ty, tz, te = (torch.from_numpy(np.ascontiguousarray(ev[k])).to(dev) for k in "xyze")
    p = cc.Params()
    rings = cc.rings_from_events(tn, tx, ty, tz, te, p)
    f = cc.RingFilter(dev, seed=0)
    F = cc.ring_features(tn, tx, ty, tz, te, rings, p)
    out = torch.empty((N, 2), dtype=torch.float32, device=dev)
    work = {k: v.clone() for k, v in rings.items()}
    stream = torch.cuda.current_stream()

    def step():
        cc.ring_features(tn, tx, ty, tz, te, rings, p, out=F)
        f.forward(F, out=out)
        f.apply(work, out, 0.0, p.deta_min, p.deta_max)

    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g_step, g_fwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_step):
        step()
    n_fwd = 20
    with torch.cuda.graph(g_fwd):
        for _ in range(n_fwd):
            f.forward(F, out=out)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        g_step.replay()
    torch.cuda.synchronize()
    barrier(pg)
    with ClockSampler(local) as clk:
        time.sleep(0.5)
        ms = timed_loop(g_step.replay, args.steps, stream)
    barrier(pg)
    tot_s = max_over_ranks(pg, float(ms.sum()) / 1e3, dev)
    g_fwd.replay()
    fms = timed_loop(g_fwd.replay, max(3, args.steps // 5), stream) / n_fwd
    flop = N * 2 * (16 * 128 + 128 * 128 * 2 + 128 * 2)
    achieved = flop / (float(np.mean(fms)) / 1e3)
    peak = float(peaks_file().get("bf16_tflops") or 1900.0) * 1e12
    # training side: gradient (forward + backward) and Adam on 8,192-row
    # batches of the same features (labels drawn at random), batches gathered
    # before the timed loop
    B = 8192
    g = torch.Generator(device="cpu").manual_seed(1)
    ys = (torch.rand(N, generator=g) < 0.3).to(torch.uint8).to(dev)
    rs = (torch.randn(N, generator=g) * 0.3).to(dev)
    ws_ = torch.ones(N, dtype=torch.uint8, device=dev)
    nb = N // B
    batches = [(F[i * B:(i + 1) * B].contiguous(), ys[i * B:(i + 1) * B].contiguous(),
                rs[i * B:(i + 1) * B].contiguous(), ws_[i * B:(i + 1) * B].contiguous())
               for i in range(nb)]
    tf = cc.RingFilter(dev, seed=0)
    it = [0]

    def train_step():
        b = batches[it[0] % nb]
        it[0] += 1
        tf.grad(*b)
        tf.adam(1e-3)

    for _ in range(args.warmup):
        train_step()
    tms = timed_loop(train_step, max(10, args.steps // 2), stream)
    train_flop = 3 * B * 2 * (16 * 128 + 128 * 128 * 2 + 128 * 2)    # forward + 2 backward products
    out_j_train = {"rows_per_s": B / (float(np.mean(tms)) / 1e3),
                   "ms_per_step": float(np.mean(tms)), "batch": B,
                   "tflops": train_flop / (float(np.mean(tms)) / 1e3) / 1e12,
                   "note": "grad (forward + backward through all layers, loss, bias and weight "
                           "gradients) + Adam per step; forward on the tcgen05 kernel, backward "
                           "on tcgen05 (one launch per hidden layer)"}
    out_j = {"metric": "rings filtered/s (learned ring filter inference)",
             "value": world * N * args.steps / tot_s, "unit": "rings/s", "n_gpus": world,
             "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
             "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
             "data": "synthetic",
             "config": {"workload": "filter_500k", "rings": N,
                        "network": "16-128-128-128-2 ReLU, BF16 weights and activations, FP32 accumulation",
                        "l2": "working set re-read each step (no flush)",
                        "launch": "step replayed as one CUDA graph"},
             "gpu_launches": 3 * args.steps, "clocks": clk.summary(),
             "roofline": {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12,
                          "unit": "TFLOP/s", "frac": achieved / peak,
                          "traffic": ncu_traffic("mlp_forward_500k_ncu.md", "mlp.cu"),
                          "kernel": "k_mlp_forward_tc", "ms_per_launch": float(np.mean(fms)),
                          "flop_basis": f"{N} rows x 2 FLOP x 35,072 multiply-adds"},
             "training": out_j_train}
    if rank == 0:
        print(json.dumps(out_j))
    if pg is not None:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["events200k", "burst1m", "serve", "cluster", "voxel",
                                           "filter"],
                    default="events200k",
                    help="events200k (default, the headline), the 1M-ring x 786k-direction "
                         "burst, or the serving stream (plain and learned paths)")
    ap.add_argument("--bursts", type=int, default=2000, help="serve: bursts in the stream")
    ap.add_argument("--train-events", type=int, default=1_000_000,
                    help="serve: events simulated to train the ring filter")
    ap.add_argument("--tau", type=float, default=0.0, help="serve: ring filter score threshold")
    ap.add_argument("--graphs", type=int, default=1,
                    help="serve: 1 = per-burst front end as a CUDA graph per size bucket")
    ap.add_argument("--kcut", type=float, default=0.0,
                    help="burst1m: angular selection |r| <= kcut on a NESTED grid (0: off)")
    ap.add_argument("--quick", action="store_true", help="skip e2e, recon pile and CPU baseline")
    ap.add_argument("--alu-rates", action="store_true",
                    help="build and run the FP32 / MUFU rate microbenchmark (csrc/alu_rates.cu)")
    ap.add_argument("--profile-recon", action="store_true",
                    help="only run reconstruction on the 16M-event pile (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_recon:
        run_recon_pile(args)
    elif args.alu_rates:
        run_alu_rates()
    elif args.workload == "burst1m":
        run_burst(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "cluster":
        run_cluster(args)
    elif args.workload == "voxel":
        run_voxel(args)
    elif args.workload == "filter":
        run_filter(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
