#!/usr/bin/env python3
"""Benchmark of the GB300 inverse ray-shooting path (one JSON line on stdout).

Workload (default, the largest single-GPU configuration): 1e8 equal-mass point lenses
(float32 masses of 1) uniform in a disc (kappa_* = 0.5, kappa_c = 0, gamma = 0.5), an
8192 x 8192 regular ray grid, a 4096 x 4096 uint32 source map.  A whole map takes about
20 minutes, so one step shoots a central block of grid rows that fills whole waves of
CTAs: zero the counts, shoot the block (deflection over all 1e8 lenses, lens map,
binning: one kernel, plus the certified re-evaluation), normalise to mu (one kernel).
Metric: lens-ray interactions per second (rays x lenses / time), and the same as a
fraction of the FP32 peak with the paper's 10 flops per interaction.  The other
configurations (100, 1e4 and 1e6 lenses, the 64-field batch) are reported as
sub-objects with their own roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

--impl reference times the FP64 CPU oracle (the reference arm) on bounded samples of
the same workload.  Under torchrun (--mode sharded, the default) every rank shoots one
whole-wave block of rows of the same map and the count maps are summed with one NCCL
all_reduce per step (weak scaling: the rows per rank stay fixed); --mode realisations
gives every rank its own lens realisation instead, with no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import rs_inputs as ri  # noqa: E402

FLOPS_PER_INTERACTION = 10  # the paper's Appendix A count
METRIC = "lens-ray interactions/s"
L2_FLUSH_BYTES = 512 << 20


def workload(name: str, seed: int):
    if name == "n1e4":
        return ri.n1e4_field(seed=seed)
    if name == "tiny":
        return ri.tiny_field(seed=seed)
    if name == "n1e6":
        return ri.n1e6_salpeter_field(seed=seed)
    if name == "n1e8":
        return ri.n1e8_field(seed=seed)
    raise SystemExit(f"unknown workload {name}")


def workload_config(spec, name):
    return {
        "workload": spec.name,
        "n_lens": spec.n_lens,
        "masses": ("unit (equal-mass kernels)" if spec.masses is None else
                   "float32, all 1 (stored; equal-mass kernels)" if bool(np.all(spec.masses == 1.0)) else
                   "per-lens float32"),
        "kappa_star": round(spec.kappa_star, 6), "kappa_c": spec.kappa_c, "gamma": spec.gamma,
        "ray_grid": list(spec.grid.n), "map": list(spec.window.npix),
        "rays_per_step": spec.grid.n_rays,
        "interactions_per_step": spec.interactions,
        "l2": "flushed between timed steps (512 MiB write)",
        "name": name,
    }


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------------- helpers

def kernel_source_hash():
    """Hash of the shoot kernel's source code with comments and blank space removed (a comment edit keeps
    a profiled traffic figure valid; any code change invalidates it)."""
    import re
    h = hashlib.sha256()
    for f in ("rs_device.cuh", "rs_shoot.cu"):
        with open(os.path.join(ROOT, "paper_0905_2453_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name):
    """DRAM bytes per launch of the shoot kernel from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split("#", 1)[0].split()
            if len(parts) >= 3 and parts[0] == workload_name and parts[1] == want:
                return float(parts[2])
    return None


def peaks(device_index: int):
    import torch
    props = torch.cuda.get_device_properties(device_index)
    sms = props.multi_processor_count
    max_mhz = None
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        try:
            max_mhz = float(json.load(open(mp)).get("sm_max_mhz"))
        except Exception:
            max_mhz = None
    if not max_mhz:
        max_mhz = 2070.0
    return sms, max_mhz


def fp32_peak_tflops(sms, mhz):
    # 128 FP32 lanes per SM, one fused multiply-add (2 flops) per lane per clock
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# --------------------------------------------------------------------------------------------- oracle arm

def oracle_rate(spec, target_s: float, max_rows=None):
    """Time the FP64 oracle on a block of grid rows sized to ~target_s seconds; returns a dict."""
    import oracle
    oracle.build()
    n0 = int(spec.grid.n[0])
    t = time.perf_counter()
    oracle.shoot_field(spec, rows=(0, 2))
    dt = max(time.perf_counter() - t, 1e-4)
    per_row = dt / 2
    rows = max(1, min(int(spec.grid.n[1]), int(target_s / per_row)))
    if max_rows:
        rows = min(rows, max_rows)
    j0 = (int(spec.grid.n[1]) - rows) // 2
    t = time.perf_counter()
    oracle.shoot_field(spec, rows=(j0, j0 + rows))
    dt = time.perf_counter() - t
    inter = rows * n0 * spec.n_lens
    return {"value": inter / dt, "seconds": dt, "rows": rows, "rays": rows * n0,
            "interactions": inter, "cores": oracle.num_threads()}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step a bounded sample of the workload
    (central grid rows when a row is cheap enough, else random rays of the grid, new ones every step)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec = workload(args.workload, seed=0)
    per_step = min(1.0, 150.0 / max(1, args.steps + args.warmup))
    n0, n1 = int(spec.grid.n[0]), int(spec.grid.n[1])
    if n0 * spec.n_lens <= 2.5e8 * per_step / 4:
        calib = oracle_rate(spec, per_step)
        rows, cores = calib["rows"], calib["cores"]

        def one(k):
            j0 = (k * rows) % max(1, n1 - rows + 1)
            oracle.shoot_field(spec, rows=(j0, j0 + rows))
            return rows * n0

        sample = f"{rows} grid rows ({rows * n0} rays) x {spec.n_lens} lenses per step"
    else:
        cal = oracle_trace_rate(spec, 8, seed=5)
        n_rays, cores = max(8, int(per_step / max(cal["seconds"] / 8, 1e-9))), cal["cores"]

        def one(k):
            oracle.trace_field(spec, ri.sample_rays(spec.grid, n_rays, seed=1000 + k))
            return n_rays

        sample = f"{n_rays} random rays of the {n0} x {n1} grid x {spec.n_lens} lenses per step (new rays each step)"
    for k in range(args.warmup):
        one(-1 - k)
    t0 = time.perf_counter()
    rays = sum(one(k) for k in range(args.steps))
    dt = time.perf_counter() - t0
    value = rays * spec.n_lens / dt
    cfg = workload_config(spec, args.workload)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                         "sample": sample + ", FP64 oracle, OpenMP over rays"},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gflops_equiv": value * FLOPS_PER_INTERACTION / 1e9,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------- our arm

FULL_LIMIT = 2e12  # grids of at most this many interactions are shot whole per step

STEP_RATE_SLACK = 0.05  # rate a shape may give up for a smaller whole-wave step


def headline_rows(rs, spec, field, sms, stream, launch_shape=None):
    """Rows [r0, r1) one step shoots, the launch shape and a description.

    Grids of at most FULL_LIMIT interactions are shot whole.  Larger ones are shot as the central block of
    the fewest rows that fill whole waves of CTAs (every CTA of the block runs at once, so the block's rate
    is the full grid's steady state); the launch shape is the tuned best or, among the shapes within
    STEP_RATE_SLACK of its rate, the one whose whole wave takes the fewest rows (every shape gives bitwise the
    same counts).  On the 8192-column grid of the 1e8-lens field a 3-CTA-per-SM shape fills whole waves only
    with 228 rows (four waves, about 35 s a step) against 76 rows (two waves, about 12 s) at two CTAs per SM,
    for a rate a few percent higher: the shorter step is kept unless the larger unit is faster by more."""
    from paper_0905_2453_gb300 import tune
    n_lens, weighted = field.info()
    if launch_shape:
        shape = parse_shape(launch_shape)
        rs.rs_set_launch_config(weighted, *shape)
        rates = {}
    else:
        shape = tuple(tune.autotune(field, spec.grid, spec.window, stream=stream)[:4])
        rates = tune.shape_rates(field, spec.grid)
    n0, n1 = int(spec.grid.n[0]), int(spec.grid.n[1])
    if spec.interactions <= FULL_LIMIT:
        return 0, n1, shape, "whole grid"

    def unit_of(sh):
        occ = rs.rs_launch_occupancy(weighted, *sh)
        return tune.wave_rows(n0, sh[0], sh[1], sms, occ), occ

    shape = choose_step_shape(shape, rates, lambda sh: unit_of(sh)[0])
    b, r = shape[0], shape[1]
    rs.rs_set_launch_config(weighted, *shape)
    unit, occ = unit_of(shape)
    warps = b // 32
    r0 = (n1 - unit) // 2 // warps * warps
    ctas = -(-n0 // (32 * r)) * (unit // warps)
    note = (f"central rows [{r0}, {r0 + unit}) of the {n0} x {n1} grid: {ctas} CTAs of {b} threads = "
            f"{ctas // (occ * sms)} whole wave(s) of {occ} CTAs x {sms} SMs")
    return r0, r0 + unit, shape, note


def choose_step_shape(best_shape, rates, unit_rows, slack=STEP_RATE_SLACK):
    """Among best_shape and the shapes rated ({"BxRxTxM": interactions/s}) within slack of it, the one whose
    whole-wave unit (unit_rows(shape)) takes the fewest rows; equal units go to the higher rate."""
    def name(sh):
        return "x".join(str(v) for v in sh)
    best = rates.get(name(best_shape))
    cands = [tuple(best_shape)]
    if best:
        cands += [parse_shape(k) for k, v in rates.items() if v >= (1 - slack) * best]
    return min(cands, key=lambda sh: (unit_rows(sh), -rates.get(name(sh), 0.0)))


def tune_for(rs, spec, stream):
    """Set (and return) the tuner's launch shape for spec's field, mass mode and grid (cached after the first
    time)."""
    from paper_0905_2453_gb300 import tune
    f = rs.Field.from_spec(spec, stream)
    try:
        return tuple(tune.autotune(f, spec.grid, spec.window, stream=stream)[:4])
    finally:
        f.close()


def parse_shape(text):
    """'128x8x512x2' (threads x rays per thread x lens tile x resident CTAs per SM; defaults 256 and 2)
    -> (128, 8, 512, 2)."""
    v = [int(x) for x in text.split("x")]
    return (v[0], v[1], v[2] if len(v) > 2 else 256, v[3] if len(v) > 3 else 2)


def oracle_sample_rate(spec, target_s: float):
    """The FP64 oracle on a bounded sample of the workload: whole central grid rows when one row takes at
    most target_s / 4, else random rays of the grid (per-ray evaluation), sized to about target_s."""
    one_row = int(spec.grid.n[0]) * spec.n_lens
    if one_row <= 2.5e8 * target_s / 4:
        r = oracle_rate(spec, target_s)
        r["sample"] = (f"{r['rows']} central grid rows ({r['rays']} rays) x {spec.n_lens} lenses, "
                       f"{r['seconds']:.1f} s, FP64 OpenMP over rays")
        return r
    cal = oracle_trace_rate(spec, 16, seed=5)
    n = max(16, int(target_s / max(cal["seconds"] / 16, 1e-9)))
    r = oracle_trace_rate(spec, n)
    r["sample"] = (f"{n} random rays of the {spec.grid.n[0]} x {spec.grid.n[1]} grid x {spec.n_lens} lenses, "
                   f"{r['seconds']:.1f} s, FP64 OpenMP over rays")
    return r


def roofline_entry(interactions, seconds, sms, max_mhz, traffic=None):
    peak = fp32_peak_tflops(sms, max_mhz)
    achieved = interactions * FLOPS_PER_INTERACTION / seconds / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic}


def run_ours(args):
    import torch
    import paper_0905_2453_gb300 as rs

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("CUDA device required for --impl ours")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # sharded (default): one map per step whose rows are split over the ranks, the count maps summed by one
    # NCCL all_reduce; realisations: every rank shoots its own realisation of the workload, no collective
    sharded = args.mode == "sharded"
    spec = workload(args.workload, seed=0 if sharded else rank)
    stream = torch.cuda.current_stream(device)
    field = rs.Field.from_spec(spec, stream)
    sms, max_mhz = peaks(local)
    r0, r1, shape, rows_note = headline_rows(rs, spec, field, sms, stream, args.launch_shape)
    if dist is not None and sharded:
        # rank 0's rows and launch shape hold on every rank: the ranks' blocks must tile one block of the map
        # (each rank's tuner times its own GPU and could, in a close call, rank two shapes the other way round)
        chosen = [(r0, r1, tuple(shape), rows_note)]
        dist.broadcast_object_list(chosen, src=0)
        r0, r1, shape, rows_note = chosen[0]
        rs.rs_set_launch_config(field.info()[1], *shape)
    from paper_0905_2453_gb300 import tune
    from paper_0905_2453_gb300.shard import device_row_shooter, shoot_sharded
    rates_headline = {} if args.launch_shape else tune.shape_rates(field, spec.grid)
    npix = (int(spec.window.npix[1]), int(spec.window.npix[0]))
    counts = torch.zeros(npix, dtype=torch.int32, device=device)
    oow = torch.zeros(1, dtype=torch.int64, device=device)
    mu = torch.empty(npix, dtype=torch.float32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    n0, n1 = int(spec.grid.n[0]), int(spec.grid.n[1])
    whole = r0 == 0 and r1 == n1
    if sharded:
        # the step's rows: the whole grid (split over the ranks: strong scaling), or one whole-wave unit per rank
        # (weak scaling of one sharded block)
        warps = shape[0] // 32
        total_rows = n1 if whole else min(n1, world * (r1 - r0))
        row0 = 0 if whole else (n1 - total_rows) // 2 // warps * warps
        shooter = device_row_shooter(field, spec.grid, spec.window, stream)
        rows_note = (rows_note if world == 1 else
                     f"rows [{row0}, {row0 + total_rows}) split over {world} ranks, counts summed by NCCL all_reduce")
        inter_step = total_rows * n0 * spec.n_lens      # the whole job's interactions per step
        rays_step = total_rows * n0
    else:
        inter_step = (r1 - r0) * n0 * spec.n_lens       # per rank
        rays_step = (r1 - r0) * n0

    def shoot():
        if sharded:
            shoot_sharded(shooter, total_rows, counts, oow, rank, world, row_begin=row0)
        else:
            rs.rs_shoot_rows(field.handle, spec.grid, r0, r1, spec.window, counts, oow, stream)

    def step():
        counts.zero_()
        oow.zero_()
        shoot()
        rs.rs_magnification(counts, spec.grid, spec.window, mu, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(device)
    clocks.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)  # evict the previous step's lines from L2 (outside the timed spans)
        e = ev[k]
        e[0].record(stream)
        counts.zero_()
        oow.zero_()
        e[1].record(stream)
        shoot()
        e[2].record(stream)
        rs.rs_magnification(counts, spec.grid, spec.window, mu, stream)
        e[3].record(stream)
    torch.cuda.synchronize(device)
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    shoot_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3)
    shoot_avg_s = max_over_ranks(statistics.mean(shoot_ms) / 1e3)
    status = field.status()
    if status != rs.RS_OK:
        raise SystemExit(f"device reported status {status}")
    conserved = int(counts.sum(dtype=torch.int64).item()) + int(oow.item()) == rays_step
    value = inter_step * args.steps * (1 if sharded else world) / total_s

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_xy = torch.from_numpy(np.ascontiguousarray(spec.lens_xy)).pin_memory()
        h_m = None if spec.masses is None else torch.from_numpy(spec.masses).pin_memory()
        h_mu = torch.empty(npix, dtype=torch.float32).pin_memory()
        h_oow = torch.empty(1, dtype=torch.int64).pin_memory()

        def e2e_step():
            f = rs.Field(h_xy.numpy(), None if h_m is None else h_m.numpy(), spec.kappa_c, spec.gamma, stream)
            counts.zero_()
            oow.zero_()
            if sharded:
                shoot_sharded(device_row_shooter(f, spec.grid, spec.window, stream), total_rows, counts, oow, rank,
                              world, row_begin=row0)
            else:
                rs.rs_shoot_rows(f.handle, spec.grid, r0, r1, spec.window, counts, oow, stream)
            rs.rs_magnification(counts, spec.grid, spec.window, mu, stream)
            h_mu.copy_(mu, non_blocking=True)
            h_oow.copy_(oow, non_blocking=True)
            torch.cuda.synchronize(device)
            f.close()

        e2e_step()
        n_e2e = max(2, min(args.steps, 20 if inter_step <= FULL_LIMIT else 2))
        barrier()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0)
        h2d = h_xy.numel() * 4 + (0 if h_m is None else h_m.numel() * 4)
        d2h = h_mu.numel() * 4 + 8
        e2e = {"value": inter_step * n_e2e * (1 if sharded else world) / dt, "unit": "interactions/s",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e,
               "includes": "field upload from pinned host memory + validation + repack, shoot of the step's rows, "
                           "normalise, D2H of mu and the out-of-window count, field release"}
    field.close()
    del counts, oow, mu
    torch.cuda.empty_cache()

    side = workload("n1e4", seed=0) if args.workload != "n1e4" else spec

    # ---------------- the other configurations (one GPU), each with its roofline
    configs = None
    if not args.no_configs and world == 1:
        names = [v for v in args.configs.split(",") if v and v != args.workload]
        configs = run_configs(rs, torch, device, stream, names, cpu=not args.no_cpu_baseline,
                              launch_shape=args.launch_shape, max_sample=args.max_sample)

    # ---------------- batched maps/s vs plain launches (64 fields)
    batched = None
    if not args.no_batch and world == 1:
        batched = run_batched(rs, torch, device, stream, reps=args.batch_reps)
        batched["small_fields"] = run_batched_small(rs, torch, device, stream)

    # ---------------- light curves over many maps (one launch)
    light = None
    if not args.no_light_curves and world == 1:
        light = run_light_curves(rs, torch, device, stream, cpu_baseline=not args.no_cpu_baseline)

    # the zoom, time-series and partition sections shoot the 1e4-lens field: its own tuned shape
    if world == 1 and not args.launch_shape and not (args.no_zoom and args.no_frames and args.no_staged):
        tune_for(rs, side, stream)

    # ---------------- zoom into the 1e4-lens map (culled shooting) vs plain shooting of the finer grid
    zoom = None
    if not args.no_zoom and world == 1:
        zoom = run_zoom(rs, torch, device, stream, side)
        zoom["culled_full_map"] = run_zoom(rs, torch, device, stream, side, factor=1, quarter=False)

    # ---------------- a time series of maps with moving lenses (one batch launch per 16 steps)
    frames = None
    if not args.no_frames and world == 1:
        frames = run_frames(rs, torch, device, stream, side)

    # ---------------- lens-partitioned shooting: device shards and host-streamed lenses
    staged = None
    if not args.no_staged and world == 1:
        staged = run_staged(rs, torch, device, stream, side)

    # ---------------- CPU baseline (oracle, bounded sample)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample_rate(spec, args.cpu_seconds)
        cpu = {"value": r["value"], "unit": "interactions/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"]}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # per GPU: the whole job's interactions of a sharded step over the ranks, the shoot span the slowest rank's
    rl = roofline_entry(inter_step / (world if sharded else 1), shoot_avg_s, sms, max_mhz,
                        profiled_traffic(args.workload))
    med = clk.get("sm_mhz")
    cfg = workload_config(spec, args.workload)
    cfg["rows_per_step"] = [row0, row0 + total_rows] if sharded else [r0, r1]
    cfg["rays_per_step"] = rays_step
    cfg["parallelism"] = (f"rows of one map sharded over {world} GPU(s), count maps summed (NCCL all_reduce)"
                          if sharded else f"{world} independent realisation(s), one per GPU, no collective")
    cfg["interactions_per_step"] = inter_step
    cfg["sample"] = rows_note
    cfg["l2"] = ("inputs larger than L2 (lenses: %.2f GB on the device); L2 also flushed between steps (512 MiB "
                 "write)" % (spec.n_lens * (24 if spec.masses is not None else 16) / 1e9)
                 if spec.n_lens * 16 > (129 << 20) else "flushed between timed steps (512 MiB write)")
    cfg["launch_shape"] = (f"{shape[0]} threads x {shape[1]} rays/thread x {shape[2]}-lens tiles, compiled for "
                           f"{shape[3]} CTAs/SM" + ("" if args.launch_shape else " (autotuned)"))
    if rates_headline:
        cfg["tuner_rates"] = rates_headline
    cfg["certified_binning"] = rs.rs_get_certified_binning()
    rl.update({"kernel": "shoot_kernel (span of rs_shoot_rows: list reset, shoot, certified re-evaluation)",
               "kernel_ms": shoot_avg_s * 1e3,
               "peak_basis": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x {max_mhz:.0f} MHz (max clock); "
                             f"10 flops per interaction (paper App. A)"})
    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "strong" if (sharded and whole) else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": cfg,
        "pct_fp32_peak": 100.0 * rl["frac"],
        "pct_fp32_peak_at_measured_clock": (100.0 * rl["achieved"] / fp32_peak_tflops(sms, med)) if med else None,
        "roofline": rl,
        "clocks": {"sm_mhz": med, "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons"),
                   "samples": clk.get("samples")},
        "e2e": e2e,
        "gpu_launches": (3 if rs.rs_get_certified_binning() else 2) * args.steps,
        "rays_conserved": conserved,
        "cpu_baseline": cpu,
        "configs": configs,
        "batched": batched,
        "light_curves": light,
        "zoom": zoom,
        "frames": frames,
        "staged": staged,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batched_small(rs, torch, device, stream, n_fields=256, reps=5):
    """Many small maps (the 100-lens, 1000^2-ray configuration, seeds 2000 + k): one persistent graph
    launch against one rs_shoot call per field (each: list allocation, shoot, re-evaluation)."""
    from paper_0905_2453_gb300 import tune
    specs = [ri.tiny_field(seed=2000 + k) for k in range(n_fields)]
    fields = [rs.Field.from_spec(s, stream) for s in specs]
    saved = rs.rs_get_launch_config(False)  # put back afterwards: later sections shoot other fields
    shape = tune.autotune(fields[0], specs[0].grid, specs[0].window, stream=stream)[:4]  # the fields' own shape
    b = rs.Batch(fields, [s.grid for s in specs], [s.window for s in specs])
    counts_plain = [torch.zeros_like(c) for c in b.counts]
    oow_plain = torch.zeros(len(specs), dtype=torch.int64, device=device)

    def plain():
        for c in counts_plain:
            c.zero_()
        oow_plain.zero_()
        for k, f in enumerate(fields):
            rs.rs_shoot(f.handle, specs[k].grid, specs[k].window, counts_plain[k], oow_plain[k:k + 1], stream)

    b.launch(stream)
    plain()
    torch.cuda.synchronize(device)
    same = all(torch.equal(b.counts[k], counts_plain[k]) for k in range(len(specs))) and \
        torch.equal(b.out_of_window, oow_plain)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize(device)
    t_batch = e0.elapsed_time(e1) / 1e3 / reps
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(reps):
        plain()
    e1.record(stream)
    torch.cuda.synchronize(device)
    t_plain = max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0) / reps
    inter = sum(s.interactions for s in specs)
    b.close()
    for f in fields:
        f.close()
    rs.rs_set_launch_config(False, *saved)
    return {"workload": f"{n_fields} fields of 100 equal-mass lenses, 1000^2 rays, 256^2 maps",
            "launch_shape": "x".join(str(v) for v in shape),
            "maps_per_s": n_fields / t_batch, "plain_maps_per_s": n_fields / t_plain, "speedup": t_plain / t_batch,
            "interactions_per_s": inter / t_batch, "bitwise_equal": bool(same), "reps": reps}


def run_batched(rs, torch, device, stream, reps=10):
    from paper_0905_2453_gb300 import tune
    specs = ri.batch_fields(64)
    fields = [rs.Field.from_spec(s, stream) for s in specs]
    big = max(range(len(specs)), key=lambda k: specs[k].interactions)
    tune.autotune(fields[big], specs[big].grid, specs[big].window, stream=stream)
    grids = [s.grid for s in specs]
    wins = [s.window for s in specs]
    b = rs.Batch(fields, grids, wins)
    counts_plain = [torch.zeros_like(c) for c in b.counts]
    oow_plain = torch.zeros(len(specs), dtype=torch.int64, device=device)

    def plain():
        for k, f in enumerate(fields):
            counts_plain[k].zero_()
        oow_plain.zero_()
        for k, f in enumerate(fields):
            rs.rs_shoot(f.handle, grids[k], wins[k], counts_plain[k], oow_plain[k:k + 1], stream)

    b.launch(stream)
    plain()
    torch.cuda.synchronize(device)
    same = all(torch.equal(b.counts[k], counts_plain[k]) for k in range(len(specs))) and \
        torch.equal(b.out_of_window, oow_plain)
    # alternate the two so that both see the same clock and temperature history; every repetition timed
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    for e in ev:
        e[0].record(stream)
        b.launch(stream)
        e[1].record(stream)
        e[2].record(stream)
        plain()
        e[3].record(stream)
    torch.cuda.synchronize(device)
    tb = [e[0].elapsed_time(e[1]) / 1e3 for e in ev]
    tp = [e[2].elapsed_time(e[3]) / 1e3 for e in ev]
    t_batch, t_plain = statistics.median(tb), statistics.median(tp)
    ratios = sorted(p / q for p, q in zip(tp, tb))
    inter = sum(s.interactions for s in specs)
    b.close()
    # the same batch with a launch shape tuned per lens-count bucket
    shapes = tune.batch_shapes(fields, grids, wins, stream=stream)
    bs = rs.Batch(fields, grids, wins, shapes=shapes)
    bs.launch(stream)
    torch.cuda.synchronize(device)
    same_shaped = all(torch.equal(bs.counts[k], counts_plain[k]) for k in range(len(specs)))
    es = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
    for e in es:
        e[0].record(stream)
        bs.launch(stream)
        e[1].record(stream)
    torch.cuda.synchronize(device)
    t_shaped = statistics.median(e[0].elapsed_time(e[1]) / 1e3 for e in es)
    bs.close()
    for f in fields:
        f.close()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    return {"workload": "64 Salpeter fields, N* log-uniform [1e2,1e5], rays 1024^2-4096^2, maps 512^2-1024^2",
            "per_bucket_shapes": {"maps_per_s": len(specs) / t_shaped, "speedup_vs_plain": t_plain / t_shaped,
                                  "bitwise_equal": bool(same_shaped),
                                  "shapes": sorted({"x".join(str(v) for v in sh) for sh in shapes})},
            "maps_per_s": len(specs) / t_batch, "plain_maps_per_s": len(specs) / t_plain,
            "speedup": t_plain / t_batch,
            "speedup_per_rep": {"min": ratios[0], "median": statistics.median(ratios), "max": ratios[-1]},
            "batch_ms": {"median": t_batch * 1e3, "min": min(tb) * 1e3, "max": max(tb) * 1e3},
            "plain_ms": {"median": t_plain * 1e3, "min": min(tp) * 1e3, "max": max(tp) * 1e3},
            "interactions_per_s": inter / t_batch, "bitwise_equal": bool(same), "reps": reps,
            "roofline": roofline_entry(inter, t_batch, sms, 2070.0)}


def support_pixels(wins, tracks, R):
    """Pixels whose centres lie within R of each sample, summed over all samples (the pixels the
    definition averages over), counted row by row in float64."""
    total = 0
    for t in tracks:
        w = wins[t.map]
        pix = [(w.hi[a] - w.lo[a]) / w.npix[a] for a in range(2)]
        k = np.arange(t.n, dtype=np.float64)
        t0 = (t.y0[0] + k * t.step[0] - w.lo[0]) / pix[0] - 0.5
        t1 = (t.y0[1] + k * t.step[1] - w.lo[1]) / pix[1] - 0.5
        rp0, rp1 = R / pix[0], R / pix[1]
        for dj in range(-int(rp1) - 1, int(rp1) + 2):
            j = np.floor(t1) + dj
            dy = j - t1
            h2 = rp0 * rp0 * (1.0 - (dy / rp1) ** 2)
            ok = (h2 >= 0) & (j >= 0) & (j < w.npix[1])
            h = np.sqrt(np.where(ok, h2, 0.0))
            lo = np.maximum(np.ceil(t0 - h), 0)
            hi = np.minimum(np.floor(t0 + h), w.npix[0] - 1)
            total += int(np.where(ok, np.maximum(hi - lo + 1, 0), 0).sum())
    return total


def run_light_curves(rs, torch, device, stream, reps=20, cpu_samples=4096, cpu_baseline=True):
    """Light curves of 1024 tracks x 2048 samples over 64 synthetic caustic maps in one launch."""
    maps, wins, tracks, s = ri.light_curve_workload()
    tmaps = [torch.from_numpy(m).to(device) for m in maps]
    rtr = [rs.Track(t.map, t.y0, t.step, t.n) for t in tracks]
    total = sum(t.n for t in tracks)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    support = support_pixels(wins, tracks, 6.0 * s)
    plan = rs.LightCurvePlan(tmaps, wins, rtr, rs.RS_PROFILE_GAUSSIAN, s)
    for _ in range(3):
        plan.launch(stream)
    torch.cuda.synchronize(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.fill_(k)
        ev[k][0].record(stream)
        plan.launch(stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize(device)
    t = statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3
    # one-shot call (validation, table upload, launch, release) from the host
    mu = torch.empty(total, dtype=torch.float64, device=device)
    dm = torch.empty_like(mu)
    rs.rs_light_curves(tmaps, wins, rs.RS_PROFILE_GAUSSIAN, s, rtr, mu, dm, stream)
    torch.cuda.synchronize(device)
    same = bool(torch.equal(mu.view(torch.int64), plan.mu.view(torch.int64)))
    t0 = time.perf_counter()
    for _ in range(5):
        rs.rs_light_curves(tmaps, wins, rs.RS_PROFILE_GAUSSIAN, s, rtr, mu, dm, stream)
    torch.cuda.synchronize(device)
    t_one = (time.perf_counter() - t0) / 5
    plan.close()
    # CPU baseline: the oracle on a bounded sample (the first cpu_samples samples, in track order)
    cpu = None
    if cpu_baseline:
        import oracle
        n_cpu, t_cpu, k = 0, 0.0, 0
        while n_cpu < cpu_samples and k < len(tracks):
            tr = tracks[k]
            w = wins[tr.map]
            m64 = maps[tr.map].astype(np.float64)
            n = min(tr.n, cpu_samples - n_cpu)
            t0 = time.perf_counter()
            oracle.light_curve(m64, w.lo, w.hi, oracle.PROFILE_GAUSSIAN, s, tr.y0, tr.step, n)
            t_cpu += time.perf_counter() - t0
            n_cpu += n
            k += 1
        cpu = {"value": n_cpu / t_cpu, "unit": "samples/s", "kind": "oracle", "cores": oracle.num_threads(),
               "sample": f"{n_cpu} samples, full-map visit per sample"}
    return {"workload": "64 caustic maps 512^2-1024^2, 1024 tracks x 2048 samples, Gaussian source 1-2 px",
            "samples_per_s": total / t, "support_pixels_per_s": support / t, "kernel_ms": t * 1e3,
            "support_pixels_per_launch": support, "samples_per_launch": total, "reps": reps,
            "one_shot_ms": t_one * 1e3, "one_shot_equal_plan": same,
            "l2": "flushed between launches",
            "cpu_baseline": cpu}


def run_zoom(rs, torch, device, stream, spec, factor=4, reps=3, quarter=True):
    """Zoom x factor into the central quarter (per axis) of the map (or the whole map with
    quarter=False): culled vs plain shooting."""
    w = spec.window
    q = [(w.hi[k] - w.lo[k]) / (8.0 if quarter else 2.0) for k in range(2)]
    c = [(w.hi[k] + w.lo[k]) / 2.0 for k in range(2)]
    lo, hi = (c[0] - q[0], c[1] - q[1]), (c[0] + q[0], c[1] + q[1])
    g = rs.zoom_grid(spec.grid, factor)
    zw = rs.zoom_window(w, lo, hi, factor)
    f = rs.Field.from_spec(spec, stream)
    npix = (int(zw.npix[1]), int(zw.npix[0]))
    cc = torch.zeros(npix, dtype=torch.int32, device=device)
    cp = torch.zeros_like(cc)
    oc = torch.zeros(1, dtype=torch.int64, device=device)
    op = torch.zeros_like(oc)
    shot = torch.zeros(1, dtype=torch.int64, device=device)
    f.shoot(g, zw, cc, oc, stream=stream, culled=True, rays_shot=shot)   # warm-up
    torch.cuda.synchronize(device)
    n_shot = int(shot.item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        cc.zero_()
        oc.zero_()
        f.shoot(g, zw, cc, oc, stream=stream, culled=True)
    e1.record(stream)
    torch.cuda.synchronize(device)
    t_c = e0.elapsed_time(e1) / 1e3 / reps
    e0.record(stream)
    f.shoot(g, zw, cp, op, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(device)
    t_p = e0.elapsed_time(e1) / 1e3
    same = bool(torch.equal(cc, cp)) and bool(torch.equal(oc, op))
    f.close()
    n = g.n[0] * g.n[1]
    region = "the central quarter of the map per axis" if quarter else "the whole map"
    return {"workload": f"{args_workload_name(spec)}: x{factor} zoom into {region}, {g.n[0]}^2 rays, "
                        f"{zw.npix[0]}^2 map",
            "rays": n, "rays_shot": n_shot, "rays_shot_frac": n_shot / n, "culled_ms": t_c * 1e3,
            "plain_ms": t_p * 1e3, "speedup": t_p / t_c, "bitwise_equal": same,
            "culled_interactions_per_s_full_grid_equivalent": n * spec.n_lens / t_c}


def run_section(args):
    import torch
    import paper_0905_2453_gb300 as rs
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    if args.section == "zoom":
        spec = workload(args.workload, seed=0)
        if args.launch_shape:
            rs.rs_set_launch_config(spec.masses is not None and not bool(np.all(spec.masses == 1.0)),
                                    *parse_shape(args.launch_shape))
        out = {"zoom": run_zoom(rs, torch, device, stream, spec),
               "culled_full_map": run_zoom(rs, torch, device, stream, spec, factor=1, quarter=False)}
    elif args.section == "batch-small":
        out = {"small_fields": run_batched_small(rs, torch, device, stream)}
    elif args.section == "batch":
        out = {"batched": run_batched(rs, torch, device, stream, reps=args.batch_reps)}
    elif args.section == "staged":
        spec = workload(args.workload, seed=0)
        out = {"staged": run_staged(rs, torch, device, stream, spec)}
    elif args.section == "configs":
        names = [v for v in args.configs.split(",") if v]
        out = {"configs": run_configs(rs, torch, device, stream, names, cpu=not args.no_cpu_baseline,
                                      launch_shape=args.launch_shape, max_sample=args.max_sample)}
    elif args.section == "frames":
        spec = workload(args.workload, seed=0)
        out = {"frames": run_frames(rs, torch, device, stream, spec)}
    else:
        out = {"light_curves": run_light_curves(rs, torch, device, stream)}
    print(json.dumps(out), flush=True)


def run_frames(rs, torch, device, stream, spec, n_frames=16, dt=1.0, sigma_v=0.1, reps=2):
    """A time series of maps of the workload field with moving lenses: n_frames moving fields in one
    batch, each stepped to its own time before every launch."""
    vel = ri.lens_velocities(spec.n_lens, sigma_v, seed=7)
    frames = [rs.Field(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, stream, velocities=vel)
              for _ in range(n_frames)]
    b = rs.Batch(frames, [spec.grid] * n_frames, [spec.window] * n_frames)

    def step(r):
        for k, fr in enumerate(frames):
            fr.set_time((r * n_frames + k) * dt, stream)
        b.launch(stream)

    step(0)
    torch.cuda.synchronize(device)
    # the batch's last frame against a plain shoot of the same moving field at the same time (bitwise)
    ref = frames[-1].shoot(spec.grid, spec.window, stream=stream)
    torch.cuda.synchronize(device)
    same = bool(torch.equal(ref, b.counts[n_frames - 1]))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(1, reps + 1):
        step(r)
    e1.record(stream)
    torch.cuda.synchronize(device)
    t = e0.elapsed_time(e1) / 1e3 / reps
    b.close()
    for fr in frames:
        fr.close()
    return {"workload": f"{args_workload_name(spec)} with Gaussian lens velocities sigma {sigma_v} per axis, "
                        f"{n_frames} time steps of {dt} per batch launch",
            "frames_per_s": n_frames / t, "ms_per_frame": t / n_frames * 1e3,
            "interactions_per_s": n_frames * spec.interactions / t, "batched_frame_equals_plain_shoot": same,
            "reps": reps}


def run_staged(rs, torch, device, stream, spec, parts=4, reps=3):
    """The workload field as lens partitions (device-resident shards) and streamed from host memory,
    against the plain one-field shoot: times and bit-equality."""
    n = spec.n_lens
    per = max(256, (n + parts - 1) // parts // 256 * 256)
    cuts = list(range(per, n, per))
    bounds = [0] + cuts + [n]
    shards = [rs.Field(spec.lens_xy[a:b], None if spec.masses is None else spec.masses[a:b], spec.kappa_c,
                       spec.gamma, stream) for a, b in zip(bounds[:-1], bounds[1:])]
    plain = rs.Field.from_spec(spec, stream)
    npix = (int(spec.window.npix[1]), int(spec.window.npix[0]))
    out = {}
    ref = torch.zeros(npix, dtype=torch.int32, device=device)
    ref_o = torch.zeros(1, dtype=torch.int64, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / reps

    def plain_fn():
        ref.zero_()
        ref_o.zero_()
        plain.shoot(spec.grid, spec.window, ref, ref_o, stream=stream)

    t_plain = timed(plain_fn)
    c = torch.zeros_like(ref)
    o = torch.zeros_like(ref_o)

    def staged_fn():
        c.zero_()
        o.zero_()
        rs.rs_shoot_staged([f.handle for f in shards], spec.grid, 0, int(spec.grid.n[1]), spec.window, c, o, stream)

    t_staged = timed(staged_fn)
    same_staged = bool(torch.equal(c, ref)) and bool(torch.equal(o, ref_o))
    per_pass = max(1024, (n + parts - 1) // parts // 1024 * 1024)

    def streamed_fn():
        c.zero_()
        o.zero_()
        rs.rs_shoot_streamed(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, per_pass, spec.grid, 0,
                             int(spec.grid.n[1]), spec.window, c, o, stream)

    t_streamed = timed(streamed_fn)
    same_streamed = bool(torch.equal(c, ref)) and bool(torch.equal(o, ref_o))
    for f in shards + [plain]:
        f.close()
    out = {"workload": f"{args_workload_name(spec)}: {len(shards)} device shards of <= {per} lenses; host-resident "
                       f"lenses streamed {per_pass} per pass",
           "plain_ms": t_plain, "staged_ms": t_staged, "streamed_ms": t_streamed,
           "staged_interactions_per_s": spec.interactions / (t_staged / 1e3),
           "streamed_interactions_per_s": spec.interactions / (t_streamed / 1e3),
           "staged_bitwise_equal": same_staged, "streamed_bitwise_equal": same_streamed, "reps": reps}
    return out


def oracle_trace_rate(spec, n_rays: int, seed: int = 11):
    """The FP64 oracle on a random subset of the grid's rays (per-ray evaluation): interactions/s."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    ij = np.stack([rng.integers(0, int(spec.grid.n[0]), n_rays), rng.integers(0, int(spec.grid.n[1]), n_rays)], 1)
    t = time.perf_counter()
    oracle.trace_field(spec, ij)
    dt = time.perf_counter() - t
    return {"value": n_rays * spec.n_lens / dt, "unit": METRIC, "seconds": dt, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{n_rays} random rays of the grid, all {spec.n_lens} lenses"}


def run_configs(rs, torch, device, stream, names, cpu=True, full_limit=2e12, max_sample=2e13, launch_shape=None):
    """Throughput of the shoot on every workload configuration (1 GPU).

    Grids of up to full_limit interactions are shot whole.  Larger ones are timed on two blocks of
    central rows, k and 2k units of rows that hold a whole number of waves of the tuned launch shape
    (a multiple of 2 x SMs CTAs: whole waves at one or two resident CTAs per SM, every launch shape
    here).  The rate of the larger block is the sample rate; the difference of the two (the work of
    k units over the difference of the times) is the steady-state rate of the full grid, whose ragged
    end of the last CTAs -- up to one CTA time, seconds with 1e8 lenses -- the difference cancels.
    """
    from paper_0905_2453_gb300 import tune
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peak = fp32_peak_tflops(sms, 2070) * 1e12

    def pct(rate):
        return 100.0 * rate * FLOPS_PER_INTERACTION / peak

    out = {}
    for name in names:
        spec = workload(name, seed=0)
        f = rs.Field.from_spec(spec, stream)
        n_lens, weighted = f.info()
        if launch_shape:
            b, r, t, mc = parse_shape(launch_shape)
            rs.rs_set_launch_config(weighted, b, r, t, mc)
        else:
            b, r, t, mc, _ = tune.autotune(f, spec.grid, spec.window, stream=stream)
        n0, n1 = int(spec.grid.n[0]), int(spec.grid.n[1])
        npix = (int(spec.window.npix[1]), int(spec.window.npix[0]))
        c = torch.zeros(npix, dtype=torch.int32, device=device)
        o = torch.zeros(1, dtype=torch.int64, device=device)
        clocks = ClockSampler(device.index or 0)
        clocks.start()

        def timed(r0, r1, warm=True):
            """ms per launch: one launch, or back-to-back launches (as a stream of maps runs) when short."""
            if warm:
                rs.rs_shoot_rows(f.handle, spec.grid, r0, r1, spec.window, c, o, stream)
            torch.cuda.synchronize(device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs.rs_shoot_rows(f.handle, spec.grid, r0, r1, spec.window, c, o, stream)
            e1.record(stream)
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1)
            if ms < 100.0:
                n = int(min(1000, max(2, 500.0 // max(ms, 1e-3))))
                e0.record(stream)
                for _ in range(n):
                    rs.rs_shoot_rows(f.handle, spec.grid, r0, r1, spec.window, c, o, stream)
                e1.record(stream)
                torch.cuda.synchronize(device)
                ms = e0.elapsed_time(e1) / n
            return ms

        entry = {"workload": spec.name, "n_lens": n_lens, "weighted_kernels": bool(weighted),
                 "launch_shape": f"{b}x{r}x{t}x{mc}", "full_grid_interactions": spec.interactions,
                 "tuner_rates": tune.shape_rates(f, spec.grid)}
        if spec.interactions <= full_limit:
            ms = timed(0, n1)
            rate = spec.interactions / (ms / 1e3)
            entry.update({"sample": "whole grid", "rows": [0, n1], "ms": ms, "interactions_per_s": rate,
                          "pct_fp32_peak_2070mhz": pct(rate)})
        else:
            warps, cpr = b // 32, -(-n0 // (32 * r))       # rows and CTAs per row group
            unit = tune.wave_rows(n0, b, r, sms, rs.rs_launch_occupancy(weighted, b, r, t, mc))
            per_unit = unit * n0 * n_lens
            k = max(1, min(n1 // (2 * unit), int(max_sample // (2 * per_unit))))
            blocks = []
            for rows in (k * unit, 2 * k * unit):
                r0 = (n1 - rows) // 2 // warps * warps
                ms = timed(r0, r0 + rows, warm=not blocks)
                blocks.append({"rows": [r0, r0 + rows], "ctas": cpr * (rows // warps), "ms": ms,
                               "interactions_per_s": rows * n0 * n_lens / (ms / 1e3)})
            steady = k * per_unit / ((blocks[1]["ms"] - blocks[0]["ms"]) / 1e3)
            entry.update({"sample": f"central row blocks of {k} and {2 * k} x {unit} rows ({blocks[0]['ctas']} and "
                                    f"{blocks[1]['ctas']} CTAs of {b} threads on {sms} SMs)",
                          "blocks": blocks, "interactions_per_s": steady, "pct_fp32_peak_2070mhz": pct(steady),
                          "sample_interactions_per_s": blocks[1]["interactions_per_s"],
                          "sample_pct_fp32_peak_2070mhz": pct(blocks[1]["interactions_per_s"])})
        entry["clocks"] = clocks.stop()
        entry["roofline"] = roofline_entry(1.0, 1.0 / entry["interactions_per_s"], sms, 2070.0, profiled_traffic(name))
        entry["full_grid_seconds_at_this_rate"] = spec.interactions / entry["interactions_per_s"]
        entry["status"] = f.status()
        f.close()
        if cpu:
            n_rays = max(16, min(100_000, int(3e9 / max(1, n_lens))))
            entry["cpu_baseline"] = oracle_trace_rate(spec, n_rays)
        out[name] = entry
        log(f"config {name}: {json.dumps(entry)}")
        del c, o
        torch.cuda.empty_cache()
    return out


def args_workload_name(spec):
    return getattr(spec, "name", "field")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["sharded", "realisations"], default="sharded",
                    help="N > 1: one map per step with its rows split over the GPUs and the counts summed (sharded), "
                         "or an independent realisation per GPU (realisations)")
    ap.add_argument("--workload", default="n1e8")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-light-curves", action="store_true")
    ap.add_argument("--no-zoom", action="store_true")
    ap.add_argument("--no-frames", action="store_true")
    ap.add_argument("--no-staged", action="store_true")
    ap.add_argument("--max-sample", type=float, default=2e13,
                    help="interactions of the larger row block of a sampled configuration (--section configs)")
    ap.add_argument("--configs", default="tiny,n1e4,n1e6",
                    help="workloads of the configs sub-object (comma-separated: tiny, n1e4, n1e6, n1e8; the "
                         "headline workload is left out)")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--section", choices=["zoom", "light-curves", "frames", "staged", "batch", "batch-small",
                                          "configs"],
                    default=None,
                    help="run one secondary measurement alone and print its JSON object (for profiling)")
    ap.add_argument("--batch-reps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--launch-shape", default=None,
                    help="fix the launch shape, e.g. 128x8x512x2 (threads x rays/thread x lens tile x CTAs/SM; skips "
                         "the autotuner)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.section is not None:
        run_section(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
