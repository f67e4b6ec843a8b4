"""Launch-shape autotuner.

The library carries kernels for several launch shapes (threads per CTA x rays per
thread, see ``rs_launch_configs``).  All of them compute bitwise identical
results, so the choice only affects speed.  ``autotune`` times every shape on a
proxy run (a block of the workload's own grid rows) with CUDA events, selects the
fastest with ``rs_set_launch_config`` and caches the choice in a JSON file keyed
by (GPU name, library version, mass mode, lens-count bucket, row-length bucket).  This replaces the
paper's occupancy-calculator choice of 128 or 256 threads (Section 2.2).
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import rs_launch_configs, rs_set_launch_config, rs_shoot_rows, rs_version

DEFAULT_CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")),
                             "rs_gb300", "tune.json")


def _bucket(v: int) -> int:
    return 0 if v <= 0 else int(round(math.log2(v)))


def cache_key(field, grid) -> str:
    n_lens, has_mass = field.info()
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return (f"{name}|{rs_version()}|mass={int(has_mass)}|N=2^{_bucket(n_lens)}"
            f"|n0=2^{_bucket(int(grid.n[0]))}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def autotune(field, grid, window, min_rays: float = 8e6, max_interactions: float = 3e11, reps: int = 3,
             cache_path: str = None, force: bool = False, stream=None):
    """Pick and set the fastest launch shape for this (field, grid); returns (block, rpt, timings_ms)."""
    cache_path = cache_path or os.environ.get("RS_TUNE_CACHE", DEFAULT_CACHE)
    n_lens, has_mass = field.info()
    key = cache_key(field, grid)
    cache = _load(cache_path)
    if not force and key in cache:
        b, r = cache[key]["block"], cache[key]["rpt"]
        rs_set_launch_config(has_mass, b, r)
        return b, r, cache[key].get("ms", {})
    # proxy: enough rays for several full waves of the largest CTA tile on every SM (a partial wave
    # would favour shapes with more, smaller CTAs), capped in work
    n0, n1 = int(grid.n[0]), int(grid.n[1])
    rows = max(64, int(min_rays // max(1, n0)))
    rows = min(rows, max(64, int(max_interactions // max(1, n0 * max(1, n_lens)))))
    rows = min(rows, n1)
    dev = torch.device("cuda", torch.cuda.current_device())
    counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev) if stream is None else stream
    timings = {}
    for block, rpt in rs_launch_configs():
        rs_set_launch_config(has_mass, block, rpt)
        rs_shoot_rows(field.handle, grid, 0, rows, window, counts, None, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rs_shoot_rows(field.handle, grid, 0, rows, window, counts, None, st)
        e1.record(st)
        e1.synchronize()
        timings[f"{block}x{rpt}"] = e0.elapsed_time(e1) / reps
    best = min(timings, key=timings.get)
    b, r = (int(t) for t in best.split("x"))
    rs_set_launch_config(has_mass, b, r)
    cache[key] = {"block": b, "rpt": r, "ms": timings, "proxy_rows": rows}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    except OSError:
        pass
    return b, r, timings
