"""Launch-shape autotuner.

The library carries kernels for several launch shapes (threads per CTA x rays per
thread x lenses per shared-memory stage x resident CTAs per SM compiled for, see
``rs_launch_configs``).  All of them
compute bitwise identical results, so the choice only affects speed.  ``autotune`` times every shape on a
proxy run (a block of the workload's own grid rows; for fields larger than the proxy,
one whole wave of CTAs per launch, and the proxy's best three again on the field itself
where a whole-wave unit of it is affordable) with CUDA events, selects the fastest with
``rs_set_launch_config`` and caches the choice in a JSON file keyed
by (GPU name, library version, mass mode, lens-count bucket, row-length bucket).  This replaces the
paper's occupancy-calculator choice of 128 or 256 threads (Section 2.2).  Fields of more than
``max_proxy_lenses`` lenses are timed on a view of their first lenses: past a few lens tiles the cost
per interaction no longer depends on the lens count, and a proxy over all 1e8 lenses of a large field
would take minutes per shape.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import rs_launch_configs, rs_launch_occupancy, rs_set_launch_config, rs_shoot_rows, rs_version

DEFAULT_CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")),
                             "rs_gb300", "tune.json")


def _bucket(v: int) -> int:
    return 0 if v <= 0 else int(round(math.log2(v)))


def cache_key(field, grid) -> str:
    n_lens, has_mass = field.info()
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    return (f"{name}|{rs_version()}|mass={int(has_mass)}|N=2^{_bucket(n_lens)}"
            f"|n0=2^{_bucket(int(grid.n[0]))}")


def wave_rows(n0: int, block: int, rpt: int, sms: int, ctas_per_sm: int = 2) -> int:
    """The smallest number of grid rows whose CTAs (of `block` threads x `rpt` rays per thread, one warp per
    row and 32 x rpt columns per CTA) fill whole waves of ctas_per_sm x sms CTAs (the default, two resident
    CTAs per SM, makes whole waves at one or two)."""
    warps, seg = block // 32, 32 * rpt
    cpr = -(-int(n0) // seg)  # CTAs per group of `warps` rows
    wave = int(ctas_per_sm) * int(sms)
    return wave // math.gcd(wave, cpr) * warps


def shape_rates(field, grid, cache_path: str = None) -> dict:
    """Steady-state interactions/s per launch shape ("block x rpt x lens_tile x min_ctas") from the tuner's cache entry for
    (field, grid): the shapes verified on the field itself if any, else every shape on the proxy ({} if the pair
    was never tuned)."""
    cache = _load(cache_path or os.environ.get("RS_TUNE_CACHE", DEFAULT_CACHE))
    entry = cache.get(cache_key(field, grid), {})
    return dict(entry.get("field_interactions_per_s") or entry.get("interactions_per_s", {}))


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _verify_on_field(field, grid, window, counts, st, rates, timings, shape_rows, has_mass, sms, n0, n1, n_lens,
                     verify_interactions, top=3):
    """Rates on the field itself of those of the proxy's best `top` shapes whose whole-wave unit of rows costs at
    most verify_interactions ({} if none): one and two units, rated by the difference (the steady state of many
    waves).  The proxy ranks shapes within a few percent only; a unit of the field settles it."""
    cands = sorted(rates, key=rates.get, reverse=True)[:top]
    verified = {}
    field_handle = field.handle
    for name in cands:
        shape = tuple(int(v) for v in name.split("x"))
        block, rpt = shape[0], shape[1]
        unit = wave_rows(n0, block, rpt, sms, rs_launch_occupancy(has_mass, *shape))
        if 2 * unit > n1 or unit * n0 * n_lens > verify_interactions:
            continue  # this shape's whole-wave unit does not fit the grid or the budget
        rs_set_launch_config(has_mass, *shape)
        warps = block // 32
        r0 = (n1 - 2 * unit) // 2 // warps * warps

        def timed(rows):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rs_shoot_rows(field_handle, grid, r0, r0 + rows, window, counts, None, st)
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1)

        timed(unit)  # warm-up
        t1, t2 = timed(unit), timed(2 * unit)
        verified[name] = (unit * n0 * n_lens / max(t2 - t1, 1e-6) * 1e3 if t2 > t1
                          else 2 * unit * n0 * n_lens / max(t2, 1e-6) * 1e3)
        timings[name + "/field"], shape_rows[name + "/field"] = t2, [unit, 2 * unit]
    return verified


def autotune(field, grid, window, min_rays: float = 8e6, max_interactions: float = 3e11, reps: int = 3,
             cache_path: str = None, force: bool = False, stream=None, max_proxy_lenses: int = 1 << 16,
             verify_interactions: float = 2e12):
    """Pick and set the fastest launch shape for this (field, grid); returns (block, rpt, lens_tile, min_ctas,
    timings_ms) with each shape's time for its own (largest) proxy block of rows."""
    cache_path = cache_path or os.environ.get("RS_TUNE_CACHE", DEFAULT_CACHE)
    n_lens, has_mass = field.info()
    key = cache_key(field, grid)
    cache = _load(cache_path)
    if not force and key in cache:
        sh = tuple(cache[key]["shape"])
        rs_set_launch_config(has_mass, *sh)
        return (*sh, cache[key].get("ms", {}))
    # proxy: blocks of the grid's rows, capped in work; very large fields through a view of their
    # first lenses.  Where the grid allows, each shape shoots k and 2k units of rows holding a whole
    # number of waves (a multiple of 2 x SMs CTAs: whole waves at one or two resident CTAs per SM) and
    # is rated by the difference, k units over the difference of the times: the steady state of a
    # large grid, without the ragged end of the last CTAs that would favour shapes with more, smaller
    # CTAs.  Small grids are timed whole, as they will run.
    proxy = field.view(0, max_proxy_lenses) if n_lens > max_proxy_lenses else field
    n_proxy = max(1, min(n_lens, max_proxy_lenses))
    n0, n1 = int(grid.n[0]), int(grid.n[1])
    rows = max(64, int(min_rays // max(1, n0)))
    rows = min(rows, max(64, int(max_interactions // max(1, n0 * n_proxy))))
    rows = min(rows, n1)
    dev = torch.device("cuda", torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev) if stream is None else stream

    def timed(nrows):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rs_shoot_rows(proxy.handle, grid, 0, nrows, window, counts, None, st)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    timings, rates, shape_rows = {}, {}, {}
    try:
        for shape in rs_launch_configs():
            block, rpt = shape[0], shape[1]
            unit = wave_rows(n0, block, rpt, sms)
            k = min(max(1, round(rows / unit)), n1 // (2 * unit))
            name = "x".join(str(v) for v in shape)
            rs_set_launch_config(has_mass, *shape)
            if proxy is not field:
                # A large field's CTAs each run for seconds, all CTAs of a wave in step with one another
                # (their warps then compete for the same pipe at the same time); short proxy CTAs drift
                # apart over many waves and hide that.  So each launch here is exactly the rows of one
                # whole wave at the shape's real occupancy, as a block of the large field runs.
                wave = wave_rows(n0, block, rpt, sms, rs_launch_occupancy(has_mass, *shape))
                if wave <= n1:
                    rs_shoot_rows(proxy.handle, grid, 0, wave, window, counts, None, st)  # warm-up
                    timings[name], shape_rows[name] = timed(wave), [wave]
                    rates[name] = wave * n0 * n_proxy / max(timings[name], 1e-6) * 1e3
                    continue
            if rows < n1 and k >= 1 and unit * n0 * n_proxy <= 4 * max_interactions:
                rs_shoot_rows(proxy.handle, grid, 0, k * unit, window, counts, None, st)  # warm-up
                t1, t2 = timed(k * unit), timed(2 * k * unit)
                timings[name], shape_rows[name] = t2, [k * unit, 2 * k * unit]
                per = k * unit * n0 * n_proxy
                rates[name] = per / max(t2 - t1, 1e-6) * 1e3 if t2 > t1 else 2 * per / max(t2, 1e-6) * 1e3
            else:
                rs_shoot_rows(proxy.handle, grid, 0, rows, window, counts, None, st)  # warm-up
                timings[name], shape_rows[name] = timed(rows), [rows]
                rates[name] = rows * n0 * n_proxy / max(timings[name], 1e-6) * 1e3
        field_rates = {}
        if proxy is not field:
            field_rates = _verify_on_field(field, grid, window, counts, st, rates, timings, shape_rows, has_mass, sms,
                                           n0, n1, n_lens, verify_interactions)
    finally:
        if proxy is not field:
            proxy.close()
    ranked = field_rates or rates
    best = max(ranked, key=ranked.get)
    sh = tuple(int(v) for v in best.split("x"))
    rs_set_launch_config(has_mass, *sh)
    cache[key] = {"shape": list(sh), "ms": timings, "rows": shape_rows, "interactions_per_s": rates,
                  "field_interactions_per_s": field_rates, "proxy_lenses": n_proxy}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    except OSError:
        pass
    return (*sh, timings)


def batch_shapes(fields, grids, windows, stream=None, cache_path: str = None, **kw):
    """A launch shape per field of a batch: fields are grouped by mass mode and lens-count bucket (the cache
    key's), the largest field (most rays) of each group is tuned, and its shape serves the group.  Returns a list
    of (block, rpt, lens_tile, min_ctas) for rs_batch_create_shaped.  The launch configuration of each mass mode is left as
    it was."""
    from . import rs_get_launch_config
    saved = {m: rs_get_launch_config(m) for m in (False, True)}
    groups = {}
    for k, (f, g) in enumerate(zip(fields, grids)):
        n_lens, has_mass = f.info()
        groups.setdefault((int(has_mass), _bucket(n_lens)), []).append(k)
    shapes = [None] * len(fields)
    try:
        for members in groups.values():
            big = max(members, key=lambda k: int(grids[k].n[0]) * int(grids[k].n[1]))
            sh = tuple(autotune(fields[big], grids[big], windows[big], stream=stream, cache_path=cache_path, **kw)[:4])
            for k in members:
                shapes[k] = sh
    finally:
        for m, sh in saved.items():
            rs_set_launch_config(m, *sh)
    return shapes
