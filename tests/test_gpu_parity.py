"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances (the method's stated targets):
  * per-ray source-position error |y_gpu - y_oracle| <= 1e-5 pixel (max over axes);
  * at most 1e-5 of rays binned into a different pixel;
  * per-pixel magnification error |N_gpu - N_oracle| <= max(1, 1e-3 N_oracle) for maps of >= 1e8 rays.
Integer results with exact inputs (no lenses, dyadic grids) must match bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import (all_rays, dev, error_stats, per_ray_bound, pixel_index, rs, shoot_gpu, trace_gpu)

pytestmark = pytest.mark.gpu

PER_RAY_TOL_PIX = 1e-5
FLIP_FRAC_TOL = 1e-5


def _no_lens_field(kappa_c, gamma, grid, window):
    return ri.Field("nolens", np.zeros((0, 2), np.float32), None, kappa_c, gamma, grid, window)


def test_device_code_targets_sm103a():
    """The runtime reports the library's kernels as built for compute capability 10.3 (sm_103a)."""
    m = rs()
    assert m.rs_device_code_version() == 103


def test_zero_lenses_uniform_map_exact():
    g = ri.cell_centred_grid(-2.0, 2.0, 1024)
    w = ri.square_window(2.0, 256)
    counts, oow = shoot_gpu(_no_lens_field(0.0, 0.0, g, w))
    assert oow == 0 and np.all(counts == 16)
    m = rs()
    c = torch.from_numpy(counts.view(np.int32)).to(dev())
    mu = m.magnification(c, g, w).cpu().numpy()
    assert np.all(mu == 1.0)


def test_linear_map_bitwise_equal_to_oracle():
    g = ri.cell_centred_grid(-2.0, 2.0, 1024)
    w = ri.square_window(1.5, 256)
    f = _no_lens_field(0.2, 0.1, g, w)
    counts, oow = shoot_gpu(f)
    ref, oow_ref = oracle.shoot_field(f)
    assert np.array_equal(counts, ref) and oow == oow_ref


def test_nonsquare_grid_window_layout():
    g = ri.RayGrid(origin=(-2.0 + 2 ** -9, -2.0 + 2 ** -8), spacing=(2 ** -8, 2 ** -7), n=(1024, 512))
    w = ri.Window(lo=(0.0, -2.0), hi=(4.0, 2.0), npix=(256, 128))
    f = _no_lens_field(0.0, 0.0, g, w)
    counts, oow = shoot_gpu(f)
    ref, oow_ref = oracle.shoot_field(f)
    assert counts.shape == (128, 256)
    assert np.array_equal(counts, ref) and oow == oow_ref == g.n_rays // 2


def _check_per_ray(spec, ij, label, rigorous=True, band_check=True):
    """Per-ray source positions.

    float32 path: within the rigorous operation-count bound for every ray, and (band_check) within its
    own band half-width (the estimate certified binning relies on) for every ray.
    float-float path (certified re-evaluation): within the 1e-5-pixel per-ray tolerance.
    """
    y_gpu, band = trace_gpu(spec, ij)
    y_ff, _ = trace_gpu(spec, ij, certified=True)
    y_ref, _, x = oracle.trace_field(spec, ij)
    fin = np.isfinite(y_ref).all(1)
    assert np.array_equal(fin, np.isfinite(y_gpu).all(1))
    assert np.array_equal(fin, np.isfinite(y_ff).all(1))
    err = np.abs(y_gpu[fin] - y_ref[fin])
    if rigorous:
        bound = per_ray_bound(spec, x[fin], y_ref[fin])
        assert np.all(err.max(1) <= bound), (label, float((err.max(1) / bound).max()))
    if band_check:
        assert np.all(err <= band[fin]), (label, float((err / band[fin]).max()))
    st = error_stats(y_gpu, y_ref, spec.window)
    st_ff = error_stats(y_ff, y_ref, spec.window)
    print(f"{label} float32 per-ray error (pixels): {st}; worst error / band = "
          f"{float((err / band[fin]).max()):.3f}")
    print(f"{label} float-float per-ray error (pixels): {st_ff}")
    assert st_ff["max"] <= PER_RAY_TOL_PIX
    return y_gpu, y_ref, st


def test_tiny_field_full_map_and_every_ray():
    """100 lenses, 1000^2 rays, 256^2 map: every ray traced against the oracle; the certified
    map equals the oracle's map; without certification the map is the binning of the traced rays."""
    f = ri.tiny_field()
    counts, oow = shoot_gpu(f)
    assert int(counts.sum()) + oow == f.grid.n_rays
    y_gpu, y_ref, st = _check_per_ray(f, all_rays(f.grid), "tiny field")
    assert st["p50"] <= 3e-5 and st["p99"] <= 2e-4
    ref, oow_ref = oracle.shoot_field(f)
    assert np.array_equal(counts, ref) and oow == oow_ref
    m = rs()
    m.rs_set_certified_binning(False)
    try:
        fast, _ = shoot_gpu(f)
    finally:
        m.rs_set_certified_binning(True)
    p = pixel_index(y_gpu, f.window)
    rebinned = np.bincount(p[p >= 0], minlength=f.window.n_pix).reshape(counts.shape)
    assert np.array_equal(rebinned, fast)
    flips = int((p != pixel_index(y_ref, f.window)).sum())
    print("tiny field float32 flips (uncertified):", flips, "of", p.size)
    assert flips / p.size <= FLIP_FRAC_TOL


def test_point_lens_map():
    g = ri.cell_centred_grid(-8.0, 8.0, 4096)
    w = ri.square_window(3.0, 120)
    f = ri.Field("point", np.zeros((1, 2), np.float32), None, 0.0, 0.0, g, w)
    counts, oow = shoot_gpu(f)
    ref, oow_ref = oracle.shoot_field(f)
    assert int(counts.sum()) + oow == g.n_rays
    diff = np.abs(counts.astype(np.int64) - ref.astype(np.int64))
    assert diff.sum() <= 2e-5 * g.n_rays
    assert np.all(diff <= np.maximum(1, 1e-3 * ref))


def test_launch_shapes_and_runs_bitwise_identical():
    m = rs()
    f = ri.disc_field("mixed", 777, 0.5, 0.05, 0.2, 300, 96, seed=5, mass="salpeter")
    f0 = ri.disc_field("equal", 513, 0.4, 0.0, 0.3, 300, 96, seed=6, mass="equal")
    for spec in (f, f0):
        has_m = spec.masses is not None
        saved = m.rs_get_launch_config(has_m)
        results = []
        try:
            for shape in m.rs_launch_configs():
                m.rs_set_launch_config(has_m, *shape)
                results.append(shoot_gpu(spec))
                results.append(shoot_gpu(spec))
        finally:
            m.rs_set_launch_config(has_m, *saved)
        for c, o in results[1:]:
            assert np.array_equal(c, results[0][0]) and o == results[0][1]


def test_row_sharding_accumulates_bitwise():
    f = ri.disc_field("shard", 300, 0.5, 0.1, 0.25, 257, 64, seed=8, mass="salpeter")
    full, oow_full = shoot_gpu(f)
    counts = torch.zeros((64, 64), dtype=torch.int32, device=dev())
    oow = torch.zeros(1, dtype=torch.int64, device=dev())
    for rows in ((0, 1), (1, 100), (100, 100), (100, 257)):
        shoot_gpu(f, rows=rows, counts=counts, oow=oow)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), full) and int(oow.item()) == oow_full


def test_sharded_step_single_process_equals_plain_shoot():
    """shoot_sharded with the device row shooter (one process: no collective) on a block of rows equals
    rs_shoot_rows of the block, bit for bit (the benchmark's N = 1 sharded step)."""
    m = rs()
    from paper_0905_2453_gb300.shard import device_row_shooter, shoot_sharded
    spec = ri.disc_field("shard1", 700, 0.5, 0.1, 0.25, 600, 96, seed=12, mass="salpeter")
    f = m.Field.from_spec(spec)
    try:
        npix = (int(spec.window.npix[1]), int(spec.window.npix[0]))
        c1 = torch.zeros(npix, dtype=torch.int32, device=dev())
        o1 = torch.zeros(1, dtype=torch.int64, device=dev())
        c2, o2 = torch.zeros_like(c1), torch.zeros_like(o1)
        blk = shoot_sharded(device_row_shooter(f, spec.grid, spec.window), 200, c1, o1, 0, 1, row_begin=150)
        m.rs_shoot_rows(f.handle, spec.grid, 150, 350, spec.window, c2, o2)
        torch.cuda.synchronize()
        assert blk == (150, 350)
        assert torch.equal(c1, c2) and int(o1.item()) == int(o2.item())
        assert int(c1.sum().item()) + int(o1.item()) == 200 * spec.grid.n[0]
    finally:
        f.close()


RAGGED_LENS_COUNTS = (1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 1279)


def _ragged_field(n_lens):
    return ri.disc_field(f"rag{n_lens}", n_lens, 0.3, 0.0, 0.1, 37, 16, seed=n_lens, mass="salpeter")


def test_ragged_sizes_and_edge_cases():
    """Lens counts around the float32 group (64 lenses), the lens pair, the lens tile and renormalisation
    period (256) and the padding (1024), one ray, rays off the tile size: every ray within the rigorous
    bound, the float-float path within 1e-5 px, rays conserved."""
    for n_lens in RAGGED_LENS_COUNTS:
        f = _ragged_field(n_lens)
        ij = all_rays(f.grid)
        _check_per_ray(f, ij, f"ragged N={n_lens}", band_check=False)
        counts, oow = shoot_gpu(f)
        assert int(counts.sum()) + oow == f.grid.n_rays
    # a single ray
    f = ri.tiny_field()
    g1 = ri.RayGrid(origin=(0.3, -0.7), spacing=(1.0, 1.0), n=(1, 1))
    counts, oow = shoot_gpu(f, grid=g1)
    assert int(counts.sum()) + oow == 1
    # empty grid: nothing launched, nothing counted
    g0 = ri.RayGrid(origin=(0.0, 0.0), spacing=(1.0, 1.0), n=(0, 5))
    counts, oow = shoot_gpu(f, grid=g0)
    assert counts.sum() == 0 and oow == 0


def test_band_covers_float32_error_on_few_lens_fields():
    """Few lenses in a small disc put many rays between lenses at distances of order 1, where the terms
    of one group cancel and the group partials understate the float32 error: the band with its near-lens
    term (16 u times the ray's largest-term bound) against the float32 error there."""
    worst = []
    for n_lens in RAGGED_LENS_COUNTS:
        f = _ragged_field(n_lens)
        ij = all_rays(f.grid)
        y_gpu, band = trace_gpu(f, ij)
        y_ref, _, _ = oracle.trace_field(f, ij)
        fin = np.isfinite(y_ref).all(1)
        worst.append((n_lens, float((np.abs(y_gpu[fin] - y_ref[fin]) / band[fin]).max())))
    print("worst float32 error / band per lens count:", worst)
    assert all(r <= 1.0 for _, r in worst), worst


@pytest.mark.parametrize("n_lens,mass,kappa", [(3, "salpeter", 0.3), (63, "salpeter", 0.3), (100, "equal", 0.3)])
def test_few_lens_certified_full_map_equals_oracle(n_lens, mass, kappa):
    """Few-lens fields, 1024^2 rays, 256^2 pixels about as wide as the ray spacing (many rays next to
    pixel edges, many between near lenses): the certified map and out-of-window count equal the
    oracle's bit for bit, and every ray is counted once."""
    f = ri.disc_field(f"few{n_lens}", n_lens, kappa, 0.0, 0.1, 1024, 256, seed=100 + n_lens, mass=mass)
    counts, oow = shoot_gpu(f)
    assert int(counts.sum()) + oow == f.grid.n_rays
    ref, oow_ref = oracle.shoot_field(f)
    moved = int(np.abs(counts.astype(np.int64) - ref.astype(np.int64)).sum()) // 2 + abs(oow - oow_ref)
    print(f"{n_lens} lenses: certified map, rays moved {moved} of {f.grid.n_rays}")
    assert np.array_equal(counts, ref) and oow == oow_ref


def test_ray_on_lens_is_out_of_window():
    g = ri.RayGrid(origin=(-1.0, -1.0), spacing=(0.25, 0.25), n=(9, 9))
    w = ri.Window(lo=(-100.0, -100.0), hi=(100.0, 100.0), npix=(4, 4))
    f = ri.Field("onlens", np.zeros((1, 2), np.float32), None, 0.0, 0.0, g, w)
    counts, oow = shoot_gpu(f)
    assert oow == 1 and counts.sum() == 80


def test_magnification_matches_oracle():
    f = ri.tiny_field()
    counts, _ = shoot_gpu(f)
    m = rs()
    c = torch.from_numpy(counts.view(np.int32).copy()).to(dev())
    mu = m.magnification(c, f.grid, f.window).cpu().numpy()
    mu_ref = oracle.magnification(counts, f.grid.spacing, f.window.lo, f.window.hi, f.window.npix)
    assert np.allclose(mu, mu_ref, rtol=2e-7, atol=0)


@pytest.mark.parametrize("n_lens,mass,side", [(100, "equal", 1024), (700, "salpeter", 768), (1024, "equal", 768)])
def test_small_field_maps_agree_across_shoot_paths(n_lens, mass, side):
    """Certified maps of small fields from rs_shoot (stream-ordered list), rs_shoot_rows_noalloc (static list)
    and rs_shoot_staged (lens partitions of 256, re-evaluated partition by partition) agree bit for bit
    (and the 100-lens one with the oracle's)."""
    m = rs()
    spec = ri.disc_field(f"paths-{n_lens}", n_lens, 0.45, 0.05, 0.3, side, 256, seed=11, mass=mass)
    n1 = int(spec.grid.n[1])
    w = spec.window
    cuts = list(range(0, n_lens, 256)) + [n_lens]
    f = m.Field.from_spec(spec)
    parts = [m.Field(spec.lens_xy[a:b], None if spec.masses is None else spec.masses[a:b], spec.kappa_c,
                     spec.gamma) for a, b in zip(cuts, cuts[1:])]
    try:
        maps = []
        for call in (lambda c, o: m.rs_shoot(f.handle, spec.grid, w, c, o),
                     lambda c, o: m.rs_shoot_rows_noalloc(f.handle, spec.grid, 0, n1, w, c, o),
                     lambda c, o: m.rs_shoot_staged([p.handle for p in parts], spec.grid, 0, n1, w, c, o)):
            c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
            o = torch.zeros(1, dtype=torch.int64, device=dev())
            call(c, o)
            torch.cuda.synchronize()
            maps.append((c.cpu().numpy().view(np.uint32), int(o.item())))
        assert f.status() == m.RS_OK and all(p.status() == m.RS_OK for p in parts)
        for k in (1, 2):
            assert np.array_equal(maps[0][0], maps[k][0]) and maps[0][1] == maps[k][1], k
        assert int(maps[0][0].sum()) + maps[0][1] == spec.grid.n_rays
        if n_lens == 100:
            ref, oref = oracle.shoot_field(spec)
            assert np.array_equal(maps[0][0], ref) and maps[0][1] == oref
    finally:
        f.close()
        for p in parts:
            p.close()


@pytest.mark.parametrize("mass", ["equal", "salpeter"])
def test_large_field_re_evaluation_several_rays_per_pass_bitwise(mass):
    """Above 2^16 lenses the listed rays of one field are re-evaluated several per pass over the lenses
    (rs_shoot) and one per pass in a batch: each ray's float-float sum has the same order either way, so the
    maps are the same bits."""
    m = rs()
    spec = ri.disc_field(f"rays-per-pass-{mass}", 70_000, 0.45, 0.05, 0.3, 1024, 256, seed=12, mass=mass)
    f = m.Field.from_spec(spec)
    try:
        assert (spec.n_lens > 1 << 16) and m.rs_get_certified_binning()
        w = spec.window
        c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot(f.handle, spec.grid, w, c, o)
        b = m.Batch([f], [spec.grid], [w])
        b.launch()
        torch.cuda.synchronize()
        assert f.status() == m.RS_OK
        assert torch.equal(b.counts[0], c) and int(b.out_of_window[0].item()) == int(o.item())
        assert int(c.sum().item()) + int(o.item()) == spec.grid.n_rays
        b.close()
    finally:
        f.close()


def test_batch_equals_plain_launches_bitwise():
    m = rs()
    specs = ri.batch_fields(n_fields=6, ray_scale=0.125)
    specs.append(ri.disc_field("eq", 200, 0.3, 0.0, 0.2, 160, 48, seed=3, mass="equal"))
    fields = [m.Field.from_spec(s) for s in specs]
    try:
        b = m.Batch(fields, [s.grid for s in specs], [s.window for s in specs])
        for rep in range(2):  # the graph zeroes the maps on every launch
            b.launch()
            torch.cuda.synchronize()
            for k, s in enumerate(specs):
                ref, oow_ref = shoot_gpu(s)
                assert np.array_equal(b.counts[k].cpu().numpy().view(np.uint32), ref), (rep, k)
                assert int(b.out_of_window[k].item()) == oow_ref
        b.close()
    finally:
        for fl in fields:
            fl.close()


def test_batch_with_per_field_shapes_equals_plain_launches(tmp_path):
    """A batch whose fields take different launch shapes (every compiled shape in turn, then the tuner's per
    lens-count bucket choice) gives each field's plain-launch counts bit for bit."""
    m = rs()
    from paper_0905_2453_gb300 import tune
    specs = ri.batch_fields(n_fields=7, ray_scale=0.125)
    specs.append(ri.disc_field("eq", 200, 0.3, 0.0, 0.2, 160, 48, seed=3, mass="equal"))
    fields = [m.Field.from_spec(s) for s in specs]
    try:
        all_shapes = m.rs_launch_configs()
        cycled = [all_shapes[k % len(all_shapes)] for k in range(len(specs))]
        tuned = tune.batch_shapes(fields, [s.grid for s in specs], [s.window for s in specs],
                                  cache_path=str(tmp_path / "tune.json"), reps=1)
        assert all(tuple(sh) in [tuple(x) for x in all_shapes] for sh in tuned)
        refs = [shoot_gpu(s) for s in specs]
        for shapes in (cycled, tuned):
            b = m.Batch(fields, [s.grid for s in specs], [s.window for s in specs], shapes=shapes)
            try:
                b.launch()
                torch.cuda.synchronize()
                for k in range(len(specs)):
                    assert np.array_equal(b.counts[k].cpu().numpy().view(np.uint32), refs[k][0]), (shapes[k], k)
                    assert int(b.out_of_window[k].item()) == refs[k][1]
            finally:
                b.close()
    finally:
        for fl in fields:
            fl.close()


def test_batch_workload_full_size_vs_oracle():
    """The 64-field batch at full size, one persistent launch as the benchmark times it: every field's
    counts conserve its rays and equal its plain launch bit for bit, and the eight smallest fields
    (1.3e8 - 3.3e8 interactions each) equal the oracle's maps exactly (certified binning)."""
    m = rs()
    specs = ri.batch_fields(64)
    fields = [m.Field.from_spec(s) for s in specs]
    try:
        b = m.Batch(fields, [s.grid for s in specs], [s.window for s in specs])
        try:
            b.launch()
            torch.cuda.synchronize()
            got = [(b.counts[k].cpu().numpy().view(np.uint32).copy(), int(b.out_of_window[k].item()))
                   for k in range(len(specs))]
        finally:
            b.close()
        assert all(f.status() == m.RS_OK for f in fields)
    finally:
        for fl in fields:
            fl.close()
    for k, s in enumerate(specs):
        c, o = got[k]
        assert int(c.sum(dtype=np.int64)) + o == s.grid.n_rays, k
        ref, oref = shoot_gpu(s)
        assert np.array_equal(c, ref) and o == oref, k
    for k in sorted(range(len(specs)), key=lambda k: specs[k].interactions)[:8]:
        ref, oref = oracle.shoot_field(specs[k])
        assert np.array_equal(got[k][0], ref) and got[k][1] == oref, k


def test_n1e4_full_size_sampled_rays():
    """1e4 lenses on the 4096^2 grid in the benchmark's launch shape: 20000 sampled rays vs the oracle."""
    f = ri.n1e4_field()
    ij = ri.sample_rays(f.grid, 20000, seed=123)
    y_gpu, y_ref, st = _check_per_ray(f, ij, "N=1e4")
    assert st["p50"] <= 3e-5 and st["p99"] <= 2e-4
    counts, oow = shoot_gpu(f)
    assert int(counts.sum()) + oow == f.grid.n_rays


def test_n1e4_full_map_vs_oracle():
    """The whole 4096^2-ray, 1024^2-pixel map of the 1e4-lens field against the oracle's map."""
    f = ri.n1e4_field()
    counts, oow = shoot_gpu(f)
    ref, oow_ref = oracle.shoot_field(f)
    d = counts.astype(np.int64) - ref.astype(np.int64)
    moved = int(np.abs(d).sum()) // 2 + abs(oow - oow_ref)
    print("N=1e4 full map: rays moved (lower bound on flips)", moved, "of", f.grid.n_rays)
    assert moved <= FLIP_FRAC_TOL * f.grid.n_rays
    assert np.all(np.abs(d) <= np.maximum(1, 1e-3 * ref))


def test_map_of_1e8_rays_flips_and_pixels():
    """1.05e8 rays (10240^2 over [-10, 10]^2) through the 100-lens field: the certified map
    against the oracle's map -- per-pixel |N - N_oracle| <= max(1, 1e-3 N_oracle) and at most
    1e-5 of the rays moved; and the float32 path alone (uncertified) measured per ray."""
    base = ri.tiny_field()
    g = ri.cell_centred_grid(-10.0, 10.0, 10240)
    f = ri.Field("tiny-1e8", base.lens_xy, base.masses, 0.0, 0.0, g, base.window)
    counts, oow = shoot_gpu(f)
    ref, oow_ref = oracle.shoot_field(f)
    assert int(counts.sum()) + oow == g.n_rays
    d = counts.astype(np.int64) - ref.astype(np.int64)
    moved = int(np.abs(d).sum()) // 2 + abs(oow - oow_ref)
    print("1e8-ray certified map: rays moved", moved, "of", g.n_rays)
    assert moved <= FLIP_FRAC_TOL * g.n_rays
    assert np.all(np.abs(d) <= np.maximum(1, 1e-3 * ref))
    # float32 decisions alone: per-ray flips, every 4th row block
    flips, n = 0, 0
    for jb in range(0, 10240, 2048):
        ij = all_rays(g, rows=(jb, jb + 512))
        y_gpu, _ = trace_gpu(f, ij)
        y_ref, _, _ = oracle.trace_field(f, ij)
        flips += int((pixel_index(y_gpu, f.window) != pixel_index(y_ref, f.window)).sum())
        n += ij.shape[0]
    print("float32-only flips:", flips, "of", n)
    assert flips <= FLIP_FRAC_TOL * n


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    """A wait that nothing completes gives up after its limit with RS_ETIMEOUT (no hang, no fault),
    and the device keeps working afterwards."""
    m = rs()
    assert m.rs_selftest_bounded_wait(10_000_000) == m.RS_ETIMEOUT
    f = ri.tiny_field()
    counts, oow = shoot_gpu(f)
    assert int(counts.sum()) + oow == f.grid.n_rays


def test_certified_trace_matches_oracle_large_fields():
    """Float-float re-evaluation on the 1e6-lens Salpeter field: sampled rays within 1e-5 pixel."""
    f = ri.n1e6_salpeter_field()
    ij = ri.sample_rays(f.grid, 512, seed=9)
    y_ff, _ = trace_gpu(f, ij, certified=True)
    y_ref, _, _ = oracle.trace_field(f, ij)
    st = error_stats(y_ff, y_ref, f.window)
    print("N=1e6 float-float per-ray error (pixels):", st)
    assert st["max"] <= PER_RAY_TOL_PIX


def test_n1e6_salpeter_sampled_rays_float32_and_map_invariants():
    """1e6 Salpeter lenses, 16384^2 grid: 1e5 sampled rays (float32 path within its band, float-float
    within 1e-5 px; the rigorous operation-count bound on 256 of them), and the certified map of a
    1024-row block conserves rays."""
    f = ri.n1e6_salpeter_field()
    ij = ri.sample_rays(f.grid, 100000, seed=31)
    _check_per_ray(f, ij[:256], "N=1e6 (bound)")
    y_gpu, y_ref, st = _check_per_ray(f, ij, "N=1e6", rigorous=False)
    counts, oow = shoot_gpu(f, rows=(7680, 8704))
    assert int(counts.sum()) + oow == 1024 * f.grid.n[0]


def test_n1e8_sampled_rays():
    """1e8 lenses with stored unit masses (2.4 GB on the device), 8192^2 grid: 512 sampled rays."""
    f = ri.n1e8_field()
    ij = ri.sample_rays(f.grid, 512, seed=41)
    _check_per_ray(f, ij, "N=1e8", rigorous=False)


def test_far_from_origin_certified_map():
    """Lenses, rays and window far from the origin (|y| ~ 3e4, pixels of 2e-3): the float-float epilogue
    must resolve u = (y - lo) / pix where y and lo nearly cancel; the certified map equals the oracle's."""
    cx, cy = 30000.0, -20000.0
    rng = np.random.default_rng(17)
    r = 6.0 * np.sqrt(rng.random(60))
    th = 2 * np.pi * rng.random(60)
    xy = np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], 1).astype(np.float32)
    g = ri.RayGrid(origin=(cx - 4.0 + 1 / 256, cy - 4.0 + 1 / 256), spacing=(1 / 128, 1 / 128), n=(1024, 1024))
    # no shear, no smooth convergence: y ~ x - alpha stays near (cx, cy)
    w = ri.Window(lo=(cx - 0.25, cy - 0.25), hi=(cx + 0.25, cy + 0.25), npix=(250, 250))
    f = ri.Field("far", xy, None, 0.0, 0.0, g, w)
    counts, oow = shoot_gpu(f)
    ref, oref = oracle.shoot_field(f)
    assert counts.sum() > 0
    assert np.array_equal(counts, ref) and oow == oref


def test_certified_list_overflow_is_reported():
    """Pixels far narrower than the rays' error bands make nearly every in-window ray uncertain, so the
    re-evaluation list (rays / 32 entries) overflows: the field's status reports RS_EOVERFLOW (those rays
    kept their float32 decision); after clearing, a normal shoot reports RS_OK."""
    m = rs()
    xy, _ = ri.disc_lenses(50, 5.0, seed=9)
    g = ri.RayGrid(origin=(-1.0 + 1 / 1024, -1.0 + 1 / 1024), spacing=(1 / 512, 1 / 512), n=(1024, 1024))
    thin = ri.Window(lo=(-0.5, -2.0), hi=(0.5, 2.0), npix=(1 << 22, 1))
    normal = ri.Window(lo=(-2.0, -2.0), hi=(2.0, 2.0), npix=(64, 64))
    f = m.Field(xy)
    try:
        c = torch.zeros((1, 1 << 22), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        f.shoot(g, thin, c, o)
        assert f.status(clear=True) == m.RS_EOVERFLOW
        assert int(c.sum().item()) + int(o.item()) == g.n_rays        # every ray still counted once
        assert f.status() == m.RS_OK
        f.shoot(g, normal)
        assert f.status() == m.RS_OK
    finally:
        f.close()
