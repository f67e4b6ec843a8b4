"""Culled shooting and zoom (Section 4's interactive zoom into a map): rs_shoot_culled must give the
counts and out-of-window count of rs_shoot bit for bit while shooting fewer rays, and a zoomed
sub-window must equal the oracle's map of the finer grid."""
import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import dev, rs, shoot_gpu

pytestmark = pytest.mark.gpu


def _culled(spec, grid=None, window=None, rows=None):
    m = rs()
    grid = grid or spec.grid
    window = window or spec.window
    f = m.Field.from_spec(spec)
    try:
        counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev())
        oow = torch.zeros(1, dtype=torch.int64, device=dev())
        shot = torch.zeros(1, dtype=torch.int64, device=dev())
        f.shoot(grid, window, counts, oow, rows=rows, culled=True, rays_shot=shot)
        torch.cuda.synchronize()
        assert f.status() == m.RS_OK
        return counts.cpu().numpy().view(np.uint32), int(oow.item()), int(shot.item())
    finally:
        f.close()


def _same_as_plain(spec, grid=None, window=None, rows=None):
    c, o, shot = _culled(spec, grid, window, rows)
    ref, oref = shoot_gpu(spec, grid=grid, window=window, rows=rows)
    assert np.array_equal(c, ref) and o == oref
    g = grid or spec.grid
    n = int(g.n[0]) * ((rows[1] - rows[0]) if rows else int(g.n[1]))
    assert shot <= n and int(c.sum()) + o == n
    return shot / max(1, n)


@pytest.mark.parametrize("certify", [True, False])
def test_tiny_field_windows_bitwise(certify):
    """Standard window, a small zoom window, a window nothing reaches, a window covering everything."""
    m = rs()
    m.rs_set_certified_binning(certify)
    try:
        spec = ri.tiny_field()
        fracs = [_same_as_plain(spec)]
        fracs.append(_same_as_plain(spec, window=ri.Window(lo=(0.5, -0.5), hi=(1.0, 0.0), npix=(64, 64))))
        fracs.append(_same_as_plain(spec, window=ri.Window(lo=(500.0, 500.0), hi=(501.0, 501.0), npix=(8, 8))))
        fracs.append(_same_as_plain(spec, window=ri.Window(lo=(-1e3, -1e3), hi=(1e3, 1e3), npix=(16, 16))))
        assert fracs[1] < 0.5 and fracs[2] < fracs[1] and fracs[3] == 1.0, fracs
    finally:
        m.rs_set_certified_binning(True)


def test_masses_shear_rows_and_ragged_grid():
    """Salpeter masses, convergence and shear, a ragged grid (not a multiple of the 16-ray cells), row blocks."""
    spec = ri.disc_field("z", 300, 0.5, 0.1, 0.3, 1000, 96, seed=8, mass="salpeter")
    g = ri.RayGrid(origin=spec.grid.origin, spacing=spec.grid.spacing, n=(1003, 997))
    w = spec.window
    sub = ri.Window(lo=(w.lo[0] * 0.3, w.lo[1] * 0.1), hi=(w.lo[0] * 0.1, w.hi[1] * 0.2), npix=(40, 24))
    _same_as_plain(spec, grid=g, window=w)
    _same_as_plain(spec, grid=g, window=sub)
    _same_as_plain(spec, grid=g, window=sub, rows=(17, 530))


def test_ray_on_lens_and_lens_in_cells():
    """A lens exactly on a ray (non-finite deflection: out of window) and lenses inside cells (always shot)."""
    g = ri.RayGrid(origin=(-1.0, -1.0), spacing=(0.25, 0.25), n=(40, 40))
    w = ri.Window(lo=(-3.0, -3.0), hi=(3.0, 3.0), npix=(8, 8))
    f = ri.Field("onlens", np.array([[0.0, 0.0], [2.3, 1.1]], np.float32), None, 0.0, 0.0, g, w)
    _same_as_plain(f)
    _same_as_plain(f, window=ri.Window(lo=(-0.2, -0.2), hi=(0.2, 0.2), npix=(4, 4)))


def test_zoom_matches_oracle_fine_map():
    """Zoom x3 into a sub-window of the tiny field's map: equals the oracle's map of the finer grid."""
    m = rs()
    spec = ri.tiny_field()
    f = m.Field.from_spec(spec)
    try:
        counts, g, w = f.zoom(spec.grid, spec.window, (0.25, -0.75), (1.0, 0.0), 3)
        torch.cuda.synchronize()
    finally:
        f.close()
    assert g.n == (3000, 3000) and w.npix == (144, 144)
    ref, _ = oracle.shoot(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, g.origin, g.spacing, g.n,
                          w.lo, w.hi, w.npix)
    got = counts.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)
    # same rays per pixel without lensing as the coarse map (N_av preserved)
    pa = ((w.hi[0] - w.lo[0]) / w.npix[0]) * ((w.hi[1] - w.lo[1]) / w.npix[1]) / (g.spacing[0] * g.spacing[1])
    pa0 = (4.0 / 256) ** 2 / (spec.grid.spacing[0] * spec.grid.spacing[1])
    assert abs(pa / pa0 - 1.0) < 1e-9


def test_n1e4_culled_equals_plain():
    """The 1e4-lens workload: full-map culled shooting equals the plain shoot bit for bit."""
    frac = _same_as_plain(ri.n1e4_field())
    assert frac < 0.9
