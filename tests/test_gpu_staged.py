"""Lens-partitioned (staged) shooting, Section 3.3: a field given as several lens partitions, the
partially deflected rays carried between passes, must give the counts of one pass over all lenses
bit for bit (float32 path alone, and with certified binning), and the oracle's map."""
import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import dev, rs, shoot_gpu

pytestmark = pytest.mark.gpu


def _staged(spec, cuts, grid=None, window=None, rows=None):
    m = rs()
    g, w = grid or spec.grid, window or spec.window
    bounds = [0] + list(cuts) + [spec.n_lens]
    parts = [m.Field(spec.lens_xy[a:b], None if spec.masses is None else spec.masses[a:b], spec.kappa_c, spec.gamma)
             for a, b in zip(bounds[:-1], bounds[1:])]
    try:
        c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        r0, r1 = rows or (0, int(g.n[1]))
        m.rs_shoot_staged([p.handle for p in parts], g, r0, r1, w, c, o)
        torch.cuda.synchronize()
        for p in parts:
            assert p.status() == m.RS_OK
        return c.cpu().numpy().view(np.uint32), int(o.item())
    finally:
        for p in parts:
            p.close()


@pytest.mark.parametrize("certify", [True, False])
@pytest.mark.parametrize("mass", ["equal", "salpeter"])
def test_partitions_equal_single_pass(certify, mass):
    m = rs()
    m.rs_set_certified_binning(certify)
    try:
        spec = ri.disc_field("st", 1000, 0.5, 0.1, 0.25, 1024, 128, seed=21, mass=mass)
        ref, oref = shoot_gpu(spec)
        for cuts in ([256], [256, 512], [256, 512, 768], [768]):
            got, o = _staged(spec, cuts)
            assert np.array_equal(got, ref) and o == oref, cuts
    finally:
        m.rs_set_certified_binning(True)


def test_row_blocks_and_rows_match():
    """A small state budget forces several row blocks; a row range of the grid; the oracle's map."""
    m = rs()
    spec = ri.disc_field("stb", 700, 0.4, 0.0, 0.3, 1000, 96, seed=4, mass="equal")
    m.rs_set_staged_state_budget(1 << 20)
    try:
        got, o = _staged(spec, [256, 512])
        got_rows, o_rows = _staged(spec, [512], rows=(100, 731))
    finally:
        m.rs_set_staged_state_budget(2 << 30)
    ref, oref = oracle.shoot_field(spec)
    assert np.array_equal(got, ref) and o == oref
    ref_rows, oref_rows = shoot_gpu(spec, rows=(100, 731))
    assert np.array_equal(got_rows, ref_rows) and o_rows == oref_rows


def test_partition_validation():
    m = rs()
    spec = ri.disc_field("stv", 600, 0.4, 0.0, 0.3, 256, 32, seed=2, mass="equal")
    a = m.Field(spec.lens_xy[:300], None, 0.0, 0.3)
    b = m.Field(spec.lens_xy[300:], None, 0.0, 0.3)
    c = m.Field(spec.lens_xy[300:], None, 0.1, 0.3)
    counts = torch.zeros((32, 32), dtype=torch.int32, device=dev())
    try:
        for hs in ([a.handle, b.handle], [b.handle, c.handle], []):
            with pytest.raises(m.RSError) as ei:
                m.rs_shoot_staged(hs, spec.grid, 0, int(spec.grid.n[1]), spec.window, counts)
            assert ei.value.code == m.RS_EINVAL
    finally:
        for f in (a, b, c):
            f.close()


def test_n1e4_in_four_partitions():
    spec = ri.n1e4_field()
    ref, oref = shoot_gpu(spec)
    got, o = _staged(spec, [2560, 5120, 7680])
    assert np.array_equal(got, ref) and o == oref


def _streamed(spec, per_pass, rows=None, window=None):
    m = rs()
    g, w = spec.grid, window or spec.window
    c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
    o = torch.zeros(1, dtype=torch.int64, device=dev())
    r0, r1 = rows or (0, int(g.n[1]))
    m.rs_shoot_streamed(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, per_pass, g, r0, r1, w, c, o)
    return c.cpu().numpy().view(np.uint32), int(o.item())


@pytest.mark.parametrize("certify", [True, False])
@pytest.mark.parametrize("mass", ["equal", "salpeter"])
def test_streamed_from_host_equals_single_pass(certify, mass):
    """Lenses streamed from host memory 1024 or 3072 at a time (5 or 2 passes)."""
    m = rs()
    m.rs_set_certified_binning(certify)
    try:
        spec = ri.disc_field("ss", 5000, 0.5, 0.05, 0.2, 768, 96, seed=31, mass=mass)
        ref, oref = shoot_gpu(spec)
        for per_pass in (1024, 3072):
            got, o = _streamed(spec, per_pass)
            assert np.array_equal(got, ref) and o == oref, per_pass
    finally:
        m.rs_set_certified_binning(True)


def test_streamed_row_blocks_rows_and_empty_field():
    m = rs()
    spec = ri.disc_field("ssb", 2500, 0.4, 0.0, 0.3, 800, 80, seed=6, mass="equal")
    m.rs_set_staged_state_budget(1 << 20)
    try:
        got, o = _streamed(spec, 1024)
        got_rows, o_rows = _streamed(spec, 2048, rows=(33, 500))
    finally:
        m.rs_set_staged_state_budget(2 << 30)
    ref, oref = oracle.shoot_field(spec)
    assert np.array_equal(got, ref) and o == oref
    ref_rows, oref_rows = shoot_gpu(spec, rows=(33, 500))
    assert np.array_equal(got_rows, ref_rows) and o_rows == oref_rows
    empty = ri.Field("e", np.zeros((0, 2), np.float32), None, 0.1, 0.2, spec.grid, spec.window)
    got0, o0 = _streamed(empty, 1024)
    ref0, oref0 = oracle.shoot_field(empty)
    assert np.array_equal(got0, ref0) and o0 == oref0
    with pytest.raises(m.RSError):
        _streamed(spec, 1000)                    # not a multiple of 1024
