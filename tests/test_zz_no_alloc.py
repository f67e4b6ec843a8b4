"""The allocation-free shoot (rs_shoot_rows_noalloc) against the allocating one (rs_shoot).

Some callers cannot allocate device memory while they run (work replayed in a CUDA graph whose
capture must not contain allocation nodes, applications whose allocator reserved the device
memory up front); rs_shoot_rows_noalloc serves them with a static device array for its list of
rays to re-evaluate.  This file is collected last on purpose, and it must pass both alone in a
fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import rs_inputs as ri
from gpu_helpers import dev, rs

pytestmark = pytest.mark.gpu


def _call(lib, m, field, grid, window, rows, counts, oow):
    g, w = m._cgrid(grid), m._cwin(window)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.rs_shoot_rows_noalloc(field.handle, ctypes.byref(g), int(rows[0]), int(rows[1]), ctypes.byref(w),
                                     counts.data_ptr(), oow.data_ptr(), stream)


def _shoot(m, field, grid, window, certified):
    counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev())
    oow = torch.zeros(1, dtype=torch.int64, device=dev())
    m.rs_set_certified_binning(certified)
    try:
        m.rs_shoot(field.handle, grid, window, counts, oow)
        torch.cuda.synchronize()
    finally:
        m.rs_set_certified_binning(True)
    return counts, int(oow.item())


def test_noalloc_equals_allocating_shoot_twice_in_a_row():
    """Two calls in a row with different windows, each against the allocating certified shoot.  The
    first window is a strip of pixels narrow enough that the float32 decision alone moves some rays
    (so a broken re-evaluation list would show in the map); the second call reuses the array the first
    one filled, on another window, so stale entries would show too."""
    m = rs()
    lib = m.load()
    spec = ri.disc_field("noalloc", 63, 0.3, 0.0, 0.1, 1024, 256, seed=21, mass="salpeter")
    field = m.Field.from_spec(spec)
    s = float(spec.window.hi[0])
    try:
        strip = None
        for npix0 in (16384, 65536, 262144):  # narrower pixels until the float32 decision alone moves rays
            w = ri.Window(lo=(-s, -s), hi=(s, s), npix=(npix0, 1))
            ref, ref_oow = _shoot(m, field, spec.grid, w, True)
            fast, _ = _shoot(m, field, spec.grid, w, False)
            if field.status(clear=True) == m.RS_OK and not torch.equal(ref, fast):
                strip = (w, ref, ref_oow)
                break
        assert strip is not None, "no window made the float32 decision move a ray"
        windows = [strip, (spec.window,) + _shoot(m, field, spec.grid, spec.window, True)]
        for call, (w, ref, ref_oow) in enumerate(windows):
            counts = torch.zeros_like(ref)
            oow = torch.zeros(1, dtype=torch.int64, device=dev())
            rc = _call(lib, m, field, spec.grid, w, (0, spec.grid.n[1]), counts, oow)
            assert rc == m.RS_OK, m.rs_last_error()
            torch.cuda.synchronize()
            assert torch.equal(counts, ref), f"call {call}: maps differ"
            assert int(oow.item()) == ref_oow
            assert int(counts.sum().item()) + int(oow.item()) == spec.grid.n_rays
        assert field.status() == m.RS_OK
    finally:
        field.close()


def test_noalloc_rejects_more_rays_than_its_list_covers():
    m = rs()
    lib = m.load()
    spec = ri.tiny_field()
    field = m.Field.from_spec(spec)
    try:
        big = ri.RayGrid(origin=(-10.0, -10.0), spacing=(1e-3, 1e-3), n=(8192, 4096))
        counts = torch.zeros((256, 256), dtype=torch.int32, device=dev())
        oow = torch.zeros(1, dtype=torch.int64, device=dev())
        # 2^24 + 8192 rays: one row more than the limit
        rc = _call(lib, m, field, big, spec.window, (0, 2049), counts, oow)
        assert rc == m.RS_EOVERFLOW
        assert "2^24" in m.rs_last_error()
        # exactly 2^24 rays fit
        rc = _call(lib, m, field, big, spec.window, (0, 2048), counts, oow)
        assert rc == m.RS_OK, m.rs_last_error()
        torch.cuda.synchronize()
        assert int(counts.sum().item()) + int(oow.item()) == 8192 * 2048
    finally:
        field.close()
