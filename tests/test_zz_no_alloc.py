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


def test_noalloc_equals_allocating_shoot_twice_in_a_row():
    m = rs()
    lib = m.load()
    assert m.rs_get_certified_binning()  # the reference calls certify, as the variant always does
    spec = ri.disc_field("noalloc", 1500, 0.5, 0.05, 0.3, 2048, 256, seed=21, mass="salpeter")
    field = m.Field.from_spec(spec)
    try:
        npix = (int(spec.window.npix[1]), int(spec.window.npix[0]))
        ref = torch.zeros(npix, dtype=torch.int32, device=dev())
        ref_oow = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot(field.handle, spec.grid, spec.window, ref, ref_oow)
        torch.cuda.synchronize()
        for call in range(2):  # the static array keeps the previous call's contents
            counts = torch.zeros(npix, dtype=torch.int32, device=dev())
            oow = torch.zeros(1, dtype=torch.int64, device=dev())
            rc = _call(lib, m, field, spec.grid, spec.window, (0, spec.grid.n[1]), counts, oow)
            assert rc == m.RS_OK, m.rs_last_error()
            torch.cuda.synchronize()
            assert torch.equal(counts, ref), f"call {call}: maps differ"
            assert int(oow.item()) == int(ref_oow.item())
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
        big = ri.RayGrid(origin=(-10.0, -10.0), spacing=(1e-3, 1e-3), n=(8192, 4096))  # 2^25 rays
        counts = torch.zeros((256, 256), dtype=torch.int32, device=dev())
        oow = torch.zeros(1, dtype=torch.int64, device=dev())
        rc = _call(lib, m, field, big, spec.window, (0, 4096), counts, oow)
        assert rc == m.RS_EOVERFLOW
        assert "2^24" in m.rs_last_error()
        # half the rows fit
        rc = _call(lib, m, field, big, spec.window, (0, 2048), counts, oow)
        assert rc == m.RS_OK, m.rs_last_error()
        torch.cuda.synchronize()
        assert int(counts.sum().item()) + int(oow.item()) == 8192 * 2048
    finally:
        field.close()
