"""Failure detection without a GPU fault: injected allocation failures (the library's test hook) make each
allocating entry point return RS_ENOMEM, release what it had allocated, and leave the device usable; the
next call succeeds with correct results."""
import numpy as np
import pytest
import torch

import rs_inputs as ri
from gpu_helpers import dev, rs, shoot_gpu

pytestmark = pytest.mark.gpu


def _expect_enomem(m, fn):
    with pytest.raises(m.RSError) as ei:
        fn()
    assert ei.value.code == m.RS_ENOMEM
    m.rs_set_alloc_failure(-1)


def test_each_allocation_of_field_and_batch_creation_fails_cleanly():
    m = rs()
    spec = ri.disc_field("af", 300, 0.4, 0.0, 0.3, 256, 32, seed=1, mass="salpeter")
    free = []
    for rep in range(4):
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        for n in range(5):                        # field: lenses, masses, status, staging xy, staging m
            m.rs_set_alloc_failure(n)
            try:
                f = m.Field.from_spec(spec)       # n beyond the allocations made: succeeds
            except m.RSError as e:
                assert e.code == m.RS_ENOMEM
                continue
            finally:
                m.rs_set_alloc_failure(-1)
            f.close()
        f = m.Field.from_spec(spec)
        try:
            for n in range(5):                    # batch: descriptors, items, counter, list, list count
                m.rs_set_alloc_failure(n)
                try:
                    b = m.Batch([f], [spec.grid], [spec.window])
                    b.close()
                except m.RSError as e:
                    assert e.code == m.RS_ENOMEM
                finally:
                    m.rs_set_alloc_failure(-1)
        finally:
            f.close()
    # the first pass loads modules and creates the graph machinery; later passes must not lose memory
    assert free[3] >= free[1] - (8 << 20), free
    ref, oref = shoot_gpu(spec)                                    # the device is still usable
    assert int(ref.sum()) + oref == spec.grid.n_rays


def test_workspace_allocations_fail_cleanly_then_succeed():
    m = rs()
    spec = ri.disc_field("aw", 600, 0.4, 0.05, 0.3, 384, 48, seed=2, mass="equal")
    ref, oref = shoot_gpu(spec)
    f = m.Field.from_spec(spec)
    parts = [m.Field(spec.lens_xy[a:b], None, spec.kappa_c, spec.gamma) for a, b in ((0, 512), (512, 600))]
    w = spec.window
    try:
        def counts():
            return (torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev()),
                    torch.zeros(1, dtype=torch.int64, device=dev()))
        calls = {
            "shoot": lambda c, o: m.rs_shoot(f.handle, spec.grid, w, c, o),
            "culled": lambda c, o: m.rs_shoot_culled(f.handle, spec.grid, 0, int(spec.grid.n[1]), w, c, o),
            "staged": lambda c, o: m.rs_shoot_staged([p.handle for p in parts], spec.grid, 0, int(spec.grid.n[1]),
                                                     w, c, o),
            "streamed": lambda c, o: m.rs_shoot_streamed(spec.lens_xy, None, spec.kappa_c, spec.gamma, 1024,
                                                         spec.grid, 0, int(spec.grid.n[1]), w, c, o),
        }
        for name, call in calls.items():
            c, o = counts()
            m.rs_set_alloc_failure(0)
            _expect_enomem(m, lambda: call(c, o))
            torch.cuda.synchronize()
            c, o = counts()
            call(c, o)
            torch.cuda.synchronize()
            assert np.array_equal(c.cpu().numpy().view(np.uint32), ref) and int(o.item()) == oref, name
        mu = torch.ones((32, 32), dtype=torch.float32, device=dev())
        win = ri.Window(lo=(-1.0, -1.0), hi=(1.0, 1.0), npix=(32, 32))
        tr = [m.Track(0, (0.0, 0.0), (0.01, 0.0), 8)]
        m.rs_set_alloc_failure(0)
        _expect_enomem(m, lambda: m.light_curves([mu], [win], tr, m.RS_PROFILE_DISC, 0.2))
        got, _ = m.light_curves([mu], [win], tr, m.RS_PROFILE_DISC, 0.2)
        assert torch.all(got == 1.0)
    finally:
        f.close()
        for p in parts:
            p.close()
