"""Lens-range views of a field (no copy).  Eq. 2 is a sum over lenses, so the deflections of views of
disjoint lens ranges add up to the whole field's; a view shoots exactly like a field created from the
same lenses; views cut at multiples of 256 lenses are resident partitions for the staged shoot
(Section 3.3) with the whole field's map bit for bit; a view of a moving field moves with it; and the
autotuner times very large fields on a view of their first lenses."""
import json

import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import all_rays, dev, rs, shoot_gpu

pytestmark = pytest.mark.gpu


def _spec(mass="salpeter", n=1500, seed=41):
    return ri.disc_field("vw", n, 0.5, 0.05, 0.3, 600, 72, seed=seed, mass=mass)


def _shoot(m, f, spec):
    g, w = spec.grid, spec.window
    c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
    o = torch.zeros(1, dtype=torch.int64, device=dev())
    f.shoot(g, w, c, o)
    torch.cuda.synchronize()
    assert f.status() == m.RS_OK
    return c.cpu().numpy().view(np.uint32), int(o.item())


@pytest.mark.parametrize("mass", ["equal", "salpeter"])
def test_view_shoots_like_a_field_of_its_lenses(mass):
    m = rs()
    spec = _spec(mass)
    parent = m.Field.from_spec(spec)
    try:
        for a, n in ((0, 1500), (256, 700), (1024, 476), (512, 0)):
            sub = ri.Field("vs", spec.lens_xy[a:a + n], None if spec.masses is None else spec.masses[a:a + n],
                           spec.kappa_c, spec.gamma, spec.grid, spec.window)
            v = parent.view(a, n)
            try:
                assert v.info() == (n, parent.info()[1])
                got = _shoot(m, v, spec)
            finally:
                v.close()
            ref = shoot_gpu(sub)
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1], (a, n)
            if n in (0, 476):
                oc, oo = oracle.shoot_field(sub)
                assert np.array_equal(got[0], oc) and got[1] == oo
    finally:
        parent.close()


def test_views_superpose_and_partition_the_staged_shoot():
    m = rs()
    spec = _spec("salpeter", n=2000, seed=8)
    parent = m.Field.from_spec(spec)
    views = [parent.view(0, 768), parent.view(768, 1024), parent.view(1792, 208)]
    try:
        # Eq. 2 is linear in the lens set: the float-float deflections of the views add up to the field's
        ij = all_rays(spec.grid, rows=(300, 302))
        _, a_all = parent.trace(spec.grid, ij, with_alpha=True, certified=True)
        parts = [v.trace(spec.grid, ij, with_alpha=True, certified=True)[1] for v in views]
        a_sum = sum(p.cpu().numpy() for p in parts)
        scale = np.abs(a_all.cpu().numpy()).max() + 1.0
        assert np.max(np.abs(a_sum - a_all.cpu().numpy())) < 1e-9 * scale
        # resident partitions for the staged shoot: the parent's map bit for bit
        g, w = spec.grid, spec.window
        c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot_staged([v.handle for v in views], g, 0, int(g.n[1]), w, c, o)
        torch.cuda.synchronize()
        ref = _shoot(m, parent, spec)
        assert np.array_equal(c.cpu().numpy().view(np.uint32), ref[0]) and int(o.item()) == ref[1]
        # the parent outlives its views
        with pytest.raises(m.RSError) as ei:
            m.rs_destroy_field(parent.handle)
        assert ei.value.code == m.RS_EINVAL
    finally:
        for v in views:
            v.close()
        parent.close()
    assert parent.handle is None


def test_view_validation_and_moving_parent():
    m = rs()
    spec = _spec("equal", n=1200, seed=3)
    vel = ri.lens_velocities(spec.n_lens, 0.2, seed=9)
    parent = m.Field(spec.lens_xy, None, spec.kappa_c, spec.gamma, velocities=vel)
    try:
        for a, n in ((100, 10), (-256, 10), (0, 1201), (1024, 177), (0, -1)):
            with pytest.raises(m.RSError) as ei:
                parent.view(a, n)
            assert ei.value.code == m.RS_EINVAL, (a, n)
        v = parent.view(256, 944)
        try:
            with pytest.raises(m.RSError):
                v.set_time(1.0)                      # views follow their parent's time
            parent.set_time(3.0)
            assert v.time == 3.0
            moved = oracle.lens_positions(spec.lens_xy, vel, 3.0)
            sub = ri.Field("vm", moved[256:], None, spec.kappa_c, spec.gamma, spec.grid, spec.window)
            got = _shoot(m, v, spec)
            ref = shoot_gpu(sub)
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
        finally:
            v.close()
    finally:
        parent.close()


def test_autotune_times_large_fields_on_a_prefix_view(tmp_path):
    m = rs()
    from paper_0905_2453_gb300 import tune
    spec = ri.disc_field("vt", 5000, 0.45, 0.0, 0.4, 1024, 128, seed=2, mass="equal")
    f = m.Field.from_spec(spec)
    old = m.rs_get_launch_config(False)
    cache = str(tmp_path / "tune.json")
    try:
        *shape, ms = tune.autotune(f, spec.grid, spec.window, cache_path=cache, force=True, reps=1,
                                   min_rays=1e6, max_proxy_lenses=1024)
        shape = tuple(shape)
        shapes = [tuple(x) for x in m.rs_launch_configs()]
        assert shape in shapes and len([k for k in ms if not k.endswith("/field")]) == len(shapes)
        assert m.rs_get_launch_config(False) == shape
        # the proxy's best shapes were timed again on the field itself; the choice is the best of those
        field_rates = tune.shape_rates(f, spec.grid, cache_path=cache)
        name = "x".join(str(v) for v in shape)
        assert 1 <= len(field_rates) <= 3 and max(field_rates, key=field_rates.get) == name, field_rates
        entry = next(iter(json.load(open(cache)).values()))
        assert entry["proxy_lenses"] == 1024
        assert f.status() == m.RS_OK
    finally:
        m.rs_set_launch_config(False, *old)
        f.close()
