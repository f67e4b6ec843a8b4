"""Masses that are all exactly 1 select the equal-mass kernels (Section 3.2: equal-mass fields need
no mass per lens).  Such a field must behave bit for bit like the same lenses given without masses,
whether the masses come from the host or the device; one mass other than 1 keeps the weighted
kernels; and a unit-mass partition next to weighted ones still gives the whole weighted field's map."""
import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import all_rays, dev, rs, shoot_gpu, trace_gpu

pytestmark = pytest.mark.gpu


def _field_spec(masses, seed=12, n=900):
    base = ri.disc_field("um", n, 0.45, 0.0, 0.35, 512, 64, seed=seed, mass="equal")
    return ri.Field("um", base.lens_xy, masses, base.kappa_c, base.gamma, base.grid, base.window)


def test_unit_masses_take_the_equal_mass_kernels():
    m = rs()
    plain = _field_spec(None)
    ones = _field_spec(np.ones(plain.n_lens, np.float32))
    one_off = np.ones(plain.n_lens, np.float32)
    one_off[417] = 0.5
    weighted = _field_spec(one_off)
    for spec, want in ((plain, 0), (ones, 0), (weighted, 1)):
        f = m.Field.from_spec(spec)
        try:
            assert f.info() == (plain.n_lens, want)
        finally:
            f.close()
    # device inputs: the same test as a reduction on the device
    xy = torch.from_numpy(plain.lens_xy).to(dev())
    for masses, want in ((np.ones(plain.n_lens, np.float32), 0), (one_off, 1)):
        f = m.Field(xy, torch.from_numpy(masses).to(dev()), plain.kappa_c, plain.gamma)
        try:
            assert f.info() == (plain.n_lens, want)
            assert f.status() == m.RS_OK  # the status word used as the flag was cleared
        finally:
            f.close()
    # maps, out-of-window counts and float32 traces equal those of the mass-free field bit for bit
    ref, oref = shoot_gpu(plain)
    got, o = shoot_gpu(ones)
    assert np.array_equal(got, ref) and o == oref
    ij = all_rays(plain.grid, rows=(200, 203))
    y0, e0 = trace_gpu(plain, ij)
    y1, e1 = trace_gpu(ones, ij)
    assert np.array_equal(y0, y1) and np.array_equal(e0, e1)
    # and the oracle's map (certified binning)
    oc, oo = oracle.shoot_field(ones)
    assert np.array_equal(got, oc) and o == oo


def test_unit_partition_next_to_weighted_partitions():
    """Partition 0 has masses all 1, partition 1 Salpeter masses: every partition runs the weighted
    kernels and the map equals one pass over the whole weighted field, bit for bit."""
    m = rs()
    sal = ri.disc_field("ump", 1024, 0.5, 0.05, 0.25, 640, 80, seed=23, mass="salpeter")
    masses = sal.masses.copy()
    masses[:512] = 1.0
    spec = ri.Field("ump", sal.lens_xy, masses, sal.kappa_c, sal.gamma, sal.grid, sal.window)
    ref, oref = shoot_gpu(spec)
    parts = [m.Field(spec.lens_xy[a:b], masses[a:b], spec.kappa_c, spec.gamma) for a, b in ((0, 512), (512, 1024))]
    try:
        assert [p.info()[1] for p in parts] == [0, 1]
        g, w = spec.grid, spec.window
        c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot_staged([p.handle for p in parts], g, 0, int(g.n[1]), w, c, o)
        torch.cuda.synchronize()
        assert all(p.status() == m.RS_OK for p in parts)
        assert np.array_equal(c.cpu().numpy().view(np.uint32), ref) and int(o.item()) == oref
        # a partition created without masses cannot join partitions that store them
        bare = m.Field(spec.lens_xy[512:], None, spec.kappa_c, spec.gamma)
        try:
            with pytest.raises(m.RSError) as ei:
                m.rs_shoot_staged([parts[0].handle, bare.handle], g, 0, int(g.n[1]), w, c, o)
            assert ei.value.code == m.RS_EINVAL
        finally:
            bare.close()
    finally:
        for p in parts:
            p.close()
    oc, oo = oracle.shoot_field(spec)
    assert np.array_equal(ref, oc) and oref == oo


def test_streamed_unit_masses_equal_mass_free():
    m = rs()
    plain = _field_spec(None, seed=5, n=2500)
    ones = _field_spec(np.ones(plain.n_lens, np.float32), seed=5, n=2500)
    outs = []
    for spec in (plain, ones):
        g, w = spec.grid, spec.window
        c = torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev())
        o = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot_streamed(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, 1024, g, 0, int(g.n[1]), w, c, o)
        outs.append((c.cpu().numpy().view(np.uint32), int(o.item())))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    ref, oref = shoot_gpu(plain)
    assert np.array_equal(outs[1][0], ref) and outs[1][1] == oref
