"""Moving lenses (Section 4): maps of a field whose stars move, one per time step, against the
oracle's maps of the moved lens positions; in-place time steps, batches of moving fields replayed
after each step, and the translation covariance of a moving lens on the device."""
import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import dev, rs

pytestmark = pytest.mark.gpu


def _counts(field, grid, window):
    c = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev())
    o = torch.zeros(1, dtype=torch.int64, device=dev())
    field.shoot(grid, window, c, o)
    torch.cuda.synchronize()
    assert field.status() == rs().RS_OK
    return c.cpu().numpy().view(np.uint32), int(o.item())


def _oracle_at(spec, vel, t, grid=None, window=None):
    g, w = grid or spec.grid, window or spec.window
    xy = oracle.lens_positions(spec.lens_xy, vel, t)
    return oracle.shoot(xy, spec.masses, spec.kappa_c, spec.gamma, g.origin, g.spacing, g.n, w.lo, w.hi, w.npix)


@pytest.mark.parametrize("mass", ["equal", "salpeter"])
def test_time_steps_match_oracle(mass):
    m = rs()
    spec = ri.disc_field("mv", 150, 0.5, 0.05, 0.2, 512, 128, seed=12, mass=mass)
    vel = ri.lens_velocities(spec.n_lens, 0.5, seed=12)
    f = m.Field(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, velocities=vel)
    try:
        first = None
        for t in (0.0, 0.7, -3.2, 5.0, 0.7):
            f.set_time(t)
            assert f.time == t
            got, oow = _counts(f, spec.grid, spec.window)
            ref, oref = _oracle_at(spec, vel, t)
            assert np.array_equal(got, ref) and oow == oref, t
            if t == 0.7:
                if first is None:
                    first = got
                else:
                    assert np.array_equal(first, got)          # stepping back reproduces the map
        sf = m.Field.from_spec(spec)
        try:
            static, _ = _counts(sf, spec.grid, spec.window)
        finally:
            sf.close()
        f.set_time(0.0)
        assert np.array_equal(_counts(f, spec.grid, spec.window)[0], static)
    finally:
        f.close()


def test_batch_of_moving_fields_replayed_after_time_steps():
    m = rs()
    spec = ri.disc_field("mvb", 120, 0.4, 0.0, 0.3, 384, 96, seed=5, mass="equal")
    vel = ri.lens_velocities(spec.n_lens, 0.3, seed=5)
    frames = [m.Field(spec.lens_xy, None, spec.kappa_c, spec.gamma, velocities=vel) for _ in range(4)]
    try:
        b = m.Batch(frames, [spec.grid] * 4, [spec.window] * 4)
        for step in range(2):
            times = [0.5 * (4 * step + k) for k in range(4)]
            for fr, t in zip(frames, times):
                fr.set_time(t)
            b.launch()
            torch.cuda.synchronize()
            for k, t in enumerate(times):
                ref, oref = _oracle_at(spec, vel, t)
                assert np.array_equal(b.counts[k].cpu().numpy().view(np.uint32), ref), (step, k)
                assert int(b.out_of_window[k].item()) == oref
        b.close()
    finally:
        for fr in frames:
            fr.close()


def test_moving_lens_translates_map_on_device():
    """A single lens moved by (16, -32) pixels moves its map by exactly that (no shear, no kappa_c)."""
    m = rs()
    pix = 1.0 / 32
    g = ri.RayGrid(origin=(-8.0 + pix / 8, -8.0 + pix / 8), spacing=(pix / 4, pix / 4), n=(2048, 2048))
    w = ri.Window(lo=(-1.5, -1.5), hi=(1.5, 1.5), npix=(96, 96))
    f = m.Field(np.array([[0.1875, -0.3125]], np.float32), None, 0.0, 0.0,
                velocities=np.array([[0.25, -0.5]], np.float32))
    try:
        m0, _ = _counts(f, g, w)
        f.set_time(2.0)
        m1, _ = _counts(f, g, w)
    finally:
        f.close()
    assert m0[40:88, 8:72].sum() > 0 and np.array_equal(m0[40:88, 8:72], m1[8:56, 24:88])


def test_set_time_validation():
    m = rs()
    static = m.Field(np.zeros((3, 2), np.float32))
    moving = m.Field(np.ones((3, 2), np.float32), velocities=np.full((3, 2), 2.0, np.float32))
    try:
        for bad in [lambda: static.set_time(1.0), lambda: moving.set_time(float("inf")),
                    lambda: moving.set_time(1e9)]:
            with pytest.raises(m.RSError) as ei:
                bad()
            assert ei.value.code == m.RS_EINVAL
        moving.set_time(-4.0)
        assert moving.time == -4.0
    finally:
        static.close()
        moving.close()
