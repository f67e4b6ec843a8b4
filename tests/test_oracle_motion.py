"""Pins for the oracle's moving lenses (Section 4: stars move between the maps of a time series).

Independent facts: at t = 0 or with zero velocity nothing moves; dyadic positions, velocities and
times move exactly; and a point lens with no shear or smooth convergence (y = x - alpha(x - x_L))
that moves by a whole number of pixels (a multiple of the ray spacing) translates its map by
exactly that many pixels, away from the edges of the ray grid.
"""
import os

import numpy as np
import pytest

import oracle
import rs_inputs as ri


def test_rest_and_still():
    rng = np.random.default_rng(1)
    xy = rng.normal(size=(50, 2)).astype(np.float32)
    v = rng.normal(size=(50, 2)).astype(np.float32)
    assert np.array_equal(oracle.lens_positions(xy, v, 0.0), xy)
    assert np.array_equal(oracle.lens_positions(xy, np.zeros_like(v), 123.4), xy)


def test_dyadic_motion_exact():
    xy = np.array([[1.5, -2.25], [0.0, 8.0]], np.float32)
    v = np.array([[0.25, -0.5], [-3.0, 0.125]], np.float32)
    assert np.array_equal(oracle.lens_positions(xy, v, 4.0), np.array([[2.5, -4.25], [-12.0, 8.5]], np.float32))
    assert np.array_equal(oracle.lens_positions(xy, v, -2.0), np.array([[1.0, -1.25], [6.0, 7.75]], np.float32))


def _moving_lens_maps():
    pix = 1.0 / 32
    g = ri.RayGrid(origin=(-8.0 + pix / 8, -8.0 + pix / 8), spacing=(pix / 4, pix / 4), n=(512 * 4, 512 * 4))
    w = ri.Window(lo=(-1.5, -1.5), hi=(1.5, 1.5), npix=(96, 96))
    x0 = np.array([[0.1875, -0.3125]], np.float32)
    v = np.array([[0.25, -0.5]], np.float32)            # t = 2: moves by (0.5, -1.0) = (16, -32) pixels
    maps = []
    for t in (0.0, 2.0):
        xt = oracle.lens_positions(x0, v, t)
        c, _ = oracle.shoot(xt, None, 0.0, 0.0, g.origin, g.spacing, g.n, w.lo, w.hi, w.npix)
        maps.append(c)
    return maps


def test_moving_lens_translates_map():
    m0, m1 = _moving_lens_maps()
    # pixel (i, j) of the t = 0 map is pixel (i + 16, j - 32) of the t = 2 map
    a = m0[40:88, 8:72]
    b = m1[8:56, 24:88]
    assert a.sum() > 0 and np.array_equal(a, b)
    assert not np.array_equal(m0, m1)


MUTATIONS = [
    ("velocity sign", "(double)xy[i] + (double)vel[i] * t", "(double)xy[i] - (double)vel[i] * t"),
    ("velocity axis", "(double)xy[i] + (double)vel[i] * t", "(double)xy[i] + (double)vel[i ^ 1] * t"),
    ("time ignored", "(double)xy[i] + (double)vel[i] * t", "(double)xy[i] + (double)vel[i]"),
]


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_motion_pins_catch_mutation(name, orig, mut, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    assert src.count(orig) == 1
    bad = tmp_path / "mut.c"
    bad.write_text(src.replace(orig, mut))
    lib = oracle.compile_source(str(bad), str(tmp_path / "libmut.so"))
    failed = 0
    with oracle.using_library(lib):
        for pin in (test_rest_and_still, test_dyadic_motion_exact, test_moving_lens_translates_map):
            try:
                pin()
            except AssertionError:
                failed += 1
    assert failed, name
