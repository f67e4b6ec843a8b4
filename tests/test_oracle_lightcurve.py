"""Pins for the oracle's light curves (Section 1: a source profile moved across the magnification
map, the magnification at each point converted to a magnitude change).

Checked against facts independent of the oracle's code: constant and linear maps (exact profile
moments), the Gauss circle lattice counts of the disc profile, the magnitude scale, and the
finite-source magnification of a Schwarzschild lens by Gauss-Hermite quadrature of the analytic
point-source law mu(u) = (u^2+2)/(u sqrt(u^2+4)).
"""
import math

import numpy as np
import pytest

import oracle

G, D = oracle.PROFILE_GAUSSIAN, oracle.PROFILE_DISC


def _centres(lo, hi, npix):
    pix = (hi - lo) / npix
    return lo + (np.arange(npix) + 0.5) * pix


@pytest.mark.parametrize("profile,s", [(G, 0.07), (D, 0.11), (G, 0.3)])
def test_constant_map(profile, s):
    mu = np.full((48, 64), 3.25)
    m, mag = oracle.light_curve(mu, (-1.0, -0.5), (1.0, 1.0), profile, s, (-0.8, -0.3), (0.013, 0.011), 90)
    assert np.all(np.abs(m - 3.25) <= 1e-12)      # rounding of a weighted mean of a few thousand terms
    assert np.allclose(mag, -2.5 * math.log10(3.25), rtol=0, atol=1e-13)


def test_magnitude_scale():
    for v, dm in ((1.0, 0.0), (10.0, -2.5), (100.0, -5.0), (0.1, 2.5)):
        mu = np.full((16, 16), v)
        _, mag = oracle.light_curve(mu, (0.0, 0.0), (1.0, 1.0), G, 0.1, (0.5, 0.5), (0.0, 0.0), 1)
        assert abs(mag[0] - dm) < 1e-12


@pytest.mark.parametrize("profile,s", [(G, 0.047), (D, 0.09)])
def test_linear_map_at_pixel_centres(profile, s):
    """mu = a + b1 x + b2 y: a profile symmetric about a pixel centre returns mu at that centre.
    The Gaussian's 6 sigma cut (5.64 pixels) and the disc radius (1.8 pixels) keep away from lattice
    distances (relative margin 0.7% and 23% in d^2), so rounding cannot break the symmetry of the
    covered pixel set."""
    npx = (80, 50)
    lo, hi = (-2.0, -1.5), (2.0, 1.5)          # pixel 0.05 x 0.06: not square, not dyadic
    cx = _centres(lo[0], hi[0], npx[0])
    cy = _centres(lo[1], hi[1], npx[1])
    a, b1, b2 = 1.7, 0.35, -0.8
    mu = a + b1 * cx[None, :] + b2 * cy[:, None]
    # samples on pixel centres: start at centre (20, 25), step two pixels right and one up
    y0 = (cx[20], cy[25])
    step = (cx[22] - cx[20], cy[26] - cy[25])
    m, _ = oracle.light_curve(mu, lo, hi, profile, s, y0, step, 12)
    k = np.arange(12)
    expect = a + b1 * (y0[0] + k * step[0]) + b2 * (y0[1] + k * step[1])
    assert np.allclose(m, expect, rtol=0, atol=1e-11)
    # off-centre samples are not exact (truncated lattice), only close
    m2, _ = oracle.light_curve(mu, lo, hi, profile, s, (y0[0] + 0.011, y0[1] - 0.007), step, 12)
    assert np.abs(m2 - (expect + b1 * 0.011 - b2 * 0.007)).max() < 0.05


@pytest.mark.parametrize("r,count", [(1, 5), (2, 13), (3, 29), (4, 49), (5, 81)])
def test_disc_lattice_count(r, count):
    """A disc of radius r pixels centred on a pixel centre covers N(r) pixels (Gauss circle numbers)."""
    npx = 32
    lo, hi = 0.0, 8.0                           # pixel 0.25, dyadic: distances exact
    mu = np.ones((npx, npx))
    c = 16
    mu[c, c] = 1.0 + count                      # the mean over the disc is exactly 2 iff it covers N(r) pixels
    y = lo + (c + 0.5) * 0.25
    m, _ = oracle.light_curve(mu, (lo, lo), (hi, hi), D, r * 0.25, (y, y), (0.0, 0.0), 1)
    assert m[0] == 2.0


def _mu_point(u):
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def test_finite_source_point_lens_against_quadrature():
    """A Gaussian source of width 0.2 crossing a unit point lens: pixel-sampled analytic map vs the
    continuous convolution by Gauss-Hermite quadrature (independent), away from the singular centre."""
    npx = 640
    lo, hi = -4.0, 4.0
    c = _centres(lo, hi, npx)
    u = np.hypot(c[None, :], c[:, None])
    mu = _mu_point(u)
    s = 0.2
    y0 = (-2.5, 0.9)
    step = (0.1, 0.0)
    n = 51
    m, mag = oracle.light_curve(mu, (lo, lo), (hi, hi), G, s, y0, step, n)
    z, wz = np.polynomial.hermite_e.hermegauss(40)      # weight exp(-z^2/2)
    wz = wz / wz.sum()
    for k in range(n):
        yx, yy = y0[0] + k * step[0], y0[1] + k * step[1]
        ux = yx + s * z[:, None]
        uy = yy + s * z[None, :]
        ref = (wz[:, None] * wz[None, :] * _mu_point(np.hypot(ux, uy))).sum()
        assert abs(m[k] / ref - 1) < 2e-3, (k, m[k], ref)


# plausible mistakes in the light-curve oracle; each must fail at least one pin above
LC_MUTATIONS = [
    ("pixel corner not centre", "const double cx = lo[0] + ((double)i + 0.5) * pix0;",
     "const double cx = lo[0] + (double)i * pix0;"),
    ("pixel size axis", "const double pix1 = (hi[1] - lo[1]) / (double)npix[1];",
     "const double pix1 = (hi[0] - lo[0]) / (double)npix[0];"),
    ("track step axis", "const double yy = y0[1] + (double)k * step[1];",
     "const double yy = y0[1] + (double)k * step[0];"),
    ("gaussian width", "const double inv2s2 = 1.0 / (2.0 * s * s);", "const double inv2s2 = 1.0 / (s * s * s);"),
    ("disc radius", ": s * s;", ": 2.0 * s * s;"),
    ("unnormalised", "swm / sw : NAN", "swm : NAN"),
    ("transposed map", "mu[(int64_t)j * npix[0] + i]", "mu[(int64_t)i * npix[1] + j]"),
    ("natural log magnitude", "-2.5 * log10(m)", "-2.5 * log(m)"),
]

_LC_PINS = [
    lambda: test_constant_map(G, 0.07),
    lambda: test_constant_map(D, 0.11),
    test_magnitude_scale,
    lambda: test_linear_map_at_pixel_centres(G, 0.047),
    lambda: test_linear_map_at_pixel_centres(D, 0.09),
    lambda: [test_disc_lattice_count(r, c) for r, c in ((1, 5), (2, 13), (3, 29))],
    test_finite_source_point_lens_against_quadrature,
]


@pytest.mark.parametrize("name,orig,mut", LC_MUTATIONS, ids=[m[0] for m in LC_MUTATIONS])
def test_light_curve_pins_catch_mutation(name, orig, mut, tmp_path):
    import os
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    assert src.count(orig) == 1, f"mutation anchor not unique/found: {orig!r}"
    bad = tmp_path / "mut.c"
    bad.write_text(src.replace(orig, mut))
    lib = oracle.compile_source(str(bad), str(tmp_path / "libmut.so"))
    failed = 0
    with oracle.using_library(lib):
        for pin in _LC_PINS:
            try:
                pin()
            except AssertionError:
                failed += 1
    assert failed, f"no pin caught mutation {name!r}"
