"""Seeded synthetic lens fields, ray grids and source windows.

This module only *draws inputs*: lens positions and masses, and the plain
parameters (grid origin/spacing/extent, window bounds) of each workload.  It
contains none of the ray-shooting arithmetic, so both the FP64 oracle
(``oracle/``) and the CUDA path (``paper_0905_2453_gb300``) can take their
inputs from here without sharing any of the method.

Workloads follow the shapes of the paper's experiments (Section 3: equal-mass
fields for the timing runs, Section 3.2 for variable masses and the
shear/convergence macro-model of Eq. 6).  The paper uses random rays; the
workloads here shoot a regular, cell-centred image-plane grid instead.

Geometry recipe (the paper gives none):
  * a lens disc of radius R holding N lenses of mean mass <m> has a mean
    surface density kappa_* = N <m> / R^2 in the units of Eq. 2 (unit mass has
    unit Einstein radius), so R = sqrt(N <m> / kappa_*);
  * the disc covers the square shooting region [-L, L]^2 by 1.5x its
    circumradius: L = R / (1.5 sqrt 2);
  * the source window is [-s, s]^2 with s = L / 5 (the ratio of the tiny
    workload: rays over [-10, 10]^2, map over [-2, 2]^2).

Masses: equal (m = 1) or Salpeter, dN/dm ~ m^-2.35 on [0.1, 1], drawn by the
inverse CDF.  Positions: uniform in the disc, r = R sqrt(u1), theta = 2 pi u2,
computed in float64 and rounded to float32 (the lens arrays are float32).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SALPETER_SLOPE = 2.35
SALPETER_MLO = 0.1
SALPETER_MHI = 1.0


def salpeter_mean_mass(slope: float = SALPETER_SLOPE, mlo: float = SALPETER_MLO,
                       mhi: float = SALPETER_MHI) -> float:
    """Analytic mean of dN/dm ~ m^-slope on [mlo, mhi]."""
    a = 1.0 - slope  # exponent of the integrated number
    b = 2.0 - slope  # exponent of the integrated mass
    num = (mhi ** b - mlo ** b) / b
    den = (mhi ** a - mlo ** a) / a
    return num / den


def salpeter_masses(u: np.ndarray, slope: float = SALPETER_SLOPE, mlo: float = SALPETER_MLO,
                    mhi: float = SALPETER_MHI) -> np.ndarray:
    """Inverse-CDF draw of power-law masses from uniforms u in [0, 1)."""
    a = 1.0 - slope
    lo, hi = mlo ** a, mhi ** a
    return (lo + u * (hi - lo)) ** (1.0 / a)


@dataclasses.dataclass
class RayGrid:
    """Regular image-plane grid: ray (i, j) sits at origin + (i, j) * spacing.

    ``n = (n0, n1)``: n0 rays along x1 (fastest), n1 along x2.
    """
    origin: tuple
    spacing: tuple
    n: tuple

    @property
    def n_rays(self) -> int:
        return int(self.n[0]) * int(self.n[1])


@dataclasses.dataclass
class Window:
    """Source-plane pixel window: half-open [lo, hi) per axis, npix pixels per axis."""
    lo: tuple
    hi: tuple
    npix: tuple

    @property
    def n_pix(self) -> int:
        return int(self.npix[0]) * int(self.npix[1])


@dataclasses.dataclass
class Field:
    """One lens realisation plus its macro-model and the grid/window it is shot on."""
    name: str
    lens_xy: np.ndarray            # float32 [n, 2]
    masses: Optional[np.ndarray]   # float32 [n] or None (all masses 1)
    kappa_c: float
    gamma: float
    grid: RayGrid
    window: Window
    kappa_star: float = 0.0
    seed: int = 0

    @property
    def n_lens(self) -> int:
        return int(self.lens_xy.shape[0])

    @property
    def interactions(self) -> int:
        return self.n_lens * self.grid.n_rays


def cell_centred_grid(lo: float, hi: float, n: int) -> RayGrid:
    """n x n cell-centred rays over [lo, hi]^2 (first ray half a cell from the edge)."""
    d = (hi - lo) / n
    o = lo + 0.5 * d
    return RayGrid(origin=(o, o), spacing=(d, d), n=(n, n))


def square_window(s: float, npix: int) -> Window:
    return Window(lo=(-s, -s), hi=(s, s), npix=(npix, npix))


def disc_lenses(n: int, radius: float, seed: int, mass: str = "equal",
                store_unit_masses: bool = False):
    """n lenses uniform in a disc of the given radius; float32 xy and masses.

    mass = "equal" (m = 1: masses None unless store_unit_masses) or "salpeter".
    """
    rng = np.random.default_rng(seed)
    u1 = rng.random(n)
    u2 = rng.random(n)
    r = radius * np.sqrt(u1)
    th = 2.0 * math.pi * u2
    xy = np.empty((n, 2), dtype=np.float32)
    xy[:, 0] = (r * np.cos(th)).astype(np.float32)
    xy[:, 1] = (r * np.sin(th)).astype(np.float32)
    if mass == "salpeter":
        m = salpeter_masses(rng.random(n)).astype(np.float32)
    elif mass == "equal":
        m = np.ones(n, dtype=np.float32) if store_unit_masses else None
    else:
        raise ValueError(f"unknown mass law {mass!r}")
    return xy, m


def disc_geometry(n_lens: int, kappa_star: float, mean_mass: float):
    """(R, L, s) of the geometry recipe in the module docstring."""
    R = math.sqrt(n_lens * mean_mass / kappa_star)
    L = R / (1.5 * math.sqrt(2.0))
    s = L / 5.0
    return R, L, s


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def tiny_field(seed: int = 0) -> Field:
    """100 equal-mass lenses in a disc of radius 12; kappa_c = gamma = 0; 1000^2 rays
    over [-10, 10]^2; 256^2 map over [-2, 2]^2 (the 1e8-interaction case)."""
    xy, m = disc_lenses(100, 12.0, seed, "equal")
    return Field("tiny-N100-1000sq", xy, m, 0.0, 0.0, cell_centred_grid(-10.0, 10.0, 1000),
                 square_window(2.0, 256), kappa_star=100 / 144.0, seed=seed)


def disc_field(name: str, n_lens: int, kappa_star: float, kappa_c: float, gamma: float,
               n_rays_side: int, npix: int, seed: int = 0, mass: str = "equal",
               store_unit_masses: bool = False) -> Field:
    mean_m = salpeter_mean_mass() if mass == "salpeter" else 1.0
    R, L, s = disc_geometry(n_lens, kappa_star, mean_m)
    xy, m = disc_lenses(n_lens, R, seed, mass, store_unit_masses)
    return Field(name, xy, m, kappa_c, gamma, cell_centred_grid(-L, L, n_rays_side),
                 square_window(s, npix), kappa_star=kappa_star, seed=seed)


def n1e4_field(seed: int = 0, n_rays_side: int = 4096, npix: int = 1024) -> Field:
    """1e4 equal-mass lenses, kappa_* = 0.45, kappa_c = 0, gamma = 0.4; 4096^2 rays; 1024^2 map."""
    return disc_field(f"N1e4-k0.45-g0.4-{n_rays_side}sq", 10_000, 0.45, 0.0, 0.4, n_rays_side, npix, seed)


def n1e6_salpeter_field(seed: int = 0, n_rays_side: int = 16384, npix: int = 2048) -> Field:
    """1e6 Salpeter lenses, kappa_* = 0.6, kappa_c = 0.1, gamma = 0.3; 16384^2 rays; 2048^2 map."""
    return disc_field(f"N1e6-salpeter-k0.6-kc0.1-g0.3-{n_rays_side}sq", 1_000_000, 0.6, 0.1, 0.3,
                      n_rays_side, npix, seed, mass="salpeter")


def n1e8_field(seed: int = 0, n_rays_side: int = 8192, npix: int = 4096, n_lens: int = 100_000_000) -> Field:
    """1e8 unit-mass lenses with stored float32 masses, kappa_* = 0.5, gamma = 0.5; 8192^2 rays; 4096^2 map."""
    return disc_field(f"N{n_lens:.0e}-k0.5-g0.5-{n_rays_side}sq", n_lens, 0.5, 0.0, 0.5, n_rays_side,
                      npix, seed, mass="equal", store_unit_masses=True)


def batch_fields(n_fields: int = 64, base_seed: int = 1000, ray_scale: float = 1.0) -> list:
    """Independent Salpeter realisations with uneven sizes (field k uses seed base_seed + k).

    N* = round(10^U(2, 5)), kappa_* ~ U(0.1, 0.8), kappa_c = 0, gamma ~ U(0, 0.6),
    ray side ~ U{1024, 1280, ..., 4096}, map side ~ U{512, 640, ..., 1024}.
    ``ray_scale`` < 1 shrinks every ray side (for quick tests), keeping multiples of 16.
    """
    out = []
    for k in range(n_fields):
        seed = base_seed + k
        rng = np.random.default_rng(seed)
        n_lens = int(round(10.0 ** rng.uniform(2.0, 5.0)))
        kstar = float(rng.uniform(0.1, 0.8))
        gamma = float(rng.uniform(0.0, 0.6))
        side = int(rng.choice(np.arange(1024, 4096 + 1, 256)))
        npix = int(rng.choice(np.arange(512, 1024 + 1, 128)))
        if ray_scale != 1.0:
            side = max(16, int(side * ray_scale) // 16 * 16)
            npix = max(16, int(npix * ray_scale) // 16 * 16)
        # positions/masses from a stream independent of the parameter draws
        f = disc_field(f"batch{k}", n_lens, kstar, 0.0, gamma, side, npix, seed=[seed, 1],
                       mass="salpeter")
        f.seed = seed
        out.append(f)
    return out


def sample_rays(grid: RayGrid, k: int, seed: int) -> np.ndarray:
    """k distinct-ish seeded ray indices (i, j) as int64 [k, 2]."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, grid.n[0], size=k, dtype=np.int64)
    j = rng.integers(0, grid.n[1], size=k, dtype=np.int64)
    return np.stack([i, j], axis=1)


# Light-curve inputs ------------------------------------------------------------------------------

@dataclasses.dataclass
class Track:
    """Straight source track: samples y_k = y0 + k step (k = 0 .. n-1) over map number ``map``."""
    map: int
    y0: tuple
    step: tuple
    n: int


def caustic_map(npix: tuple, seed: int, n_caustics: int = 12) -> np.ndarray:
    """A synthetic float32 magnification map [npix1, npix0] with the structure of a microlensing map:
    a lognormal background around mu ~ 1 and fold caustics, closed curves (here circles of random
    centre and radius) outside of which mu rises as A / sqrt(distance) within a few pixels (the
    fold's inverse-square-root law), up to a few hundred."""
    rng = np.random.default_rng(seed)
    n0, n1 = int(npix[0]), int(npix[1])
    mu = rng.lognormal(0.0, 0.25, size=(n1, n0))
    for _ in range(n_caustics):
        cx, cy = rng.uniform(0, n0), rng.uniform(0, n1)
        r = rng.uniform(0.05, 0.4) * min(n0, n1)
        amp = rng.uniform(1.0, 4.0)
        # only the pixels within the ring's bounding box can lie within 15 pixels outside it
        i0, i1 = max(0, int(cx - r - 16)), min(n0, int(cx + r + 17))
        j0, j1 = max(0, int(cy - r - 16)), min(n1, int(cy + r + 17))
        ii = np.arange(i0, i1, dtype=np.float64)[None, :]
        jj = np.arange(j0, j1, dtype=np.float64)[:, None]
        d = np.hypot(ii - cx, jj - cy) - r          # > 0 outside the curve
        out = (d > 0) & (d < 15)
        sub = mu[j0:j1, i0:i1]
        sub[out] += amp / np.sqrt(np.maximum(d[out], 1e-3))
    return np.minimum(mu, 500.0).astype(np.float32)


def random_tracks(windows: list, n_per_map: int, n_samples: int, step_pix: float, seed: int,
                  margin_pix: float = 0.0) -> list:
    """Tracks with uniformly random start points inside each window (shrunk by margin_pix) and
    uniformly random directions, sample spacing step_pix pixels of axis 0."""
    rng = np.random.default_rng(seed)
    out = []
    for m, w in enumerate(windows):
        pix0 = (w.hi[0] - w.lo[0]) / w.npix[0]
        pix1 = (w.hi[1] - w.lo[1]) / w.npix[1]
        for _ in range(n_per_map):
            y0 = (rng.uniform(w.lo[0] + margin_pix * pix0, w.hi[0] - margin_pix * pix0),
                  rng.uniform(w.lo[1] + margin_pix * pix1, w.hi[1] - margin_pix * pix1))
            th = rng.uniform(0.0, 2.0 * np.pi)
            step = (step_pix * pix0 * np.cos(th), step_pix * pix0 * np.sin(th))
            out.append(Track(m, (float(y0[0]), float(y0[1])), (float(step[0]), float(step[1])), int(n_samples)))
    return out


def light_curve_workload(n_maps: int = 64, tracks_per_map: int = 16, n_samples: int = 2048, base_seed: int = 3000):
    """Light curves over many maps: n_maps synthetic caustic maps with the batch's map sides
    (U{512, 640, ..., 1024} pixels) over the window [-1, 1]^2, tracks_per_map random tracks of
    n_samples samples spaced 0.25 pixel (of a 1024-pixel map) each, and a Gaussian source of
    standard deviation 2 pixels of a 1024-pixel map (1 to 2 pixels of the actual maps).
    Returns (maps, windows, tracks, s)."""
    maps, wins = [], []
    for k in range(n_maps):
        rng = np.random.default_rng(base_seed + k)
        npix = int(rng.choice(np.arange(512, 1024 + 1, 128)))
        wins.append(Window(lo=(-1.0, -1.0), hi=(1.0, 1.0), npix=(npix, npix)))
        maps.append(caustic_map((npix, npix), seed=base_seed + 10_000 + k))
    px = 2.0 / 1024
    tracks = []
    rng = np.random.default_rng(base_seed - 1)
    for m in range(n_maps):
        for _ in range(tracks_per_map):
            y0 = (float(rng.uniform(-0.9, 0.9)), float(rng.uniform(-0.9, 0.9)))
            th = float(rng.uniform(0.0, 2.0 * np.pi))
            tracks.append(Track(m, y0, (0.25 * px * math.cos(th), 0.25 * px * math.sin(th)), n_samples))
    return maps, wins, tracks, 2.0 * px


def lens_velocities(n: int, sigma_v: float, seed: int) -> np.ndarray:
    """Isotropic Gaussian lens velocities, float32 [n, 2], standard deviation sigma_v per axis
    (Einstein radii per unit time): the random stellar motions of a time series of maps."""
    rng = np.random.default_rng([seed, 2])
    return (rng.normal(size=(n, 2)) * sigma_v).astype(np.float32)


def disc_lenses_large(n: int, radius: float, seed: int, chunk: int = 1 << 24, threads: int = 16) -> np.ndarray:
    """float32 [n, 2] unit-mass lens positions uniform in a disc, for lens counts beyond what the
    float64 temporaries of disc_lenses allow (billions): chunk k of `chunk` lenses is drawn from its
    own stream (seed [seed, 7, k]) with r = R sqrt(u1), theta = 2 pi u2, several chunks in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    xy = np.empty((n, 2), dtype=np.float32)

    def fill(k):
        a = k * chunk
        m = min(chunk, n - a)
        rng = np.random.default_rng([seed, 7, k])
        u = rng.random((2, m))
        r = radius * np.sqrt(u[0])
        th = 2.0 * math.pi * u[1]
        xy[a:a + m, 0] = r * np.cos(th)
        xy[a:a + m, 1] = r * np.sin(th)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(fill, range((n + chunk - 1) // chunk)))
    return xy
