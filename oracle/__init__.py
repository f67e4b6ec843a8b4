"""FP64 CPU oracle for direct inverse ray-shooting -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never calls it and shares no code with it.

The arithmetic lives in ``rs_oracle.c`` (plain C, double precision, OpenMP
over rays, no fused multiply-add, no fast-math); this module compiles it with
gcc and exposes it through ctypes with numpy arrays.  What each function
computes and which passage of the paper it follows is stated in the C file:
Eq. 2 with the per-lens steps of Appendix A (deflection), Eq. 6 (lens map with
kappa_c and gamma), Eq. 4 (mu = N / N_av), Section 2.1 step 4 (binning),
the light curves of Section 1 (a source profile moved across the map) and the
moving lenses of Section 4 (positions per time step).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(exact rational brute force, zero-lens and linear-map lattice counts, the
single point-lens magnification law, mirror symmetry, conservation,
superposition and the 2-D Gauss law of a uniform disc); ``light_curve`` by
``tests/test_oracle_lightcurve.py`` (constant and linear maps, Gauss circle
lattice counts of the disc profile, the magnitude scale, and a point lens seen
through a Gaussian source against Gauss-Hermite quadrature of the analytic law);
``lens_positions`` by ``tests/test_oracle_motion.py`` (rest and still cases, and
the translation covariance of a moving lens's map).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off (no fast-math) of one C file into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile rs_oracle.c into liboracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        _lib = load_library(_LIB)
        return _lib


def load_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.oracle_trace.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp, vp, vp,
                                 ctypes.c_int64, vp, vp, vp]
    lib.oracle_trace.restype = None
    lib.oracle_shoot_rows.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp, vp,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp, vp, vp, vp, vp]
    lib.oracle_shoot_rows.restype = ctypes.c_int
    lib.oracle_bin_positions.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp]
    lib.oracle_bin_positions.restype = ctypes.c_uint64
    lib.oracle_magnification.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.oracle_magnification.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_num_threads.restype = None
    lib.oracle_light_curve.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp, vp, ctypes.c_int64, vp, vp]
    lib.oracle_light_curve.restype = None
    lib.oracle_lens_positions.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_double, vp]
    lib.oracle_lens_positions.restype = None
    return lib


@contextlib.contextmanager
def using_library(path: str):
    """Route this module's calls to another build of the oracle (used by the mutation tests)."""
    global _lib
    _load()
    old = _lib
    _lib = load_library(path)
    try:
        yield
    finally:
        _lib = old


def _f32(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _d2(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(2))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def trace(lens_xy, masses, kappa_c, gamma, origin, spacing, ray_ij):
    """Source positions y (float64 [k, 2]), deflections alpha and ray positions x of listed rays.

    ray_ij: int64 [k, 2] of (i, j) grid indices.  Returns (y, alpha, x).
    """
    lib = _load()
    xy = _f32(lens_xy).reshape(-1, 2)
    m = _f32(masses)
    if m is not None and m.shape[0] != xy.shape[0]:
        raise ValueError("masses length differs from lens count")
    ij = np.ascontiguousarray(np.asarray(ray_ij, dtype=np.int64).reshape(-1, 2))
    k = ij.shape[0]
    y = np.empty((k, 2), np.float64)
    al = np.empty((k, 2), np.float64)
    x = np.empty((k, 2), np.float64)
    o, s = _d2(origin), _d2(spacing)
    lib.oracle_trace(_ptr(xy), _ptr(m), xy.shape[0], float(kappa_c), float(gamma), _ptr(o), _ptr(s),
                     _ptr(ij), k, _ptr(y), _ptr(al), _ptr(x))
    return y, al, x


def shoot(lens_xy, masses, kappa_c, gamma, origin, spacing, n, lo, hi, npix, rows=None,
          counts=None, out_of_window=0):
    """Count map (uint32 [npix2, npix1]) and out-of-window count of the grid's rays.

    rows = (j_begin, j_end) restricts to a block of grid rows; counts accumulate
    into ``counts`` when given.  Returns (counts, out_of_window).
    """
    lib = _load()
    xy = _f32(lens_xy).reshape(-1, 2)
    m = _f32(masses)
    n0, n1 = int(n[0]), int(n[1])
    jb, je = (0, n1) if rows is None else (int(rows[0]), int(rows[1]))
    npx = np.ascontiguousarray(np.asarray(npix, dtype=np.int32).reshape(2))
    if counts is None:
        counts = np.zeros((int(npx[1]), int(npx[0])), np.uint32)
    assert counts.dtype == np.uint32 and counts.flags.c_contiguous
    assert counts.shape == (int(npx[1]), int(npx[0]))
    oow = np.array([out_of_window], np.uint64)
    o, s, l, h = _d2(origin), _d2(spacing), _d2(lo), _d2(hi)
    rc = lib.oracle_shoot_rows(_ptr(xy), _ptr(m), xy.shape[0], float(kappa_c), float(gamma), _ptr(o),
                               _ptr(s), n0, jb, je, _ptr(l), _ptr(h), _ptr(npx), _ptr(counts), _ptr(oow))
    if rc != 0:
        raise MemoryError("oracle work buffer allocation failed")
    return counts, int(oow[0])


def bin_positions(y, lo, hi, npix, counts=None):
    """Bin source positions (float64 [k, 2]); returns (counts, out_of_window)."""
    lib = _load()
    yy = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(-1, 2))
    npx = np.ascontiguousarray(np.asarray(npix, dtype=np.int32).reshape(2))
    if counts is None:
        counts = np.zeros((int(npx[1]), int(npx[0])), np.uint32)
    l, h = _d2(lo), _d2(hi)
    oow = lib.oracle_bin_positions(_ptr(yy), yy.shape[0], _ptr(l), _ptr(h), _ptr(npx), _ptr(counts))
    return counts, int(oow)


def magnification(counts, spacing, lo, hi, npix):
    """Eq. 4: mu = N / N_av as float64 [npix2, npix1]."""
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    npx = np.ascontiguousarray(np.asarray(npix, dtype=np.int32).reshape(2))
    mu = np.empty(c.shape, np.float64)
    s, l, h = _d2(spacing), _d2(lo), _d2(hi)
    lib.oracle_magnification(_ptr(c), _ptr(s), _ptr(l), _ptr(h), _ptr(npx), _ptr(mu))
    return mu


PROFILE_GAUSSIAN = 0
PROFILE_DISC = 1


def light_curve(mu, lo, hi, profile, s, y0, step, n):
    """Light curve of a magnification map (float64 [npix1, npix0]) along y_k = y0 + k step.

    profile: PROFILE_GAUSSIAN (s = standard deviation, cut at 6 s) or PROFILE_DISC (s = radius).
    Returns (mu_k, dm_k) as float64 arrays of length n.
    """
    lib = _load()
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    npx = np.ascontiguousarray(np.array([m.shape[1], m.shape[0]], dtype=np.int32))
    out = np.empty(int(n), np.float64)
    mag = np.empty(int(n), np.float64)
    l, h, a, b = _d2(lo), _d2(hi), _d2(y0), _d2(step)
    lib.oracle_light_curve(_ptr(m), _ptr(npx), _ptr(l), _ptr(h), int(profile), float(s), _ptr(a), _ptr(b),
                           int(n), _ptr(out), _ptr(mag))
    return out, mag


def lens_positions(lens_xy, vel_xy, t):
    """Positions float32 [n, 2] of lenses moving in straight lines, at time t (see the C file)."""
    lib = _load()
    xy = np.ascontiguousarray(np.asarray(lens_xy, dtype=np.float32).reshape(-1, 2))
    v = np.ascontiguousarray(np.asarray(vel_xy, dtype=np.float32).reshape(-1, 2))
    if xy.shape != v.shape:
        raise ValueError("positions and velocities differ in shape")
    out = np.empty_like(xy)
    lib.oracle_lens_positions(_ptr(xy), _ptr(v), int(xy.shape[0]), float(t), _ptr(out))
    return out


# Convenience wrappers over rs_inputs.Field objects --------------------------------

def trace_field(field, ray_ij):
    g = field.grid
    return trace(field.lens_xy, field.masses, field.kappa_c, field.gamma, g.origin, g.spacing, ray_ij)


def shoot_field(field, rows=None, counts=None, out_of_window=0):
    g, w = field.grid, field.window
    return shoot(field.lens_xy, field.masses, field.kappa_c, field.gamma, g.origin, g.spacing, g.n,
                 w.lo, w.hi, w.npix, rows=rows, counts=counts, out_of_window=out_of_window)
