"""Python binding of librs.so, the GB300 inverse ray-shooting library.

Thin argument marshalling over the C ABI declared in ``include/rs.h``: the
functions below carry the C names (``rs_create_field``, ``rs_shoot``, ...)
and take torch CUDA tensors for device buffers.  Every step of the method runs
in the library's CUDA kernels; there is no CPU fallback, and importing this
package fails if ``librs.so`` is missing (build it with ``build.build()`` or
``__graft_entry__.build()``).

Method (Thompson, Fluke, Barnes & Barsdell 2009): direct many-Schwarzschild
deflection (Eq. 2) for every ray of a regular image-plane grid, the
macro-model lens equation with smooth convergence and shear (Eq. 6), binning
into source-plane counts and mu = N / N_av (Eq. 4).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

__all__ = [
    "RS_OK", "RS_EINVAL", "RS_ENOMEM", "RS_ECUDA", "RS_EOVERFLOW", "RS_ETIMEOUT", "RS_PROFILE_GAUSSIAN",
    "RS_PROFILE_DISC", "RSError", "RayGrid", "Window", "Track", "Field", "Batch", "LightCurvePlan", "load",
    "lib_path", "magnification", "light_curves", "zoom_grid", "zoom_window", "EXPORTED_SYMBOLS",
    "rs_create_field", "rs_destroy_field", "rs_field_info", "rs_shoot", "rs_shoot_rows", "rs_trace",
    "rs_magnification", "rs_batch_create", "rs_batch_launch", "rs_batch_destroy", "rs_shoot_batch",
    "rs_field_status", "rs_last_error", "rs_version", "rs_set_launch_config", "rs_get_launch_config",
    "rs_launch_configs", "rs_trace_certified", "rs_set_certified_binning", "rs_get_certified_binning",
    "rs_selftest_bounded_wait", "rs_shoot_rows_noalloc", "rs_light_curves", "rs_shoot_culled",
    "rs_create_moving_field", "rs_field_set_time", "rs_field_time", "rs_shoot_staged", "rs_shoot_streamed",
    "rs_set_staged_state_budget", "rs_set_alloc_failure", "rs_light_curve_plan_create", "rs_light_curve_plan_samples",
    "rs_light_curve_plan_launch", "rs_light_curve_plan_destroy", "rs_create_field_view", "rs_device_code_version", "rs_launch_occupancy",
    "rs_partition_buffer_bytes", "rs_partition_pass", "rs_partition_recheck", "rs_batch_create_shaped",
]

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_EOVERFLOW, RS_ETIMEOUT = 0, 1, 2, 3, 4, 5
_NAMES = {0: "RS_OK", 1: "RS_EINVAL", 2: "RS_ENOMEM", 3: "RS_ECUDA", 4: "RS_EOVERFLOW", 5: "RS_ETIMEOUT"}

EXPORTED_SYMBOLS = (
    "rs_create_field", "rs_destroy_field", "rs_field_info", "rs_shoot", "rs_shoot_rows", "rs_trace",
    "rs_magnification", "rs_batch_create", "rs_batch_launch", "rs_batch_destroy", "rs_shoot_batch",
    "rs_field_status", "rs_last_error", "rs_version", "rs_set_launch_config", "rs_get_launch_config",
    "rs_launch_configs", "rs_trace_certified", "rs_set_certified_binning", "rs_get_certified_binning",
    "rs_selftest_bounded_wait", "rs_shoot_rows_noalloc", "rs_light_curves", "rs_shoot_culled",
    "rs_create_moving_field", "rs_field_set_time", "rs_field_time", "rs_shoot_staged", "rs_shoot_streamed",
    "rs_set_staged_state_budget", "rs_set_alloc_failure",
    "rs_light_curve_plan_create", "rs_light_curve_plan_samples", "rs_light_curve_plan_launch",
    "rs_light_curve_plan_destroy", "rs_create_field_view", "rs_device_code_version", "rs_launch_occupancy",
    "rs_partition_buffer_bytes", "rs_partition_pass", "rs_partition_recheck", "rs_batch_create_shaped",
)


class RSError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_NAMES.get(code, code)}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 2), ("spacing", ctypes.c_double * 2), ("n", ctypes.c_int64 * 2)]


class _Window(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2), ("npix", ctypes.c_int32 * 2)]


class _Track(ctypes.Structure):
    _fields_ = [("map", ctypes.c_int32), ("reserved", ctypes.c_int32), ("y0", ctypes.c_double * 2),
                ("step", ctypes.c_double * 2), ("n", ctypes.c_int64)]


RS_PROFILE_GAUSSIAN = 0
RS_PROFILE_DISC = 1


@dataclass
class Track:
    """Straight source track: samples y_k = y0 + k step, k = 0 .. n-1, over map number ``map``."""
    map: int
    y0: tuple
    step: tuple
    n: int


@dataclass
class RayGrid:
    """Ray (i, j) at ((float)fma(i, spacing[0], origin[0]), (float)fma(j, spacing[1], origin[1]))."""
    origin: tuple
    spacing: tuple
    n: tuple

    @property
    def n_rays(self) -> int:
        return int(self.n[0]) * int(self.n[1])


@dataclass
class Window:
    """Half-open source-plane window [lo, hi) per axis with npix pixels per axis."""
    lo: tuple
    hi: tuple
    npix: tuple


def lib_path() -> str:
    return _build.LIB


_lib = None


def load():
    """Load librs.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"librs.so not found at {path}; build it first (paper_0905_2453_gb300.build.build())")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    gp, wp = ctypes.POINTER(_Grid), ctypes.POINTER(_Window)
    sig = {
        "rs_create_field": ([vp, vp, i64, dbl, dbl, i32, vp, ctypes.POINTER(vp)], i32),
        "rs_create_moving_field": ([vp, vp, vp, i64, dbl, dbl, i32, vp, ctypes.POINTER(vp)], i32),
        "rs_field_set_time": ([vp, dbl, vp], i32),
        "rs_field_time": ([vp, ctypes.POINTER(dbl)], i32),
        "rs_destroy_field": ([vp], i32),
        "rs_create_field_view": ([vp, i64, i64, ctypes.POINTER(vp)], i32),
        "rs_field_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i32)], i32),
        "rs_shoot": ([vp, gp, wp, vp, vp, vp], i32),
        "rs_shoot_rows": ([vp, gp, i64, i64, wp, vp, vp, vp], i32),
        "rs_trace": ([vp, gp, vp, i64, vp, vp, vp, vp], i32),
        "rs_trace_certified": ([vp, gp, vp, i64, vp, vp, vp], i32),
        "rs_set_certified_binning": ([i32], i32),
        "rs_get_certified_binning": ([ctypes.POINTER(i32)], i32),
        "rs_selftest_bounded_wait": ([i64, ctypes.POINTER(i32)], i32),
        "rs_shoot_rows_noalloc": ([vp, gp, i64, i64, wp, vp, vp, vp], i32),
        "rs_shoot_culled": ([vp, gp, i64, i64, wp, vp, vp, vp, vp], i32),
        "rs_shoot_staged": ([i32, vp, gp, i64, i64, wp, vp, vp, vp], i32),
        "rs_set_staged_state_budget": ([ctypes.c_uint64], i32),
        "rs_set_alloc_failure": ([i64], i32),
        "rs_shoot_streamed": ([vp, vp, i64, dbl, dbl, i64, gp, i64, i64, wp, vp, vp, vp], i32),
        "rs_magnification": ([vp, gp, wp, vp, vp], i32),
        "rs_light_curves": ([i32, vp, vp, i32, dbl, i32, vp, vp, vp, vp], i32),
        "rs_light_curve_plan_create": ([i32, vp, vp, i32, dbl, i32, vp, ctypes.POINTER(vp)], i32),
        "rs_light_curve_plan_samples": ([vp, ctypes.POINTER(i64)], i32),
        "rs_light_curve_plan_launch": ([vp, vp, vp, vp], i32),
        "rs_light_curve_plan_destroy": ([vp], i32),
        "rs_batch_create": ([i32, vp, vp, vp, vp, vp, ctypes.POINTER(vp)], i32),
        "rs_batch_create_shaped": ([i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(vp)], i32),
        "rs_batch_launch": ([vp, vp], i32),
        "rs_batch_destroy": ([vp], i32),
        "rs_shoot_batch": ([i32, vp, vp, vp, vp, vp, vp], i32),
        "rs_field_status": ([vp, i32, ctypes.POINTER(i32)], i32),
        "rs_last_error": ([], ctypes.c_char_p),
        "rs_version": ([], ctypes.c_char_p),
        "rs_device_code_version": ([ctypes.POINTER(i32)], i32),
        "rs_set_launch_config": ([i32, i32, i32, i32, i32], i32),
        "rs_get_launch_config": ([i32] + [ctypes.POINTER(i32)] * 4, i32),
        "rs_launch_configs": ([ctypes.POINTER(i32), i32, ctypes.POINTER(i32)], i32),
        "rs_launch_occupancy": ([i32, i32, i32, i32, i32, ctypes.POINTER(i32)], i32),
        "rs_partition_buffer_bytes": ([gp, i64, i64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64)], i32),
        "rs_partition_pass": ([vp, i32, gp, i64, i64, wp, vp, i32, i32, vp, vp, vp, vp], i32),
        "rs_partition_recheck": ([vp, i32, gp, i64, i64, wp, vp, vp, i32, i32, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != RS_OK:
        raise RSError(rc, where, load().rs_last_error().decode(errors="replace"))


def _cgrid(g) -> _Grid:
    s = _Grid()
    for k in range(2):
        s.origin[k] = float(g.origin[k])
        s.spacing[k] = float(g.spacing[k])
        s.n[k] = int(g.n[k])
    return s


def _cwin(w) -> _Window:
    s = _Window()
    for k in range(2):
        s.lo[k] = float(w.lo[k])
        s.hi[k] = float(w.hi[k])
        s.npix[k] = int(w.npix[k])
    return s


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


_COUNT_DTYPES = (torch.int32, torch.uint32)
_OOW_DTYPES = (torch.int64, torch.uint64)


def _dptr(t, dtype, name, numel=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype (or tuple of dtypes)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    ok = t.dtype in dtype if isinstance(dtype, tuple) else t.dtype == dtype
    if not ok or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor (got {t.dtype})")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


# ------------------------------------------------------------------------------------------- C names

def rs_version() -> str:
    return load().rs_version().decode()


def rs_device_code_version() -> int:
    """Compute capability the library's device code targets, as the CUDA runtime reports it (103)."""
    v = ctypes.c_int32(0)
    _check(load().rs_device_code_version(ctypes.byref(v)), "rs_device_code_version")
    return int(v.value)


def rs_last_error() -> str:
    return load().rs_last_error().decode(errors="replace")


def _lens_inputs(lens_xy, masses, vel_xy=None):
    """Contiguous float32 copies (device tensors stay on the device) and their pointers."""
    on_dev = isinstance(lens_xy, torch.Tensor) and lens_xy.is_cuda
    if on_dev:
        xy = lens_xy.detach().to(torch.float32).contiguous()
        n = xy.numel() // 2
        m = None if masses is None else masses.detach().to(device=xy.device, dtype=torch.float32).contiguous()
        v = None if vel_xy is None else torch.as_tensor(vel_xy).detach().to(device=xy.device,
                                                                             dtype=torch.float32).contiguous()
        ptr = lambda a: None if a is None else a.data_ptr()  # noqa: E731
        size = lambda a: a.numel()  # noqa: E731
    else:
        import numpy as np

        def host(a):
            return None if a is None else np.ascontiguousarray(
                np.asarray(a.cpu() if isinstance(a, torch.Tensor) else a, dtype=np.float32))
        xy, m, v = host(lens_xy), host(masses), host(vel_xy)
        n = xy.size // 2
        ptr = lambda a: None if a is None or a.size == 0 else a.ctypes.data  # noqa: E731
        size = lambda a: a.size  # noqa: E731
    if m is not None and size(m) != n:
        raise ValueError("masses length differs from lens count")
    if v is not None and size(v) != 2 * n:
        raise ValueError("velocities must have one (v1, v2) pair per lens")
    return on_dev, n, (xy, m, v), (ptr(xy), ptr(m), ptr(v))


def rs_create_field(lens_xy, masses, kappa_c: float, gamma: float, stream=None) -> int:
    """Create a field from lens positions [n, 2] and masses [n] (or None for unit masses).

    Host inputs (numpy arrays / CPU tensors) are copied by the library; CUDA
    tensors are read on the device.  Returns the opaque handle (int).
    """
    lib = load()
    on_dev, n, keep, (pxy, pm, _) = _lens_inputs(lens_xy, masses)
    h = ctypes.c_void_p()
    st = _stream(stream)
    rc = lib.rs_create_field(pxy, pm, n, float(kappa_c), float(gamma), 1 if on_dev else 0, st, ctypes.byref(h))
    _check(rc, "rs_create_field")
    if on_dev:
        torch.cuda.ExternalStream(st).synchronize()  # device inputs may be freed after return
    return h.value


def rs_create_moving_field(lens_xy, vel_xy, masses, kappa_c: float, gamma: float, stream=None) -> int:
    """A field whose lenses move with velocities vel_xy [n, 2]; starts at t = 0 (see rs_field_set_time)."""
    lib = load()
    on_dev, n, keep, (pxy, pm, pv) = _lens_inputs(lens_xy, masses, vel_xy)
    h = ctypes.c_void_p()
    st = _stream(stream)
    _check(lib.rs_create_moving_field(pxy, pv, pm, n, float(kappa_c), float(gamma), 1 if on_dev else 0, st,
                                      ctypes.byref(h)), "rs_create_moving_field")
    return h.value


def rs_field_set_time(handle: int, t: float, stream=None) -> None:
    _check(load().rs_field_set_time(handle, float(t), _stream(stream)), "rs_field_set_time")


def rs_field_time(handle: int) -> float:
    t = ctypes.c_double()
    _check(load().rs_field_time(handle, ctypes.byref(t)), "rs_field_time")
    return float(t.value)


def rs_destroy_field(handle: int) -> None:
    _check(load().rs_destroy_field(handle), "rs_destroy_field")


def rs_create_field_view(handle: int, lens_begin: int, n_lens: int) -> int:
    """A field of lenses [lens_begin, lens_begin + n_lens) of the field `handle` (no copy)."""
    h = ctypes.c_void_p()
    _check(load().rs_create_field_view(handle, int(lens_begin), int(n_lens), ctypes.byref(h)), "rs_create_field_view")
    return h.value


def rs_field_info(handle: int):
    n = ctypes.c_int64()
    hm = ctypes.c_int()
    _check(load().rs_field_info(handle, ctypes.byref(n), ctypes.byref(hm)), "rs_field_info")
    return int(n.value), bool(hm.value)


def rs_shoot(handle: int, grid, window, counts: torch.Tensor, out_of_window: torch.Tensor = None, stream=None):
    """Accumulate the binned counts of every ray of ``grid`` into ``counts`` (uint32 [npix1, npix0])."""
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot(handle, ctypes.byref(g), ctypes.byref(w), pc, po, _stream(stream)), "rs_shoot")


def rs_shoot_rows(handle: int, grid, row_begin: int, row_end: int, window, counts, out_of_window=None, stream=None):
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot_rows(handle, ctypes.byref(g), int(row_begin), int(row_end), ctypes.byref(w), pc, po,
                                _stream(stream)), "rs_shoot_rows")


def rs_shoot_rows_noalloc(handle: int, grid, row_begin: int, row_end: int, window, counts, out_of_window=None,
                          stream=None):
    """rs_shoot_rows with certified binning that allocates no device memory (for callers that
    cannot allocate while they run); at most 2^24 rays per call, see include/rs.h."""
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot_rows_noalloc(handle, ctypes.byref(g), int(row_begin), int(row_end), ctypes.byref(w), pc,
                                        po, _stream(stream)), "rs_shoot_rows_noalloc")


def rs_shoot_culled(handle: int, grid, row_begin: int, row_end: int, window, counts, out_of_window=None,
                    rays_shot=None, stream=None):
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    pr = _dptr(rays_shot, _OOW_DTYPES, "rays_shot", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot_culled(handle, ctypes.byref(g), int(row_begin), int(row_end), ctypes.byref(w), pc, po, pr,
                                  _stream(stream)), "rs_shoot_culled")


def rs_shoot_staged(handles, grid, row_begin: int, row_end: int, window, counts, out_of_window=None, stream=None):
    """Shoot a field given as lens partitions (handles, in lens order; all but the last a multiple of 256)."""
    n = len(handles)
    H = (ctypes.c_void_p * max(1, n))(*handles)
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot_staged(n, H, ctypes.byref(g), int(row_begin), int(row_end), ctypes.byref(w), pc, po,
                                  _stream(stream)), "rs_shoot_staged")


def rs_partition_buffer_bytes(grid, row_begin: int, row_end: int):
    """(state, list, float-float) device buffer bytes of a partition pass over rows [row_begin, row_end)."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    g = _cgrid(grid)
    _check(load().rs_partition_buffer_bytes(ctypes.byref(g), int(row_begin), int(row_end), ctypes.byref(a),
                                            ctypes.byref(b), ctypes.byref(c)), "rs_partition_buffer_bytes")
    return int(a.value), int(b.value), int(c.value)


def _byte_ptr(t, name, nbytes):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    if t.numel() * t.element_size() < nbytes:
        raise ValueError(f"{name} holds {t.numel() * t.element_size()} bytes, needs {nbytes}")
    return t.data_ptr()


def rs_partition_pass(handle, weighted: bool, grid, row_begin: int, row_end: int, window, state, first: bool,
                      last: bool, counts=None, out_of_window=None, lst=None, stream=None):
    """One lens partition's pass over rows [row_begin, row_end): adds its lenses to `state`; the last one maps
    and bins into counts / out_of_window and lists the rays to re-evaluate in `lst` (device byte buffers of
    rs_partition_buffer_bytes' sizes)."""
    sb, lb, _ = rs_partition_buffer_bytes(grid, row_begin, row_end)
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx) if last else None
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1) if last else None
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_partition_pass(handle, int(bool(weighted)), ctypes.byref(g), int(row_begin), int(row_end),
                                    ctypes.byref(w), _byte_ptr(state, "state", sb), int(bool(first)), int(bool(last)),
                                    pc, po, _byte_ptr(lst, "list", lb) if last else None, _stream(stream)),
           "rs_partition_pass")


def rs_partition_recheck(handle, weighted: bool, grid, row_begin: int, row_end: int, window, lst, ff, first: bool,
                         last: bool, counts=None, out_of_window=None, stream=None):
    """One lens partition's float-float share of the listed rays (added to ff); the last call bins them."""
    _, lb, fb = rs_partition_buffer_bytes(grid, row_begin, row_end)
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx) if last else None
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1) if last else None
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_partition_recheck(handle, int(bool(weighted)), ctypes.byref(g), int(row_begin), int(row_end),
                                       ctypes.byref(w), _byte_ptr(lst, "list", lb), _byte_ptr(ff, "ff", fb),
                                       int(bool(first)), int(bool(last)), pc, po, _stream(stream)),
           "rs_partition_recheck")


def rs_shoot_streamed(lens_xy, masses, kappa_c: float, gamma: float, lenses_per_pass: int, grid, row_begin: int,
                      row_end: int, window, counts, out_of_window=None, stream=None):
    """Shoot lenses held in host memory (numpy [n, 2] float32, masses [n] or None), streamed through the
    device lenses_per_pass at a time.  Synchronous."""
    import numpy as np
    xy = np.ascontiguousarray(np.asarray(lens_xy, dtype=np.float32).reshape(-1, 2))
    m = None if masses is None else np.ascontiguousarray(np.asarray(masses, dtype=np.float32).reshape(-1))
    n = xy.shape[0]
    if m is not None and m.size != n:
        raise ValueError("masses length differs from lens count")
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    po = _dptr(out_of_window, _OOW_DTYPES, "out_of_window", 1)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_shoot_streamed(xy.ctypes.data if n else None, None if m is None else m.ctypes.data, n,
                                    float(kappa_c), float(gamma), int(lenses_per_pass), ctypes.byref(g),
                                    int(row_begin), int(row_end), ctypes.byref(w), pc, po, _stream(stream)),
           "rs_shoot_streamed")


def rs_set_alloc_failure(n: int) -> None:
    """Make the n-th following library allocation fail once (n = -1 disarms); failure-detection tests."""
    _check(load().rs_set_alloc_failure(int(n)), "rs_set_alloc_failure")


def rs_set_staged_state_budget(nbytes: int) -> None:
    _check(load().rs_set_staged_state_budget(int(nbytes)), "rs_set_staged_state_budget")


def rs_trace(handle: int, grid, ray_ij: torch.Tensor, y: torch.Tensor, alpha: torch.Tensor = None,
             err: torch.Tensor = None, stream=None):
    """Source positions (float64 [k, 2]) of listed rays (int64 [k, 2]) into ``y`` (and ``alpha``,
    and ``err``: the per-axis band half-width of the float32 result)."""
    k = ray_ij.numel() // 2
    pij = _dptr(ray_ij, torch.int64, "ray_ij")
    py = _dptr(y, torch.float64, "y", 2 * k)
    pa = _dptr(alpha, torch.float64, "alpha", 2 * k)
    pe = _dptr(err, torch.float64, "err", 2 * k)
    g = _cgrid(grid)
    _check(load().rs_trace(handle, ctypes.byref(g), pij, k, py, pa, pe, _stream(stream)), "rs_trace")


def rs_trace_certified(handle: int, grid, ray_ij: torch.Tensor, y: torch.Tensor, alpha: torch.Tensor = None,
                       stream=None):
    """Source positions of listed rays with the float-float deflection sum (certified binning's evaluation)."""
    k = ray_ij.numel() // 2
    pij = _dptr(ray_ij, torch.int64, "ray_ij")
    py = _dptr(y, torch.float64, "y", 2 * k)
    pa = _dptr(alpha, torch.float64, "alpha", 2 * k)
    g = _cgrid(grid)
    _check(load().rs_trace_certified(handle, ctypes.byref(g), pij, k, py, pa, _stream(stream)),
           "rs_trace_certified")


def rs_selftest_bounded_wait(limit_ns: int) -> int:
    """Run the bounded-wait self-test kernel; returns RS_ETIMEOUT when the wait gave up as designed."""
    st = ctypes.c_int()
    _check(load().rs_selftest_bounded_wait(int(limit_ns), ctypes.byref(st)), "rs_selftest_bounded_wait")
    return int(st.value)


def rs_set_certified_binning(enabled: bool) -> None:
    _check(load().rs_set_certified_binning(1 if enabled else 0), "rs_set_certified_binning")


def rs_get_certified_binning() -> bool:
    v = ctypes.c_int()
    _check(load().rs_get_certified_binning(ctypes.byref(v)), "rs_get_certified_binning")
    return bool(v.value)


def rs_magnification(counts: torch.Tensor, grid, window, mu: torch.Tensor, stream=None):
    npx = int(window.npix[0]) * int(window.npix[1])
    pc = _dptr(counts, _COUNT_DTYPES, "counts", npx)
    pm = _dptr(mu, torch.float32, "mu", npx)
    g, w = _cgrid(grid), _cwin(window)
    _check(load().rs_magnification(pc, ctypes.byref(g), ctypes.byref(w), pm, _stream(stream)), "rs_magnification")


def _lc_arrays(maps, windows, tracks):
    n_maps = len(maps)
    if len(windows) != n_maps:
        raise ValueError("maps and windows must have the same length")
    M = (ctypes.c_void_p * max(1, n_maps))(*[_dptr(m, torch.float32, f"maps[{k}]",
                                                     int(windows[k].npix[0]) * int(windows[k].npix[1]))
                                               for k, m in enumerate(maps)])
    W = (_Window * max(1, n_maps))(*[_cwin(w) for w in windows])
    T = (_Track * max(1, len(tracks)))()
    for k, t in enumerate(tracks):
        T[k].map = int(t.map)
        T[k].n = int(t.n)
        for a in range(2):
            T[k].y0[a] = float(t.y0[a])
            T[k].step[a] = float(t.step[a])
    return n_maps, M, W, T


def rs_light_curves(maps, windows, profile: int, s: float, tracks, mu_out: torch.Tensor, dm_out: torch.Tensor = None,
                    stream=None):
    """Light curves of ``tracks`` over ``maps`` (float32 CUDA tensors [npix1, npix0]) into float64 outputs."""
    n_maps, M, W, T = _lc_arrays(maps, windows, tracks)
    total = sum(int(t.n) for t in tracks)
    pm = _dptr(mu_out, torch.float64, "mu_out", total)
    pd = _dptr(dm_out, torch.float64, "dm_out", total)
    _check(load().rs_light_curves(n_maps, M, W, int(profile), float(s), len(tracks), T, pm, pd, _stream(stream)),
           "rs_light_curves")


def rs_light_curve_plan_create(maps, windows, profile: int, s: float, tracks) -> int:
    n_maps, M, W, T = _lc_arrays(maps, windows, tracks)
    p = ctypes.c_void_p()
    _check(load().rs_light_curve_plan_create(n_maps, M, W, int(profile), float(s), len(tracks), T, ctypes.byref(p)),
           "rs_light_curve_plan_create")
    return p.value


def rs_light_curve_plan_samples(plan: int) -> int:
    n = ctypes.c_int64()
    _check(load().rs_light_curve_plan_samples(plan, ctypes.byref(n)), "rs_light_curve_plan_samples")
    return int(n.value)


def rs_light_curve_plan_launch(plan: int, mu_out: torch.Tensor, dm_out: torch.Tensor = None, stream=None):
    n = rs_light_curve_plan_samples(plan)
    pm = _dptr(mu_out, torch.float64, "mu_out", n)
    pd = _dptr(dm_out, torch.float64, "dm_out", n)
    _check(load().rs_light_curve_plan_launch(plan, pm, pd, _stream(stream)), "rs_light_curve_plan_launch")


def rs_light_curve_plan_destroy(plan: int):
    _check(load().rs_light_curve_plan_destroy(plan), "rs_light_curve_plan_destroy")


class LightCurvePlan:
    """Tracks over maps, validated and uploaded once; ``launch`` fills ``mu`` and ``dm`` (float64)."""

    def __init__(self, maps, windows, tracks, profile: int = 0, s: float = 1.0):
        self.maps = list(maps)      # the plan reads these buffers at every launch
        self.handle = rs_light_curve_plan_create(self.maps, windows, profile, s, tracks)
        n = rs_light_curve_plan_samples(self.handle)
        dev = self.maps[0].device if self.maps else torch.device("cuda", torch.cuda.current_device())
        self.mu = torch.empty(n, dtype=torch.float64, device=dev)
        self.dm = torch.empty(n, dtype=torch.float64, device=dev)

    def launch(self, stream=None):
        rs_light_curve_plan_launch(self.handle, self.mu, self.dm, stream)

    def close(self):
        if getattr(self, "handle", None):
            rs_light_curve_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def light_curves(maps, windows, tracks, profile: int = RS_PROFILE_GAUSSIAN, s: float = 1.0, stream=None):
    """Returns (mu, dm) as float64 CUDA tensors with the tracks' samples concatenated in order."""
    total = sum(int(t.n) for t in tracks)
    dev = maps[0].device if maps else torch.device("cuda", torch.cuda.current_device())
    mu = torch.empty(max(total, 0), dtype=torch.float64, device=dev)
    dm = torch.empty_like(mu)
    if total:
        rs_light_curves(maps, windows, profile, s, tracks, mu, dm, stream)
    return mu, dm


def _batch_arrays(handles, grids, windows, counts_list, oow):
    n = len(handles)
    if not (len(grids) == len(windows) == len(counts_list) == n):
        raise ValueError("fields, grids, windows and counts must have the same length")
    H = (ctypes.c_void_p * n)(*handles)
    G = (_Grid * n)(*[_cgrid(g) for g in grids])
    W = (_Window * n)(*[_cwin(w) for w in windows])
    C = (ctypes.c_void_p * n)(*[_dptr(c, _COUNT_DTYPES, f"counts[{k}]",
                                      int(windows[k].npix[0]) * int(windows[k].npix[1]))
                                for k, c in enumerate(counts_list)])
    po = _dptr(oow, _OOW_DTYPES, "out_of_window", n)
    return n, H, G, W, C, po


def rs_batch_create(handles, grids, windows, counts_list, out_of_window=None) -> int:
    n, H, G, W, C, po = _batch_arrays(handles, grids, windows, counts_list, out_of_window)
    b = ctypes.c_void_p()
    _check(load().rs_batch_create(n, H, G, W, C, po, ctypes.byref(b)), "rs_batch_create")
    return b.value


def rs_batch_create_shaped(handles, grids, windows, counts_list, out_of_window=None, shapes=None) -> int:
    """rs_batch_create with a launch shape (block, rays per thread, lens tile, min_ctas) per field (None: the
    defaults)."""
    n, H, G, W, C, po = _batch_arrays(handles, grids, windows, counts_list, out_of_window)
    S = None
    if shapes is not None:
        if len(shapes) != n:
            raise ValueError("one launch shape per field")
        S = (ctypes.c_int * (4 * n))(*[int(v) for sh in shapes for v in sh])
    b = ctypes.c_void_p()
    _check(load().rs_batch_create_shaped(n, H, G, W, C, po, S, ctypes.byref(b)), "rs_batch_create_shaped")
    return b.value


def rs_batch_launch(batch: int, stream=None):
    _check(load().rs_batch_launch(batch, _stream(stream)), "rs_batch_launch")


def rs_batch_destroy(batch: int):
    _check(load().rs_batch_destroy(batch), "rs_batch_destroy")


def rs_shoot_batch(handles, grids, windows, counts_list, out_of_window=None, stream=None):
    n, H, G, W, C, po = _batch_arrays(handles, grids, windows, counts_list, out_of_window)
    _check(load().rs_shoot_batch(n, H, G, W, C, po, _stream(stream)), "rs_shoot_batch")


def rs_field_status(handle: int, clear: bool = False) -> int:
    st = ctypes.c_int()
    _check(load().rs_field_status(handle, 1 if clear else 0, ctypes.byref(st)), "rs_field_status")
    return int(st.value)


def rs_set_launch_config(has_masses: bool, block: int, rays_per_thread: int, lens_tile: int = 256,
                         min_ctas: int = 2) -> None:
    _check(load().rs_set_launch_config(1 if has_masses else 0, int(block), int(rays_per_thread), int(lens_tile),
                                       int(min_ctas)), "rs_set_launch_config")


def rs_get_launch_config(has_masses: bool):
    """(block, rays_per_thread, lens_tile, min_ctas) of the mass mode's current launch shape."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().rs_get_launch_config(1 if has_masses else 0, *[ctypes.byref(x) for x in v]),
           "rs_get_launch_config")
    return tuple(int(x.value) for x in v)


def rs_launch_configs():
    """The compiled launch shapes as (block, rays_per_thread, lens_tile, min_ctas) quadruples."""
    cnt = ctypes.c_int()
    buf = (ctypes.c_int * 128)()
    _check(load().rs_launch_configs(buf, 32, ctypes.byref(cnt)), "rs_launch_configs")
    return [tuple(buf[4 * i + j] for j in range(4)) for i in range(min(cnt.value, 32))]


def rs_launch_occupancy(has_masses: bool, block: int, rays_per_thread: int, lens_tile: int = 256,
                        min_ctas: int = 2) -> int:
    """Resident CTAs per SM of a launch shape's shoot kernel on the current device."""
    v = ctypes.c_int(0)
    _check(load().rs_launch_occupancy(int(bool(has_masses)), int(block), int(rays_per_thread), int(lens_tile),
                                      int(min_ctas), ctypes.byref(v)), "rs_launch_occupancy")
    return int(v.value)


# ------------------------------------------------------------------------------------------- objects

class Field:
    """Owning wrapper of an rs_field handle."""

    def __init__(self, lens_xy, masses=None, kappa_c: float = 0.0, gamma: float = 0.0, stream=None,
                 velocities=None):
        if velocities is None:
            self.handle = rs_create_field(lens_xy, masses, kappa_c, gamma, stream)
        else:
            self.handle = rs_create_moving_field(lens_xy, velocities, masses, kappa_c, gamma, stream)
        self.kappa_c, self.gamma = float(kappa_c), float(gamma)

    def set_time(self, t: float, stream=None):
        """Move the lenses of a moving field to time t (stream-ordered, in place)."""
        rs_field_set_time(self.handle, t, stream)

    @property
    def time(self) -> float:
        return rs_field_time(self.handle)

    @classmethod
    def from_spec(cls, spec, stream=None):
        """From any object with lens_xy, masses, kappa_c and gamma attributes."""
        return cls(spec.lens_xy, spec.masses, spec.kappa_c, spec.gamma, stream)

    def info(self):
        return rs_field_info(self.handle)

    def view(self, lens_begin: int, n_lens: int) -> "Field":
        """The lenses [lens_begin, lens_begin + n_lens) of this field as a field of their own, reading
        this field's device arrays (lens_begin a multiple of 256).  Close views before this field."""
        v = Field.__new__(Field)
        v.handle = rs_create_field_view(self.handle, lens_begin, n_lens)
        v.kappa_c, v.gamma = self.kappa_c, self.gamma
        v._parent = self  # keeps the parent alive while the view is
        return v

    def shoot(self, grid, window, counts=None, out_of_window=None, stream=None, rows=None, culled=False,
              rays_shot=None):
        """Shoot (accumulate) the grid's rays into counts; culled=True skips cells of rays that provably
        miss the window (same results; rays_shot, if given, accumulates the rays actually shot)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if counts is None:
            counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev)
        r0, r1 = (0, int(grid.n[1])) if rows is None else rows
        if culled:
            rs_shoot_culled(self.handle, grid, r0, r1, window, counts, out_of_window, rays_shot, stream)
        elif rows is None:
            rs_shoot(self.handle, grid, window, counts, out_of_window, stream)
        else:
            rs_shoot_rows(self.handle, grid, r0, r1, window, counts, out_of_window, stream)
        return counts

    def zoom(self, grid, window, lo, hi, factor: int, stream=None):
        """Zoom into the source-plane region [lo, hi) of a map made with (grid, window): the map of that
        region at `factor` times the pixel resolution, shot with `factor` times the ray density per axis
        (so N_av is unchanged) and culled to the rays that can reach the region.  Returns
        (counts, fine_grid, fine_window)."""
        g, w = zoom_grid(grid, factor), zoom_window(window, lo, hi, factor)
        return self.shoot(g, w, culled=True, stream=stream), g, w

    def trace(self, grid, ray_ij, with_alpha=False, with_err=False, certified=False, stream=None):
        """Source positions of listed rays: float32 path (default) or float-float (certified=True)."""
        dev = torch.device("cuda", torch.cuda.current_device())
        ij = torch.as_tensor(ray_ij, dtype=torch.int64).reshape(-1, 2).to(dev).contiguous()
        y = torch.empty((ij.shape[0], 2), dtype=torch.float64, device=dev)
        a = torch.empty_like(y) if with_alpha else None
        e = torch.empty_like(y) if (with_err and not certified) else None
        if certified:
            rs_trace_certified(self.handle, grid, ij, y, a, stream)
        else:
            rs_trace(self.handle, grid, ij, y, a, e, stream)
        out = (y,) + ((a,) if with_alpha else ()) + ((e,) if (with_err and not certified) else ())
        return out if len(out) > 1 else y

    def status(self, clear=False) -> int:
        return rs_field_status(self.handle, clear)

    def close(self):
        if getattr(self, "handle", None):
            rs_destroy_field(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zoom_grid(grid, factor: int) -> RayGrid:
    """The ray grid over the same image-plane cells with factor x factor rays per original ray cell
    (cell-centred sub-rays)."""
    f = int(factor)
    if f < 1:
        raise ValueError("factor must be >= 1")
    sp = tuple(float(grid.spacing[k]) / f for k in range(2))
    org = tuple(float(grid.origin[k]) - 0.5 * float(grid.spacing[k]) + 0.5 * sp[k] for k in range(2))
    return RayGrid(org, sp, tuple(int(grid.n[k]) * f for k in range(2)))


def zoom_window(window, lo, hi, factor: int) -> Window:
    """The source-plane window [lo, hi) with pixels `factor` times smaller than the window's."""
    npix = []
    for k in range(2):
        pix = (float(window.hi[k]) - float(window.lo[k])) / int(window.npix[k]) / int(factor)
        npix.append(max(1, int(round((float(hi[k]) - float(lo[k])) / pix))))
    return Window(tuple(float(v) for v in lo), tuple(float(v) for v in hi), tuple(npix))


def magnification(counts, grid, window, stream=None):
    mu = torch.empty(counts.shape, dtype=torch.float32, device=counts.device)
    rs_magnification(counts, grid, window, mu, stream)
    return mu


class Batch:
    """A planned batch of fields (persistent kernel captured in a CUDA graph)."""

    def __init__(self, fields, grids, windows, counts_list=None, out_of_window=None, shapes=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        if counts_list is None:
            counts_list = [torch.zeros((int(w.npix[1]), int(w.npix[0])), dtype=torch.int32, device=dev)
                           for w in windows]
        if out_of_window is None:
            out_of_window = torch.zeros(len(fields), dtype=torch.int64, device=dev)
        self.fields = list(fields)
        self.counts = counts_list
        self.out_of_window = out_of_window
        self.handle = rs_batch_create_shaped([f.handle for f in self.fields], grids, windows, counts_list,
                                             out_of_window, shapes)

    def launch(self, stream=None):
        rs_batch_launch(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            rs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Load eagerly so that a missing library fails at import time, not at first use.
load()
