"""Host-side checks of the C-ABI library (no GPU needed, no kernel launched).

* librs.so builds for sm_103a and loads;
* it exports every function include/rs.h declares, and the Python binding
  names the same set;
* argument validation rejects bad input with the documented status codes
  before any CUDA call is made.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_0905_2453_gb300 as rs
    return rs


def _declared():
    src = open(os.path.join(ROOT, "include", "rs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:int|const char\*)\s+(rs_\w+)\s*\(", src, flags=re.M))


def test_header_declares_boundary():
    names = _declared()
    for must in ("rs_create_field", "rs_shoot", "rs_magnification", "rs_shoot_batch", "rs_trace"):
        assert must in names


def test_library_exports_every_declared_symbol(rs):
    out = subprocess.run(["nm", "-D", "--defined-only", rs.lib_path()], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\bT\s+(rs_\w+)", out.stdout))
    missing = _declared() - exported
    assert not missing, missing
    assert set(rs.EXPORTED_SYMBOLS) == _declared()
    lib = ctypes.CDLL(rs.lib_path())
    for name in _declared():
        assert hasattr(lib, name)


def test_library_targets_sm103a(rs):
    """The build compiles device code for sm_103a only (the runtime query of a built kernel's target is
    a GPU test: tests/test_gpu_parity.py::test_device_code_targets_sm103a)."""
    from paper_0905_2453_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version(rs):
    assert "sm_103a" in rs.rs_version()


def test_validation_codes(rs):
    lib = rs.load()
    h = ctypes.c_void_p()
    assert lib.rs_create_field(None, None, -1, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    assert "n_lens" in rs.rs_last_error()
    assert lib.rs_create_field(None, None, 5, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    xy = (ctypes.c_float * 2)(0.0, float("nan"))
    assert lib.rs_create_field(xy, None, 1, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    xy = (ctypes.c_float * 2)(0.0, 1.0)
    assert lib.rs_create_field(xy, None, 1, float("inf"), 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    m = (ctypes.c_float * 1)(-1.0)
    assert lib.rs_create_field(xy, m, 1, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    assert lib.rs_create_field(xy, None, 1 << 31, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EOVERFLOW
    # NULL field / grid / window
    g = rs._cgrid(rs.RayGrid((0.0, 0.0), (1.0, 1.0), (4, 4)))
    w = rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), (4, 4)))
    assert lib.rs_shoot(None, ctypes.byref(g), ctypes.byref(w), None, None, None) == rs.RS_EINVAL
    assert lib.rs_trace(None, ctypes.byref(g), None, 1, None, None, None, None) == rs.RS_EINVAL
    assert lib.rs_trace_certified(None, ctypes.byref(g), None, 1, None, None, None) == rs.RS_EINVAL
    assert lib.rs_batch_create(0, None, None, None, None, None, ctypes.byref(h)) == rs.RS_EINVAL
    assert lib.rs_destroy_field(None) == rs.RS_OK
    assert lib.rs_batch_destroy(None) == rs.RS_OK


def test_grid_window_validation(rs):
    lib = rs.load()
    fake = ctypes.c_void_p(1)  # never dereferenced: validation fails first
    bad_grids = [
        rs.RayGrid((0.0, 0.0), (0.0, 1.0), (4, 4)),            # zero spacing
        rs.RayGrid((float("nan"), 0.0), (1.0, 1.0), (4, 4)),   # non-finite origin
        rs.RayGrid((0.0, 0.0), (1.0, 1.0), (-1, 4)),           # negative extent
        rs.RayGrid((0.0, 0.0), (1e18, 1.0), (4, 4)),           # beyond the coordinate limit
    ]
    w = rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), (4, 4)))
    for bg in bad_grids:
        g = rs._cgrid(bg)
        assert lib.rs_shoot(fake, ctypes.byref(g), ctypes.byref(w), ctypes.c_void_p(16), None, None) == rs.RS_EINVAL
    g = rs._cgrid(rs.RayGrid((0.0, 0.0), (1.0, 1.0), (4, 4)))
    for bw in [rs.Window((1.0, -1.0), (1.0, 1.0), (4, 4)), rs.Window((-1.0, -1.0), (1.0, 1.0), (0, 4)),
               rs.Window((-1.0, float("inf")), (1.0, 1.0), (4, 4)),
               rs.Window((-1.0, -1.0), (1.0, 1.0), ((1 << 22) + 1, 1))]:
        ww = rs._cwin(bw)
        assert lib.rs_shoot(fake, ctypes.byref(g), ctypes.byref(ww), ctypes.c_void_p(16), None, None) == rs.RS_EINVAL
    # row range outside the grid
    assert lib.rs_shoot_rows(fake, ctypes.byref(g), 2, 9, ctypes.byref(w), ctypes.c_void_p(16), None,
                             None) == rs.RS_EINVAL
    # unknown launch shape
    assert lib.rs_set_launch_config(0, 96, 3, 256, 2) == rs.RS_EINVAL
    assert lib.rs_set_launch_config(0, 128, 8, 384, 2) == rs.RS_EINVAL   # no such lens tile
    assert lib.rs_set_launch_config(0, 128, 8, 512, 5) == rs.RS_EINVAL   # no such occupancy floor
    shapes = rs.rs_launch_configs()
    assert len(shapes) >= 4 and {s[2] for s in shapes} == {256, 512} and {s[3] for s in shapes} >= {2, 3}
    assert len(set(shapes)) == len(shapes)
    saved = rs.rs_get_launch_config(False)
    try:
        rs.rs_set_launch_config(False, 128, 8, 512, 3)
        assert rs.rs_get_launch_config(False) == (128, 8, 512, 3)
    finally:
        rs.rs_set_launch_config(False, *saved)


def test_struct_layouts_match_binding(rs, tmp_path):
    """sizeof/offsetof of the ABI structs as a C compiler sees include/rs.h equal the ctypes mirrors."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rs.h"\n'
        'int main(void) {\n'
        '  printf("%zu %zu %zu %zu\\n", sizeof(rs_ray_grid), offsetof(rs_ray_grid, n), sizeof(rs_window),'
        ' offsetof(rs_window, npix));\n'
        '  printf("%zu %zu %zu %zu\\n", sizeof(rs_track), offsetof(rs_track, y0), offsetof(rs_track, step),'
        ' offsetof(rs_track, n));\n'
        '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    g, w, t = rs._Grid, rs._Window, rs._Track
    assert [int(v) for v in lines[0].split()] == [ctypes.sizeof(g), g.n.offset, ctypes.sizeof(w), w.npix.offset]
    assert [int(v) for v in lines[1].split()] == [ctypes.sizeof(t), t.y0.offset, t.step.offset, t.n.offset]


def test_light_curve_validation(rs):
    lib = rs.load()
    maps = (ctypes.c_void_p * 1)(16)
    win = (rs._Window * 1)(rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), (64, 64))))
    out = ctypes.c_void_p(16)

    def call(tracks, profile=rs.RS_PROFILE_GAUSSIAN, s=0.1, n_maps=1, m=maps, w=win, o=out):
        T = (rs._Track * max(1, len(tracks)))()
        for k, (mp, y0, st, n) in enumerate(tracks):
            T[k].map, T[k].n = mp, n
            T[k].y0[0], T[k].y0[1] = y0
            T[k].step[0], T[k].step[1] = st
        return lib.rs_light_curves(n_maps, m, w, profile, s, len(tracks), T, o, None, None)

    good = (0, (0.0, 0.0), (0.01, 0.0), 10)
    assert call([], s=0.1) == rs.RS_OK                                   # nothing to do: no CUDA call
    assert call([(0, (0.0, 0.0), (0.0, 0.0), 0)], n_maps=0, m=None, w=None, o=None) == rs.RS_OK
    assert call([good], profile=7) == rs.RS_EINVAL
    assert call([good], s=0.0) == rs.RS_EINVAL
    assert call([good], s=float("nan")) == rs.RS_EINVAL
    assert call([(1, (0.0, 0.0), (0.01, 0.0), 10)]) == rs.RS_EINVAL      # map index out of range
    assert "map 1" in rs.rs_last_error()
    assert call([(0, (0.0, 0.0), (0.01, 0.0), -1)]) == rs.RS_EINVAL      # negative sample count
    assert call([(0, (float("inf"), 0.0), (0.01, 0.0), 10)]) == rs.RS_EINVAL
    assert call([(0, (0.0, 0.0), (1e9, 0.0), 10)]) == rs.RS_EINVAL       # last sample beyond 1e9
    assert call([good], s=1e6) == rs.RS_EINVAL                          # support beyond 2^20 pixels
    assert call([good], o=None) == rs.RS_EINVAL
    assert call([(0, (0.0, 0.0), (0.0, 0.0), 1 << 41)]) == rs.RS_EOVERFLOW
    bad_win = (rs._Window * 1)(rs._cwin(rs.Window((1.0, -1.0), (1.0, 1.0), (64, 64))))
    assert call([good], w=bad_win) == rs.RS_EINVAL
    big = (rs._Window * 1)(rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), ((1 << 24) + 1, 64))))
    assert call([good], w=big) == rs.RS_EINVAL
    far = (rs._Window * 1)(rs._cwin(rs.Window((1e8, -1.0), (1e8 + 1e-3, 1.0), (64, 64))))
    assert call([good], w=far) == rs.RS_EINVAL                           # |lo| / pixel beyond 2^30


def test_culled_shoot_validation(rs):
    lib = rs.load()
    g = rs._cgrid(rs.RayGrid((0.0, 0.0), (1.0, 1.0), (4, 4)))
    w = rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), (4, 4)))
    fake = ctypes.c_void_p(1)  # never dereferenced: validation fails first
    assert lib.rs_shoot_culled(None, ctypes.byref(g), 0, 4, ctypes.byref(w), ctypes.c_void_p(16), None, None,
                               None) == rs.RS_EINVAL
    assert lib.rs_shoot_culled(fake, ctypes.byref(g), 3, 9, ctypes.byref(w), ctypes.c_void_p(16), None, None,
                               None) == rs.RS_EINVAL
    assert lib.rs_shoot_culled(fake, ctypes.byref(g), 0, 4, ctypes.byref(w), None, None, None, None) == rs.RS_EINVAL
    bad = rs._cwin(rs.Window((1.0, -1.0), (1.0, 1.0), (4, 4)))
    assert lib.rs_shoot_culled(fake, ctypes.byref(g), 0, 4, ctypes.byref(bad), ctypes.c_void_p(16), None, None,
                               None) == rs.RS_EINVAL


def test_zoom_geometry(rs):
    g = rs.RayGrid((-10.0 + 0.01, -10.0 + 0.01), (0.02, 0.02), (1000, 1000))
    z = rs.zoom_grid(g, 4)
    assert z.n == (4000, 4000) and abs(z.spacing[0] - 0.005) < 1e-15
    assert abs(z.origin[0] - (-10.0 + 0.0025)) < 1e-12           # cell-centred sub-rays
    w = rs.Window((-2.0, -2.0), (2.0, 2.0), (256, 256))
    zw = rs.zoom_window(w, (0.0, -1.0), (1.0, 0.5), 4)
    assert zw.npix == (256, 384)


def test_python_names_cover_the_boundary(rs):
    """Every C entry point has a Python function of the same name, listed in __all__."""
    for name in rs.EXPORTED_SYMBOLS:
        assert name in rs.__all__ and callable(getattr(rs, name)), name
    assert all(hasattr(rs, n) for n in rs.__all__)


def test_widening_entry_points_validate_before_cuda(rs):
    """Moving fields, staged and streamed shoots, plans and the injection hook reject bad arguments on the
    host (no CUDA call is made, so these run without a GPU)."""
    lib = rs.load()
    h = ctypes.c_void_p()
    xy = (ctypes.c_float * 4)(0.0, 1.0, 2.0, 3.0)
    v_bad = (ctypes.c_float * 4)(0.0, float("nan"), 0.0, 0.0)
    assert lib.rs_create_moving_field(xy, None, None, 2, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    assert lib.rs_create_moving_field(xy, v_bad, None, 2, 0.0, 0.0, 0, None, ctypes.byref(h)) == rs.RS_EINVAL
    assert lib.rs_field_set_time(None, 1.0, None) == rs.RS_EINVAL
    t = ctypes.c_double()
    assert lib.rs_field_time(None, ctypes.byref(t)) == rs.RS_EINVAL
    g = rs._cgrid(rs.RayGrid((0.0, 0.0), (1.0, 1.0), (4, 4)))
    w = rs._cwin(rs.Window((-1.0, -1.0), (1.0, 1.0), (4, 4)))
    assert lib.rs_shoot_staged(0, None, ctypes.byref(g), 0, 4, ctypes.byref(w), ctypes.c_void_p(16), None,
                               None) == rs.RS_EINVAL
    parts = (ctypes.c_void_p * 1)(None)
    assert lib.rs_shoot_staged(1, parts, ctypes.byref(g), 0, 4, ctypes.byref(w), ctypes.c_void_p(16), None,
                               None) == rs.RS_EINVAL
    for per_pass in (0, 1000, 3 << 30):
        assert lib.rs_shoot_streamed(xy, None, 2, 0.0, 0.0, per_pass, ctypes.byref(g), 0, 4, ctypes.byref(w),
                                     ctypes.c_void_p(16), None, None) == rs.RS_EINVAL
    bad_xy = (ctypes.c_float * 4)(0.0, float("inf"), 2.0, 3.0)
    assert lib.rs_shoot_streamed(bad_xy, None, 2, 0.0, 0.0, 1024, ctypes.byref(g), 0, 4, ctypes.byref(w),
                                 ctypes.c_void_p(16), None, None) == rs.RS_EINVAL
    assert lib.rs_light_curve_plan_launch(None, None, None, None) == rs.RS_EINVAL
    assert lib.rs_light_curve_plan_destroy(None) == rs.RS_OK
    assert lib.rs_set_alloc_failure(-2) == rs.RS_EINVAL
    assert lib.rs_set_alloc_failure(-1) == rs.RS_OK
    assert lib.rs_set_staged_state_budget(1000) == rs.RS_EINVAL
    assert lib.rs_create_field_view(None, 0, 0, ctypes.byref(h)) == rs.RS_EINVAL
    assert lib.rs_create_field_view(None, 0, 0, None) == rs.RS_EINVAL
