"""Mutation check of the oracle's pins: plant plausible mistakes in a copy of the
oracle's C source (on the CPU) and require that at least one pin fails for each.

The mutated copies are built in a temporary directory; the committed oracle is
never modified.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins

# (name, original text, mutated text)
MUTATIONS = [
    ("deflection sign x1", "double f1 = x[0] - xi1;", "double f1 = xi1 - x[0];"),
    ("dropped mass", "double m = masses ? (double)masses[i] : 1.0;", "double m = 1.0;"),
    ("wrong mass index", "(double)masses[i]", "(double)masses[0]"),
    ("transposed lens operand", "double xi2 = (double)lens_xy[2 * i + 1];", "double xi2 = (double)lens_xy[2 * i];"),
    ("wrong index in r^2", "m / (f1 * f1 + f2 * f2)", "m / (f1 * f1 + f1 * f2)"),
    ("1/r instead of 1/r^2", "m / (f1 * f1 + f2 * f2)", "m / sqrt(f1 * f1 + f2 * f2)"),
    ("shear sign", "double lam1 = (1.0 - kappa_c) - gamma;", "double lam1 = (1.0 - kappa_c) + gamma;"),
    ("dropped kappa_c", "double lam2 = (1.0 - kappa_c) + gamma;", "double lam2 = 1.0 + gamma;"),
    ("alpha added", "y[0] = lam1 * x[0] - alpha[0];", "y[0] = lam1 * x[0] + alpha[0];"),
    ("alpha axis swap", "y[1] = lam2 * x[1] - alpha[1];", "y[1] = lam2 * x[1] - alpha[0];"),
    ("transposed map", "return p2 * (int64_t)npix[0] + p1;", "return p1 * (int64_t)npix[1] + p2;"),
    ("ray spacing axis", "fma((double)j, spacing[1], origin[1])", "fma((double)j, spacing[0], origin[1])"),
    ("ray not rounded to float", "x[0] = (double)(float)fma((double)i, spacing[0], origin[0]);",
     "x[0] = fma((double)i, spacing[0], origin[0]);"),
    ("bin scale axis", "scale[1] = (double)npix[1] / (hi[1] - lo[1]);\n  const",
     "scale[1] = (double)npix[0] / (hi[0] - lo[0]);\n  const"),
    ("N_av spacing axis", "n_av = pix_area / (spacing[0] * spacing[1]);", "n_av = pix_area / (spacing[0] * spacing[0]);"),
    ("no compensation", "    a->c += (a->s - u) + t;\n  else\n    a->c += (t - u) + a->s;",
     "    a->c += 0.0;\n  else\n    a->c += 0.0;"),
    ("closed window edge", "u1 < (double)npix[0]", "u1 <= (double)npix[0]"),
]

PINS = [
    lambda: pins.test_exact_rational_bruteforce(1, True),
    lambda: pins.test_exact_rational_bruteforce(2, False),
    pins.test_exact_with_cancellation,
    pins.test_compensated_sum_alternating_large_terms,
    pins.test_zero_lenses_uniform_map,
    pins.test_zero_lenses_linear_map_lattice_counts,
    pins.test_zero_lenses_nonsquare_grid_and_map,
    pins.test_point_lens_closed_form_positions,
    pins.test_point_lens_disc_counts,
    pins.test_mirror_symmetry_map,
    pins.test_superposition,
    pins.test_gauss_law_uniform_disc,
    pins.test_ray_on_lens_is_out_of_window,
]


def _edge_case_window():
    """Rays exactly on the upper window edge must be out of window (half-open [lo, hi))."""
    import numpy as np
    g = pins.ri.RayGrid(origin=(0.0, 0.0), spacing=(0.5, 0.5), n=(5, 5))  # x in {0, .5, 1, 1.5, 2}
    counts, oow = oracle.shoot(np.zeros((0, 2), np.float32), None, 0, 0, g.origin, g.spacing, g.n,
                               (0.0, 0.0), (2.0, 2.0), (4, 4))
    assert oow == 9 and counts.sum() == 16


PINS.append(_edge_case_window)


def test_edge_case_window_on_true_oracle():
    _edge_case_window()


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(name, orig, mut, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rs_oracle.c")).read()
    assert src.count(orig) == 1, f"mutation anchor not unique/found: {orig!r}"
    bad = tmp_path / "mut.c"
    bad.write_text(src.replace(orig, mut))
    lib = oracle.compile_source(str(bad), str(tmp_path / "libmut.so"))
    failed = []
    with oracle.using_library(lib):
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failed.append(getattr(pin, "__name__", "pin"))
    assert failed, f"no pin caught mutation {name!r}"
