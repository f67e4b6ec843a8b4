"""Host logic of the benchmark that needs no GPU: the launch shape of a sampled step and its whole-wave unit."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_0905_2453_gb300.tune import wave_rows  # noqa: E402

# The tuner's proxy rates (interactions/s) of every shape on the 1e8-lens field, GB300, one run.
RATES_1E8 = {"128x8x512x3": 5.559e12, "128x8x256x3": 5.531e12, "128x8x512x2": 5.420e12, "256x8x256x1": 5.416e12,
             "128x8x256x2": 5.321e12, "128x4x256x4": 5.224e12, "256x6x256x1": 5.211e12, "64x8x512x2": 5.162e12,
             "128x4x512x2": 5.152e12, "64x8x256x2": 5.076e12, "128x4x256x2": 5.065e12, "256x4x256x1": 4.958e12}


def _units_8192(shape):
    """Rows of the 8192-column grid that fill whole waves at the shape's compiled occupancy on 152 SMs."""
    return wave_rows(8192, shape[0], shape[1], 152, shape[3])


def test_three_cta_units_of_the_1e8_grid():
    # three CTAs of 128 x 8 per SM fill whole waves only with 228 rows (four waves); two do with 76 (two waves)
    assert _units_8192((128, 8, 512, 3)) == 228 and _units_8192((128, 8, 512, 2)) == 76
    assert 228 // 4 * 32 == 4 * 3 * 152  # 57 row groups of 32 CTAs = 1824 CTAs = 4 waves of 456


def test_step_shape_keeps_two_wave_steps_on_the_1e8_field():
    """The fastest shape (three CTAs per SM, 2.6 % ahead) needs four-wave steps; the two-CTA 128x8x512 is within
    the 5 % slack and fills whole waves with a third of the rows, so the step takes it."""
    got = bench.choose_step_shape((128, 8, 512, 3), RATES_1E8, _units_8192)
    assert got == (128, 8, 512, 2)
    assert _units_8192(got) == 76


def test_step_shape_breaks_equal_units_by_rate():
    """128x8x256x2 and 128x8x512x2 have the same 76-row unit; the faster of the two is taken whatever the
    dictionary order."""
    rates = dict(sorted(RATES_1E8.items()))  # 128x8x256x2 listed before 128x8x512x2
    assert bench.choose_step_shape((128, 8, 512, 3), rates, _units_8192) == (128, 8, 512, 2)


def test_step_shape_takes_a_larger_unit_when_it_is_much_faster():
    """A shape more than the slack faster than every smaller-unit shape keeps its larger unit."""
    rates = {"128x8x512x3": 6.0e12, "128x8x512x2": 5.0e12, "64x8x256x2": 4.9e12}
    assert bench.choose_step_shape((128, 8, 512, 3), rates, _units_8192) == (128, 8, 512, 3)
    # wider slacks admit the 76-row two-CTA shape (18 %), then the 38-row 64-thread one (20 %)
    assert _units_8192((64, 8, 256, 2)) == 38
    assert bench.choose_step_shape((128, 8, 512, 3), rates, _units_8192, slack=0.18) == (128, 8, 512, 2)
    assert bench.choose_step_shape((128, 8, 512, 3), rates, _units_8192, slack=0.2) == (64, 8, 256, 2)


def test_step_shape_without_rates_is_the_given_shape():
    assert bench.choose_step_shape((64, 8, 256, 2), {}, _units_8192) == (64, 8, 256, 2)
