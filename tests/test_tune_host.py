"""Host logic of the launch-shape tuner: the row unit that fills whole waves of CTAs (no GPU needed)."""
import pytest

from paper_0905_2453_gb300.tune import wave_rows


@pytest.mark.parametrize("n0", [1000, 1024, 4096, 8192, 16384, 1280, 3072, 37])
@pytest.mark.parametrize("block,rpt", [(64, 8), (128, 4), (128, 8), (256, 4), (256, 8), (256, 6)])
@pytest.mark.parametrize("sms", [152, 148, 1])
def test_wave_rows_fill_whole_waves_minimally(n0, block, rpt, sms):
    warps = block // 32
    cpr = -(-n0 // (32 * rpt))                  # CTAs per group of `warps` rows
    unit = wave_rows(n0, block, rpt, sms)
    assert unit % warps == 0
    groups = unit // warps
    assert (groups * cpr) % (2 * sms) == 0      # whole waves at one or two CTAs per SM
    for g in range(1, groups):                  # and no smaller number of row groups does it
        assert (g * cpr) % (2 * sms) != 0


def test_wave_rows_of_the_workloads():
    # 1e4-, 1e6- and 1e8-lens grids on 152 SMs with the tuned 4-warp, 8-ray CTAs: 76 rows = 19 row groups
    for n0 in (4096, 16384, 8192):
        assert wave_rows(n0, 128, 8, 152) == 76
    assert wave_rows(16384, 64, 8, 152) == 38
    assert wave_rows(16384, 256, 8, 152) == 152


@pytest.mark.parametrize("occ", [1, 2, 3, 4])
def test_wave_rows_at_other_occupancies(occ):
    for n0 in (4096, 8192, 16384, 1000):
        for block, rpt in ((64, 8), (128, 8), (128, 4)):
            warps, cpr = block // 32, -(-n0 // (32 * rpt))
            unit = wave_rows(n0, block, rpt, 152, occ)
            assert unit % warps == 0 and ((unit // warps) * cpr) % (occ * 152) == 0
    # the 1e8-lens grid: 64-thread CTAs four to an SM fill one wave with 38 rows
    assert wave_rows(8192, 64, 8, 152, 4) == 38


class _FakeField:
    def __init__(self, n_lens, has_mass):
        self.n_lens, self.has_mass = n_lens, has_mass

    def info(self):
        return self.n_lens, self.has_mass


class _FakeGrid:
    def __init__(self, side):
        self.n = (side, side)


def test_batch_shapes_tune_the_largest_field_of_each_mass_mode_and_lens_bucket(monkeypatch):
    """Fields are grouped by (mass mode, lens-count bucket); the field with the most rays of each group is tuned
    and its shape serves the group; the launch configuration of both mass modes is put back afterwards."""
    import paper_0905_2453_gb300 as rs
    from paper_0905_2453_gb300 import tune
    tuned = []

    def fake_autotune(field, grid, window, **kw):
        tuned.append((field.n_lens, field.has_mass, grid.n[0]))
        shape = (128, 8, 512, 3) if field.n_lens > 5000 else (128, 4, 256, 4)
        rs.rs_set_launch_config(field.has_mass, *shape)  # as the tuner does
        return (*shape, {})

    monkeypatch.setattr(tune, "autotune", fake_autotune)
    before = {m: rs.rs_get_launch_config(m) for m in (False, True)}
    fields = [_FakeField(100, False), _FakeField(110, False), _FakeField(100, True), _FakeField(10000, True),
              _FakeField(11000, True), _FakeField(100, False)]
    grids = [_FakeGrid(s) for s in (1024, 2048, 1024, 1024, 4096, 512)]
    shapes = tune.batch_shapes(fields, grids, [None] * len(fields))
    # groups: unit masses ~100 lenses (fields 0, 1, 5), masses ~100 (2), masses ~1e4 (3, 4)
    assert sorted(tuned) == sorted([(110, False, 2048), (100, True, 1024), (11000, True, 4096)])
    assert shapes == [(128, 4, 256, 4)] * 3 + [(128, 8, 512, 3)] * 2 + [(128, 4, 256, 4)]
    assert {m: rs.rs_get_launch_config(m) for m in (False, True)} == before
