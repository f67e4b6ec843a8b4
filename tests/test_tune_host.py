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
