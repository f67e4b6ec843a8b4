"""Beyond one field: 2^31 + 2^20 lenses (more than a field's 32-bit lens count allows), streamed from
host memory through the device (Section 3.3's billion-lens runs), against the oracle on one grid row."""
import math
import time

import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import dev, rs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_streamed_beyond_2_31_lenses_one_row_vs_oracle():
    m = rs()
    n = (1 << 31) + (1 << 20)
    kappa = 0.5
    radius = math.sqrt(n / kappa)            # unit masses: kappa_* = N / R^2
    t0 = time.perf_counter()
    xy = ri.disc_lenses_large(n, radius, seed=2024)
    t1 = time.perf_counter()
    # 16 x 16 rays in a small patch near the centre, a 4 x 4 map around their images
    g = ri.RayGrid(origin=(1.0 + 1 / 16, -2.0 + 1 / 16), spacing=(0.125, 0.125), n=(16, 16))
    w = ri.Window(lo=(-40.0, -40.0), hi=(40.0, 40.0), npix=(4, 4))
    counts = torch.zeros((4, 4), dtype=torch.int32, device=dev())
    oow = torch.zeros(1, dtype=torch.int64, device=dev())
    m.rs_shoot_streamed(xy, None, 0.0, 0.1, 1 << 28, g, 7, 8, w, counts, oow)
    got = counts.cpu().numpy().view(np.uint32)
    t2 = time.perf_counter()
    # the oracle's source positions of the 16 rays, one ray per host thread (each call single-threaded)
    from concurrent.futures import ThreadPoolExecutor

    def one(i):
        oracle.set_num_threads(1)
        return oracle.trace(xy, None, 0.0, 0.1, g.origin, g.spacing, np.array([[i, 7]], np.int64))[0][0]

    with ThreadPoolExecutor(max_workers=16) as ex:
        y = np.array(list(ex.map(one, range(16))))
    ref, oref = oracle.bin_positions(y, w.lo, w.hi, w.npix)
    t3 = time.perf_counter()
    print(f"lenses {t1 - t0:.1f} s, streamed shoot {t2 - t1:.1f} s, oracle {t3 - t2:.1f} s")
    assert int(got.sum()) + int(oow.item()) == 16
    assert np.array_equal(got, ref) and int(oow.item()) == oref
