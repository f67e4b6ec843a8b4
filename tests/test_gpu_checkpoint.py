"""Checkpoint/resume on the device: a map shot in row blocks, interrupted and resumed from its checkpoint
file, equals one rs_shoot of the whole grid bit for bit."""
import numpy as np
import pytest

import rs_inputs as ri
from gpu_helpers import rs, shoot_gpu

pytestmark = pytest.mark.gpu


def test_device_checkpoint_resume(tmp_path):
    m = rs()
    from paper_0905_2453_gb300 import checkpoint as ck
    spec = ri.disc_field("ckd", 2000, 0.45, 0.05, 0.3, 1000, 128, seed=12, mass="salpeter")
    f = m.Field.from_spec(spec)
    try:
        shoot = ck.device_block_shooter(f, spec.grid, spec.window)
        path = str(tmp_path / "ck.npz")
        _, _, row = ck.shoot_checkpointed(shoot, spec.grid.n[1], spec.window.npix, path, 96, max_blocks=3)
        assert row == 288
        counts, oow, row = ck.shoot_checkpointed(shoot, spec.grid.n[1], spec.window.npix, path, 96)
    finally:
        f.close()
    ref, oref = shoot_gpu(spec)
    assert row == spec.grid.n[1] and np.array_equal(counts, ref) and oow == oref
