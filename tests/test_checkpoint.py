"""Checkpoint/resume of a map in row blocks (host logic, with the oracle as the row shooter on CPU) and
headless map output."""
import numpy as np
import pytest

import oracle
import rs_inputs as ri
from paper_0905_2453_gb300 import checkpoint as ck


def _oracle_rows(spec):
    def shoot(b, e):
        return oracle.shoot_field(spec, rows=(b, e))
    return shoot


def test_interrupted_and_resumed_map_equals_single_run(tmp_path):
    spec = ri.disc_field("ck", 40, 0.5, 0.0, 0.2, 97, 24, seed=3, mass="equal")
    path = str(tmp_path / "map.ckpt.npz")
    meta = {"field": "ck", "seed": 3}
    c1, o1, row = ck.shoot_checkpointed(_oracle_rows(spec), spec.grid.n[1], spec.window.npix, path, 10,
                                        meta=meta, max_blocks=4)
    assert row == 40
    counts, oow, nxt, saved = ck.load_checkpoint(path)
    assert nxt == 40 and np.array_equal(counts, c1) and oow == o1 and saved["field"] == "ck"
    c2, o2, row2 = ck.shoot_checkpointed(_oracle_rows(spec), spec.grid.n[1], spec.window.npix, path, 10, meta=meta)
    assert row2 == spec.grid.n[1]
    ref, oref = oracle.shoot_field(spec)
    assert np.array_equal(c2, ref) and o2 == oref
    with pytest.raises(ValueError):
        ck.shoot_checkpointed(_oracle_rows(spec), spec.grid.n[1], spec.window.npix, path, 10, meta={"field": "x"})


def test_save_map_npy_and_pgm(tmp_path):
    mu = np.exp(np.random.default_rng(0).normal(size=(12, 20))).astype(np.float32)
    ck.save_map(mu, str(tmp_path / "m.npy"))
    assert np.array_equal(np.load(tmp_path / "m.npy"), mu)
    ck.save_map(mu, str(tmp_path / "m.pgm"))
    data = (tmp_path / "m.pgm").read_bytes()
    assert data.startswith(b"P5\n20 12\n255\n") and len(data) == len(b"P5\n20 12\n255\n") + 240
