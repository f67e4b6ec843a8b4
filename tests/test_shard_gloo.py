"""Multi-process row sharding of one map (world size 2, gloo on CPU).

The host logic of the multi-GPU path -- row partition, per-rank accumulation,
sum of the count maps -- runs in two CPU processes; the FP64 oracle stands in
for the per-rank device shoot.  The summed map must equal a single-process map
bit for bit, and the partition must cover every row exactly once.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, row_begin=0, n_rows=None):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    import rs_inputs as ri
    from paper_0905_2453_gb300.shard import shoot_sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        f = ri.disc_field("shard", 150, 0.5, 0.1, 0.2, 97, 48, seed=4, mass="salpeter")
        counts = torch.zeros((48, 48), dtype=torch.int32)
        oow = torch.zeros(1, dtype=torch.int64)

        def shoot_rows(b, e, c, o):
            cn = c.numpy().view(np.uint32)
            _, oo = oracle.shoot_field(f, rows=(b, e), counts=cn)
            o += oo

        blk = shoot_sharded(shoot_rows, f.grid.n[1] if n_rows is None else n_rows, counts, oow, rank, world,
                            row_begin=row_begin)
        q.put((rank, blk, counts.numpy().copy(), int(oow.item())))
    finally:
        dist.destroy_process_group()


def test_row_partition_covers_rows():
    from paper_0905_2453_gb300.shard import row_partition
    for n, w in ((0, 3), (1, 4), (97, 2), (100, 7), (4096, 8)):
        parts = row_partition(n, w)
        assert len(parts) == w and parts[0][0] == 0 and parts[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [e - b for b, e in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        row_partition(10, 0)


def test_two_rank_map_equals_single_process():
    import oracle
    import rs_inputs as ri
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = ri.disc_field("shard", 150, 0.5, 0.1, 0.2, 97, 48, seed=4, mass="salpeter")
    ref, oow_ref = oracle.shoot_field(f)
    blocks = sorted(r[1] for r in res)
    assert blocks == [(0, 49), (49, 97)]
    for _, _, counts, oow in res:
        assert np.array_equal(counts.view(np.uint32), ref)
        assert oow == oow_ref


def test_two_rank_block_with_row_offset_equals_single_process():
    """The benchmark's sharded step: a block of rows [row_begin, row_begin + n) split over two ranks and summed
    equals one process shooting the block."""
    import oracle
    import rs_inputs as ri
    world, row_begin, n = 2, 17, 44
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, row_begin, n)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = ri.disc_field("shard", 150, 0.5, 0.1, 0.2, 97, 48, seed=4, mass="salpeter")
    ref, oow_ref = oracle.shoot_field(f, rows=(row_begin, row_begin + n))
    assert sorted(r[1] for r in res) == [(17, 39), (39, 61)]
    for _, _, counts, oow in res:
        assert np.array_equal(counts.view(np.uint32), ref)
        assert oow == oow_ref
