"""The ring of lens partitions across processes (Section 3.3): schedule, transfers and the assembled map.

On CPU the FP64 oracle stands in for the device passes: each process adds the oracle's deflection of its own
lens shard to the per-ray state it received and hands it on; the last one maps and bins.  The map must equal the
oracle's single-process map of all the lenses.  The GPU test drives the same schedule with the library's partition
passes, every process of the ring simulated in one (transfers are device copies), against rs_shoot_staged.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0905_2453_gb300.lens_ring import ray_blocks, rank_program, run_dist, run_loopback

SPLIT = (0, 256, 512, 600)  # three shards: 256, 256 and 88 lenses


def _field():
    import rs_inputs as ri
    return ri.disc_field("ring", 600, 0.45, 0.05, 0.3, 90, 40, seed=7, mass="salpeter")


class OracleOps:
    """Partition passes by the FP64 oracle: the state is the per-ray deflection summed so far (float64)."""

    def __init__(self, spec, shard, blocks, log=None):
        import oracle
        self.oracle, self.spec, self.blocks, self.log = oracle, spec, blocks, log
        a, b = shard
        self.xy = spec.lens_xy[a:b]
        self.m = None if spec.masses is None else spec.masses[a:b]
        n0 = int(spec.grid.n[0])
        rays = max((e - s) * n0 for s, e in blocks)
        self._state = [torch.zeros((rays, 2), dtype=torch.float64) for _ in range(2)]
        self._list = [torch.zeros(4, dtype=torch.int64) for _ in blocks]
        self._ff = [torch.zeros(4, dtype=torch.float64) for _ in blocks]
        npx = (int(spec.window.npix[1]), int(spec.window.npix[0]))
        self.counts = np.zeros(npx, np.uint32)
        self.oow = 0

    def _rays(self, b, e):
        n0 = int(self.spec.grid.n[0])
        jj, ii = np.meshgrid(np.arange(b, e), np.arange(n0), indexing="ij")
        return np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int64)

    def state(self, k):
        return self._state[k % 2]

    def list(self, k):
        return self._list[k]

    def ff(self, k):
        return self._ff[k]

    def pass_(self, k, b, e, first, last):
        g = self.spec.grid
        ij = self._rays(b, e)
        _, alpha, _ = self.oracle.trace(self.xy, self.m, self.spec.kappa_c, self.spec.gamma, g.origin, g.spacing, ij)
        st = self.state(k)[:ij.shape[0]]
        if first:
            st.zero_()
        st += torch.from_numpy(alpha)
        if last:
            # Eq. 6 of the oracle itself: lambda x from a trace without lenses, minus the summed deflection
            y0, _, _ = self.oracle.trace(np.zeros((0, 2), np.float32), None, self.spec.kappa_c, self.spec.gamma,
                                         g.origin, g.spacing, ij)
            y = y0 - st.numpy()
            w = self.spec.window
            _, oow = self.oracle.bin_positions(y, w.lo, w.hi, w.npix, counts=self.counts)
            self.oow += oow
        if self.log is not None:
            self.log.append(("pass", k, first, last))

    def recheck(self, k, b, e, first, last):
        self.ff(k).add_(1.0)  # the ring order is what is checked
        if self.log is not None:
            self.log.append(("recheck", k, first, last, float(self.ff(k)[0]), int(self.list(k)[0])))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        spec = _field()
        blocks = ray_blocks(3, 87, 16)
        shards = [(0, 512), (512, 600)]
        ops = OracleOps(spec, shards[rank], blocks)
        run_dist(rank_program(rank, world, blocks, ops, certify=False))
        q.put((rank, ops.counts.copy(), ops.oow))
    finally:
        dist.destroy_process_group()


def test_ray_blocks_cover_rows():
    assert ray_blocks(3, 87, 16) == [(3, 19), (19, 35), (35, 51), (51, 67), (67, 83), (83, 87)]
    assert ray_blocks(5, 5, 4) == []
    with pytest.raises(ValueError):
        ray_blocks(0, 10, 0)


def test_two_process_ring_equals_single_process_oracle():
    """World size 2 over gloo: process 0 holds lenses [0, 512), process 1 [512, 600); rows 3..86 in blocks of 16."""
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (c, o)) for r, c, o in (q.get(timeout=300) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = _field()
    ref, oow_ref = oracle.shoot_field(spec, rows=(3, 87))
    counts, oow = res[world - 1]
    assert np.array_equal(counts, ref) and oow == oow_ref
    assert res[0][0].sum() == 0  # only the last process bins


def test_loopback_schedule_three_processes_with_recheck_ring():
    """Three simulated processes: the map equals the oracle's, every block's re-evaluation visits the processes
    in ring order after the last process's list was broadcast, and the float-float buffer accumulates along it."""
    import oracle
    spec = _field()
    blocks = ray_blocks(0, 90, 32)
    logs = [[] for _ in range(3)]
    ops = [OracleOps(spec, (SPLIT[r], SPLIT[r + 1]), blocks, logs[r]) for r in range(3)]
    for k in range(len(blocks)):
        ops[2].list(k)[0] = 100 + k  # the last process's list of block k
    run_loopback([rank_program(r, 3, blocks, ops[r], certify=True) for r in range(3)])
    ref, oow_ref = oracle.shoot_field(spec)
    assert np.array_equal(ops[2].counts, ref) and ops[2].oow == oow_ref
    for r in range(3):
        passes = [x for x in logs[r] if x[0] == "pass"]
        assert [x[1] for x in passes] == list(range(len(blocks)))
        assert all(x[2] == (r == 0) and x[3] == (r == 2) for x in passes)
        rech = [x for x in logs[r] if x[0] == "recheck"]
        # block k's float-float buffer arrives having visited processes 0 .. r - 1, and every process sees the
        # last process's list of that block
        assert [(x[1], x[4], x[5]) for x in rech] == [(k, float(r + 1), 100 + k) for k in range(len(blocks))]


def test_loopback_reports_a_deadlock():
    def waits_forever(r):
        yield ("recv", torch.zeros(1), 1 - r)
    with pytest.raises(RuntimeError, match="deadlocked"):
        run_loopback([waits_forever(0), waits_forever(1)])


@pytest.mark.gpu
def test_device_ring_two_partitions_equals_staged_shoot():
    """The library's partition passes driven by the ring schedule (two partitions, every process simulated in
    one, transfers as device copies; certified binning on) give rs_shoot_staged's counts bit for bit."""
    from gpu_helpers import dev, rs
    from paper_0905_2453_gb300.lens_ring import DeviceOps
    m = rs()
    import rs_inputs as ri
    spec = ri.disc_field("ring-gpu", 1300, 0.45, 0.05, 0.3, 700, 160, seed=8, mass="salpeter")
    cuts = (0, 768, 1300)
    parts = [m.Field(spec.lens_xy[a:b], spec.masses[a:b], spec.kappa_c, spec.gamma) for a, b in zip(cuts, cuts[1:])]
    try:
        weighted = any(p.info()[1] for p in parts)
        npx = (int(spec.window.npix[1]), int(spec.window.npix[0]))
        ref = torch.zeros(npx, dtype=torch.int32, device=dev())
        ref_o = torch.zeros(1, dtype=torch.int64, device=dev())
        m.rs_shoot_staged([p.handle for p in parts], spec.grid, 0, int(spec.grid.n[1]), spec.window, ref, ref_o)
        counts = torch.zeros_like(ref)
        oow = torch.zeros_like(ref_o)
        blocks = ray_blocks(0, int(spec.grid.n[1]), 96)
        ops = [DeviceOps(parts[0], weighted, spec.grid, spec.window, blocks),
               DeviceOps(parts[1], weighted, spec.grid, spec.window, blocks, counts, oow)]
        run_loopback([rank_program(r, 2, blocks, ops[r], certify=m.rs_get_certified_binning()) for r in range(2)])
        torch.cuda.synchronize()
        assert all(p.status() == m.RS_OK for p in parts)
        assert torch.equal(counts, ref) and torch.equal(oow, ref_o)
        assert int(counts.sum().item()) + int(oow.item()) == spec.grid.n_rays
    finally:
        for p in parts:
            p.close()
