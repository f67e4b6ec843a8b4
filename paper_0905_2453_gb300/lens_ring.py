"""Lens partitions held by different processes: the ring of partially deflected rays (Section 3.3).

The paper sums the deflection of every ray over lens subsets, passing the partially deflected rays from GPU to
GPU.  Here process r holds lens partition r (a field of shard r of the lenses, in lens order; every partition but
the last a multiple of 256 lenses).  The grid rows are cut into ray blocks, and block k visits the processes in
order 0, 1, ..., W - 1: each adds its lenses to the block's per-ray state (``rs_partition_pass``) and hands the
state (28 bytes per ray) on; the last one maps and bins.  The blocks are pipelined: while process r works on
block k, process r + 1 works on block k - 1.  With certified binning on, the last process's list of rays to
re-evaluate then goes to every process (one broadcast per block), and their float-float partial deflections of
those rays travel the same ring (``rs_partition_recheck``, 16 bytes per listed ray); the last process bins them.
The map is complete on the last process and equals ``rs_shoot_staged`` over the same partitions bit for bit.

A process's schedule is a generator (``rank_program``) that performs its own steps through an ``ops`` object
and yields the transfers it needs -- ("recv", buffer, src), ("send", buffer, dst), ("bcast", buffer, src) -- so
the same schedule runs over ``torch.distributed`` (``run_dist``: NCCL point-to-point on GPUs, gloo on CPUs) or
with every process of the ring simulated in one (``run_loopback``).
"""
from __future__ import annotations

from collections import defaultdict, deque
from typing import Callable, List, Sequence, Tuple


def ray_blocks(row_begin: int, row_end: int, block_rows: int) -> List[Tuple[int, int]]:
    """Contiguous row blocks [(begin, end)] of at most block_rows rows covering [row_begin, row_end)."""
    if block_rows < 1 or row_end < row_begin:
        raise ValueError("block_rows >= 1 and row_end >= row_begin required")
    return [(b, min(b + block_rows, row_end)) for b in range(row_begin, row_end, block_rows)]


def rank_program(rank: int, world: int, blocks: Sequence[Tuple[int, int]], ops, certify: bool):
    """The schedule of one process of the ring (a generator yielding its transfers; see the module text).

    ops.state(k), ops.list(k), ops.ff(k): the buffers of block k (state buffers may be shared between blocks
    two apart); ops.pass_(k, b, e, first, last) and ops.recheck(k, b, e, first, last) enqueue the process's
    steps for block k over rows [b, e)."""
    first, last = rank == 0, rank == world - 1
    for k, (b, e) in enumerate(blocks):
        if not first:
            yield ("recv", ops.state(k), rank - 1)
        ops.pass_(k, b, e, first, last)
        if not last:
            yield ("send", ops.state(k), rank + 1)
    if certify:
        for k, (b, e) in enumerate(blocks):
            yield ("bcast", ops.list(k), world - 1)
            if not first:
                yield ("recv", ops.ff(k), rank - 1)
            ops.recheck(k, b, e, first, last)
            if not last:
                yield ("send", ops.ff(k), rank + 1)


def run_dist(program, group=None) -> None:
    """Run one process's schedule with torch.distributed point-to-point transfers and broadcasts."""
    import torch.distributed as dist
    for kind, buf, peer in program:
        if kind == "send":
            dist.send(buf, peer, group=group)
        elif kind == "recv":
            dist.recv(buf, peer, group=group)
        else:
            dist.broadcast(buf, peer, group=group)


def run_loopback(programs: Sequence, copy: Callable = None) -> None:
    """Run the schedules of every process of a ring in one process: transfers are copies between the processes'
    buffers (copy(dst, src); default dst.copy_(src)), in the order each pair of processes issued them."""
    copy = copy or (lambda dst, src: dst.copy_(src))
    queues = defaultdict(deque)            # (src, dst) -> buffers sent, in order
    posted = defaultdict(list)             # src -> buffers broadcast, in order
    bcast_seen = defaultdict(int)          # (rank, src) -> broadcasts already received
    pending = [next(p, None) for p in programs]
    while any(op is not None for op in pending):
        progress = False
        for r, op in enumerate(pending):
            while op is not None:
                kind, buf, peer = op
                if kind == "send":
                    queues[(r, peer)].append(buf.clone())
                elif kind == "recv":
                    if not queues[(peer, r)]:
                        break
                    copy(buf, queues[(peer, r)].popleft())
                else:
                    if r == peer:
                        posted[peer].append(buf.clone())
                    else:
                        seen = bcast_seen[(r, peer)]
                        if seen >= len(posted[peer]):
                            break
                        copy(buf, posted[peer][seen])
                    bcast_seen[(r, peer)] += 1
                op = next(programs[r], None)
                progress = True
            pending[r] = op
        if not progress:
            raise RuntimeError("ring schedule deadlocked: every process waits for a transfer nobody sent")


class DeviceOps:
    """The library's partition passes for one process of the ring: its partition field, the grid, window and
    ray blocks, and device buffers (two state buffers used by block parity; a list and a float-float buffer per
    block).  counts / out_of_window receive the map on the last process."""

    def __init__(self, part, weighted: bool, grid, window, blocks, counts=None, out_of_window=None, stream=None,
                 device=None):
        import torch

        from . import rs_partition_buffer_bytes
        self.part, self.weighted, self.grid, self.window = part, bool(weighted), grid, window
        self.counts, self.out_of_window, self.stream = counts, out_of_window, stream
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        sizes = [rs_partition_buffer_bytes(grid, b, e) for b, e in blocks]
        sb = max((s[0] for s in sizes), default=16)
        self._state = [torch.zeros(max(sb, 16), dtype=torch.uint8, device=dev) for _ in range(2)]
        self._list = [torch.zeros(s[1], dtype=torch.uint8, device=dev) for s in sizes]
        self._ff = [torch.zeros(s[2], dtype=torch.uint8, device=dev) for s in sizes]

    def state(self, k):
        return self._state[k % 2]

    def list(self, k):
        return self._list[k]

    def ff(self, k):
        return self._ff[k]

    def pass_(self, k, b, e, first, last):
        from . import rs_partition_pass
        rs_partition_pass(self.part.handle, self.weighted, self.grid, b, e, self.window, self.state(k), first, last,
                          self.counts, self.out_of_window, self._list[k], self.stream)

    def recheck(self, k, b, e, first, last):
        from . import rs_partition_recheck
        rs_partition_recheck(self.part.handle, self.weighted, self.grid, b, e, self.window, self._list[k],
                             self._ff[k], first, last, self.counts, self.out_of_window, self.stream)


def shoot_lens_ring(part, weighted: bool, grid, row_begin: int, row_end: int, window, counts, out_of_window,
                    rank: int, world: int, block_rows: int = 256, stream=None, group=None) -> None:
    """This process's share of a lens-partitioned shoot over rows [row_begin, row_end) with torch.distributed
    transfers between the holders of the partitions (process r holds partition r).  The counts accumulate on
    the last process (world - 1); `weighted` must be the same everywhere (1 if any partition's masses are not
    all 1)."""
    from . import rs_get_certified_binning
    blocks = ray_blocks(row_begin, row_end, block_rows)
    ops = DeviceOps(part, weighted, grid, window, blocks, counts, out_of_window, stream)
    run_dist(rank_program(rank, world, blocks, ops, bool(rs_get_certified_binning())), group=group)
