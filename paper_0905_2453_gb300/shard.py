"""Row sharding of one magnification map over several processes (one per GPU).

Rays are independent (Section 2 of the paper), so a map's grid rows can be split
into contiguous blocks, each block shot into a local map (``rs_shoot_rows``), and
the local maps summed with one reduction.  Ray positions depend only on (i, j), so
the summed map equals a single-process map bit for bit.  This is the paper's
multi-GPU ray partition (Section 2.3) with the binning moved to the devices and
the host-side merge replaced by a collective sum of uint32 counts.

The shoot itself is passed in as a callable, so the same host logic runs with
device shoots (NCCL) or, in tests, with any other row shooter (gloo on CPU).
"""
from __future__ import annotations

from typing import Callable, List, Tuple


def row_partition(n_rows: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous, balanced row blocks [(begin, end)] for ranks 0..world-1 (sizes differ by <= 1)."""
    if world < 1 or n_rows < 0:
        raise ValueError("world >= 1 and n_rows >= 0 required")
    base, extra = divmod(n_rows, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def shoot_sharded(shoot_rows: Callable, n_rows: int, counts, out_of_window, rank: int, world: int, group=None,
                  row_begin: int = 0):
    """Shoot this rank's block of rows [row_begin, row_begin + n_rows) into ``counts``/``out_of_window`` and sum
    them over ranks in place.

    shoot_rows(begin, end, counts, out_of_window) accumulates the rows' counts.
    counts: int32 tensor (uint32 bit patterns; the sum wraps like uint32);
    out_of_window: int64 tensor of one element.  Both must start at zero on every rank.
    Returns this rank's row block (grid rows).
    """
    import torch.distributed as dist
    b, e = row_partition(n_rows, world)[rank]
    b, e = b + row_begin, e + row_begin
    if e > b:
        shoot_rows(b, e, counts, out_of_window)
    if world > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(out_of_window, op=dist.ReduceOp.SUM, group=group)
    return b, e


def device_row_shooter(field, grid, window, stream=None):
    """A shoot_rows callable backed by the library's rs_shoot_rows on the current device."""
    from . import rs_shoot_rows

    def shoot(b, e, counts, out_of_window):
        rs_shoot_rows(field.handle, grid, b, e, window, counts, out_of_window, stream)

    return shoot
