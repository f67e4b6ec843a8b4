"""Checkpoint and resume of long map computations, and headless map output.

A map accumulates over grid rows (``rs_shoot_rows`` adds into the caller's counts, and ray positions
depend only on (i, j)), so the state of a partly finished map is its counts, its out-of-window count
and the next row: the paper's multi-day runs (Section 3.3) would restart from exactly that.
``shoot_checkpointed`` shoots a map in row blocks, writes that state atomically after every block,
and resumes from it; the resumed map equals an uninterrupted one bit for bit.

The shoot is passed in as a callable (as in ``shard``), so the same host logic runs with device
shoots or, in tests, with any other row shooter.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Optional

import numpy as np


def _save(path: str, counts: np.ndarray, oow: int, next_row: int, meta: dict) -> None:
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "wb") as fh:
        np.savez(fh, counts=counts, out_of_window=np.array([oow], np.uint64), next_row=np.array([next_row]),
                 meta=np.array(json.dumps(meta, sort_keys=True)))
    os.replace(tmp, path)


def load_checkpoint(path: str):
    """(counts uint32 [npix1, npix0], out_of_window, next_row, meta dict) of a checkpoint file."""
    with np.load(path, allow_pickle=False) as z:
        return (z["counts"].astype(np.uint32), int(z["out_of_window"][0]), int(z["next_row"][0]),
                json.loads(str(z["meta"])))


def shoot_checkpointed(shoot_rows: Callable, n_rows: int, npix, path: str, rows_per_block: int,
                       meta: Optional[dict] = None, max_blocks: Optional[int] = None):
    """Shoot rows [0, n_rows) in blocks, checkpointing to ``path`` after each block; resume if it exists.

    shoot_rows(begin, end) -> (counts uint32 [npix1, npix0], out_of_window) shoots one block from zero.
    meta: identifies the computation (field, grid, window, ...); a checkpoint with different meta is
    refused.  max_blocks stops after that many blocks (an interrupted run).  Returns (counts,
    out_of_window, next_row); the map is complete when next_row == n_rows.
    """
    if rows_per_block < 1:
        raise ValueError("rows_per_block must be >= 1")
    meta = dict(meta or {})
    meta["n_rows"] = int(n_rows)
    meta["npix"] = [int(npix[0]), int(npix[1])]
    if os.path.exists(path):
        counts, oow, row, saved = load_checkpoint(path)
        if saved != meta:
            raise ValueError(f"checkpoint {path} belongs to another computation: {saved} != {meta}")
    else:
        counts, oow, row = np.zeros((int(npix[1]), int(npix[0])), np.uint32), 0, 0
    done = 0
    while row < n_rows and (max_blocks is None or done < max_blocks):
        end = min(n_rows, row + rows_per_block)
        c, o = shoot_rows(row, end)
        counts = counts + np.asarray(c, np.uint32)      # uint32 arithmetic, as the device counts
        oow += int(o)
        row = end
        _save(path, counts, oow, row, meta)
        done += 1
    return counts, oow, row


def device_block_shooter(field, grid, window, stream=None):
    """A shoot_rows callable for shoot_checkpointed backed by rs_shoot_rows on the current device."""
    import torch

    from . import rs_shoot_rows

    dev = torch.device("cuda", torch.cuda.current_device())

    def shoot(b, e):
        c = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev)
        o = torch.zeros(1, dtype=torch.int64, device=dev)
        rs_shoot_rows(field.handle, grid, b, e, window, c, o, stream)
        return c.cpu().numpy().view(np.uint32), int(o.item())

    return shoot


def save_map(mu, path: str) -> None:
    """Write a magnification map (2-D array or tensor) headless: ``.npy`` as float32, ``.pgm`` as an 8-bit
    image of log10(mu) scaled between its 0.5 and 99.5 percentiles (row 0 of the map at the bottom)."""
    a = mu.detach().cpu().numpy() if hasattr(mu, "detach") else np.asarray(mu)
    a = np.asarray(a, np.float32)
    if path.endswith(".npy"):
        np.save(path, a)
        return
    if not path.endswith(".pgm"):
        raise ValueError("save_map writes .npy or .pgm")
    lg = np.log10(np.maximum(a, 1e-3))
    lo, hi = np.percentile(lg, [0.5, 99.5])
    img = np.clip((lg - lo) / max(hi - lo, 1e-12) * 255.0 + 0.5, 0, 255).astype(np.uint8)[::-1]
    with open(path, "wb") as fh:
        fh.write(f"P5\n{img.shape[1]} {img.shape[0]}\n255\n".encode())
        fh.write(img.tobytes())
