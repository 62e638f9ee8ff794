"""Template sharding across GPUs.

Templates are independent (each is its own resampling, FFT and 2F), so a
multi-GPU run needs no collective on the data path: each rank takes a
contiguous range of templates, balanced by the FFT work sum(N_f log N_f)
(equal shares when every template has the same FFT length), and writes its
own 2F values.  Only timing (a barrier and a max-reduction) is exchanged.
"""
from __future__ import annotations

import math

import numpy as np


def work_of(n_fft) -> np.ndarray:
    n = np.asarray(n_fft, dtype=np.float64)
    return n * np.log2(np.maximum(n, 2.0))


def shard_ranges(n_fft, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, end) template ranges, one per rank, with nearly
    equal FFT work.  ``n_fft``: FFT length of every template."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = work_of(n_fft)
    n = w.size
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(cum, target, side="left"))
        # pick the nearer of the two neighbouring boundaries, keep order
        if i > 0 and abs(cum[i - 1] - target) <= abs(cum[min(i, n)] - target):
            i -= 1
        cuts.append(min(max(i, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard(templates, rank: int, world: int, n_fft=None):
    """The rank's contiguous slice of a template array."""
    nf = np.full(len(templates), 1, np.int64) if n_fft is None else n_fft
    s, e = shard_ranges(nf, world)[rank]
    return templates[s:e], (s, e)
