"""Per-band top-k candidates of a 2F spectrum (test oracle).

The paper computes 2F in every frequency bin (Eq. 6, step 7 of
Sec. III.A.2) for searches over many frequencies (Sec. I); it defines no
candidate stage.  A search keeps the loudest bins: for each band of
``band_len`` consecutive bins, the ``k`` largest 2F values in descending
order with their bin indices.  Plain definition, written out: a stable sort
of each band by descending value (ties: lower bin first); NaN bins are
skipped; a band with fewer than k finite values is padded with
(-inf, -1).  Pinned by brute force and by the invariants of a selection in
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np


def band_top_k(two_f, band_len: int, k: int):
    """two_f [n_rows, row_len] -> (values [n_rows, n_bands, k] float64,
    bins [n_rows, n_bands, k] int64), bins counted within the row."""
    a = np.atleast_2d(np.asarray(two_f, np.float64))
    n_rows, row_len = a.shape
    if row_len % band_len:
        raise ValueError("band_len must divide the row length")
    n_bands = row_len // band_len
    vals = np.full((n_rows, n_bands, k), -np.inf)
    bins = np.full((n_rows, n_bands, k), -1, np.int64)
    for r in range(n_rows):
        for b in range(n_bands):
            seg = a[r, b * band_len:(b + 1) * band_len]
            idx = np.nonzero(np.isfinite(seg))[0]
            # descending value, ties by ascending bin: lexsort's last key is primary
            order = idx[np.lexsort((idx, -seg[idx]))][:k]
            vals[r, b, :len(order)] = seg[order]
            bins[r, b, :len(order)] = order + b * band_len
    return vals, bins
