"""Membrane fluctuation from a series of upper-rim height maps
("Validation and Benchmark": the RMS of the instantaneous vertical
fluctuation dh(x, y) along the upper rim of a cell held in place).

The maps come from ``System.height_map`` (orbc_height_map, on the GPU);
what is left here is arithmetic on a few thousand bins per frame."""
from __future__ import annotations

import numpy as np


def fluctuation(maps, counts, min_count: int = 1):
    """dh(x, y, t) = h(x, y, t) - <h(x, y)>_t over the bins that hold at
    least ``min_count`` lipids in every frame.

    maps, counts: [T, ny, nx] (or sequences of [ny, nx]) from successive
    height maps on the same grid.  Returns (dh, rms): dh [T, ny, nx] with NaN
    in the bins left out, rms = sqrt(mean over frames and kept bins of dh^2).
    Raises ValueError when fewer than two frames or no bin qualifies."""
    h = np.asarray(maps, dtype=np.float64)
    c = np.asarray(counts)
    if h.ndim != 3 or h.shape != c.shape:
        raise ValueError("maps and counts must both be [T, ny, nx]")
    if h.shape[0] < 2:
        raise ValueError("need at least two frames")
    keep = (c >= min_count).all(axis=0)
    if not keep.any():
        raise ValueError("no bin holds lipids in every frame")
    dh = np.full_like(h, np.nan)
    mean = h[:, keep].mean(axis=0)
    dh[:, keep] = h[:, keep] - mean
    rms = float(np.sqrt(np.mean(dh[:, keep] ** 2)))
    return dh, rms
