"""Row-band evaluation of the FP64 oracle's Wishart statistic over host processes.

The oracle is plain single-threaded C; a 4096 x 4096 pair takes it minutes on
one core.  Its window functions only read rows within the window radius r of
an output row, so the image splits into bands of output rows: a band is
evaluated on the sub-image of its rows plus r rows each side (cut at the image
border, where the oracle clamps, exactly as on the full image), and the bands'
sums are added in band order.  Workers are started with `spawn` (a process
forked after the GPU was initialised may hang), read the two dates from .npy
files by memory map, and run the unmodified oracle.  Test infrastructure only.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _band(args):
    path1, path2, y_lo, y_hi, r, win, weights, want_grad = args
    import oracle
    o = oracle.load()
    s1 = np.load(path1, mmap_mode="r")
    s2 = np.load(path2, mmap_mode="r")
    H = s1.shape[1]
    h0, h1 = max(0, y_lo - r), min(H, y_hi + r)
    b1 = np.ascontiguousarray(s1[:, h0:h1])
    b2 = np.ascontiguousarray(s2[:, h0:h1])
    _, q = o.wishart_fwd(b1, b2, win, weights, want_map=True)
    W = s1.shape[2]
    q = q.reshape(h1 - h0, W)[y_lo - h0:y_hi - h0]
    loss = float(np.sum(q))  # numpy's pairwise sum, in row-major order
    grad = None
    if want_grad:
        grad = o.wishart_bwd(b1, b2, win, weights, 1.0, rows=(y_lo - h0, y_hi - h0))
    return loss, grad


def wishart_by_bands(path1: str, path2: str, H: int, win: int, weights, band_rows: int = 64,
                     want_grad: bool = True, processes: int | None = None):
    """(L, dL/dw) of the full image from the oracle, row band by row band in
    `processes` spawned workers (default: every host core)."""
    r = (win - 1) // 2
    weights = np.asarray(weights, dtype=np.float64)
    tasks = [(path1, path2, y, min(H, y + band_rows), r, win, weights, want_grad)
             for y in range(0, H, band_rows)]
    nproc = processes or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(min(nproc, len(tasks))) as pool:
        parts = pool.map(_band, tasks, chunksize=1)
    loss = 0.0
    grad = np.zeros(win * win) if want_grad else None
    for l_b, g_b in parts:  # band order
        loss += l_b
        if want_grad:
            grad += g_b
    return loss, grad
