"""Autotuning of the cell-list edge and the tile shape.

Both settings change only the speed (labels, statistics and particle sets are the same for
every candidate). A single job is tuned by the library itself (``seg.autotune`` ->
``seg_autotune``), which times each candidate alone; that favours small tiles, which give a
latency-bound job more blocks. A batch of many jobs fills the GPU, where small tiles only add
per-block staging overhead, so ``autotune_batch`` times each candidate on a batch: a sample of
the jobs, stepped together for a few iterations through ``seg.Batch``.
"""
from __future__ import annotations

import math
import time

from . import seg

# (cell-edge multiple of ceil(cutoff), tile in pixels)
CANDIDATES_2D = [(1, (16, 16)), (1, (32, 32)), (1, (32, 64)), (1, (64, 64)), (2, (32, 32)), (2, (32, 64)),
                 (2, (64, 64))]
CANDIDATES_3D = [(1, (8, 8, 32)), (1, (16, 16, 16)), (1, (8, 16, 32)), (2, (8, 8, 32)), (2, (16, 16, 16))]


def autotune_batch(jobs, iters: int = 5, sample: int = 128, stream=None, candidates=None, sync=None):
    """jobs: list of (image, labels0, kwargs for seg.Context), all of one dimensionality.
    Returns ({"cell_edge": e, "tile": t}, [(cell_edge_multiple, tile, seconds per iteration), ...]).
    The first ``sample`` jobs (evenly spaced over the list) are stepped as one batch with each
    candidate: one untimed iteration (graph capture), then ``iters`` timed iterations."""
    if not jobs:
        raise ValueError("no jobs")
    ndim = len(jobs[0][0].shape)
    cands = candidates or (CANDIDATES_2D if ndim == 2 else CANDIDATES_3D)
    stride = max(1, len(jobs) // sample)
    chosen = jobs[::stride][:sample]
    table = []
    best, best_t = None, math.inf
    for mult, tile in cands:
        ctxs = []
        try:
            for image, labels0, kw in chosen:
                base = max(1, math.ceil(kw.get("cutoff", 3.0)))
                ctxs.append(seg.Context(image, labels0, stream=stream, cell_edge=base * mult, tile=tile, **kw))
            b = seg.Batch(stream=stream)
            for c in ctxs:
                b.add(c)
            b.step(1)
            t0 = time.perf_counter()
            b.step(iters)
            dt = (time.perf_counter() - t0) / iters
            b.close()
        except seg.SegError:
            dt = math.inf
        finally:
            for c in ctxs:
                c.close()
        table.append((mult, tuple(tile), dt))
        if dt < best_t:
            best_t, best = dt, (mult, tuple(tile))
    if best is None:
        raise RuntimeError("no candidate ran")
    return {"cell_multiple": best[0], "tile": best[1]}, table
