"""Autotuning of the cell edge and tile shape: every candidate gives the same labels, the
same statistics and the same particle sets as the default configuration (only speed may
differ), and the chosen configuration is one that ran."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu


def _run(w, iters, **kw):
    ctx = seg.Context.from_workload(w, **kw)
    ctx.step(iters)
    p = ctx.particles()
    order = np.lexsort((p["c"], p["idx"]))
    out = (ctx.labels().copy(), ctx.stats(), p["idx"][order], p["c"][order], ctx.get_state())
    ctx.close()
    return out


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    assert a[4] == b[4]


@pytest.mark.parametrize("make", [
    lambda: synth.disks(160, 224, seed=3),
    lambda: synth.ellipses(192, 256, seed=4),
    lambda: synth.ellipsoids(40, 48, 64, seed=5),
])
def test_autotune_candidates_agree(make):
    w = make()
    if w.image.ndim == 3:
        w.labels0 = synth.cube_grid_labels(*w.image.shape, 16, 8)
    args = dict(model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff, ps_radius=w.ps_radius)
    best, table = seg.autotune(w.image, w.labels0, iters=3, **args)
    ran = [t for t in table if t[3] == 0]
    assert ran, table
    assert (best["cell_edge"], best["tile"]) in {(t[0], t[1]) for t in ran}
    assert min(t[2] for t in ran) == [t[2] for t in ran if (t[0], t[1]) == (best["cell_edge"], best["tile"])][0]
    ref = _run(w, 8)
    for cell, tile, ms, st in ran:
        _same(_run(w, 8, cell_edge=cell, tile=tile), ref)
