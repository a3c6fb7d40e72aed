"""Kernel launch accounting (seg_kernel_launches) and per-stage timing of a batch."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu

# one iteration of a 2D piecewise-constant job: extraction with the energy differences, Eq. 6 with
# the candidates, neighbour lists with the order certificates, FP64 recompute, selection rounds,
# moves, finish
KERNELS_PER_ITERATION = 7


def test_graph_replays_count_every_kernel():
    w = synth.disks(96, 112, seed=5)
    ctx = seg.Context.from_workload(w)
    ctx.step(1)                                   # set-up and graph capture happen here
    a = seg.kernel_launches()
    ctx.step(1)
    b = seg.kernel_launches()
    ctx.step(4)
    c = seg.kernel_launches()
    one, four = b - a, c - b
    # each step adds its iterations' kernels and a fixed number of status reads
    assert four - one == 3 * KERNELS_PER_ITERATION, (one, four)
    assert 1 <= one - KERNELS_PER_ITERATION <= 2, one
    ctx.close()


def test_batch_stage_times():
    jobs = [synth.disks(80, 90, seed=s) for s in (1, 2, 3)]
    ctxs = [seg.Context.from_workload(w) for w in jobs]
    b = seg.Batch()
    for c in ctxs:
        b.add(c)
    b.step(1)
    b.profile(True)
    b.step(1)
    st = b.stage_times()
    assert set(st) == set(seg.Context.STAGES)
    assert all(v >= 0.0 for v in st.values())
    assert st["extract"] > 0.0 and st["sobolev"] > 0.0 and st["rounds"] > 0.0
    b.profile(False)
    with pytest.raises(seg.SegError):
        b.stage_times()                           # timing is off
    b.close()
    for c in ctxs:
        c.close()
