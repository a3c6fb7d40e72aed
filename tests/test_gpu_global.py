"""Eq. 6 with the length scale set to the contour length, E = |Gamma| (all particle pairs),
against the oracle iteration by iteration: particle sets, gradients within their bounds and
1e-5 of the oracle's scale, FP64-recomputed keys bit for bit, labels bit for bit."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step, pair

pytestmark = pytest.mark.gpu


def test_global_length_scale_disks_128():
    w = synth.disks()
    ctx, run = pair(w, gradient="sobolev_global")
    fixed = 0
    for it in range(25):
        st, stats = compare_step(ctx, run, f"global disks it{it}")
        assert st["mode_used"] == seg.SEG_SOBOLEV_GLOBAL
        fixed += stats.get("fixed", 0)
    ctx.close()


@pytest.mark.parametrize("seed", [21, 22])
def test_global_uneven_with_switch_to_l2(seed):
    w = synth.disks(71, 90, seed=seed)
    ctx, run = pair(w, gradient="sobolev_global", osc_window=3)
    modes = []
    for it in range(30):
        st, _ = compare_step(ctx, run, f"global uneven{seed} it{it}")
        modes.append(st["mode_used"])
    assert modes[0] == seg.SEG_SOBOLEV_GLOBAL and seg.SEG_L2 in modes
    ctx.close()


def test_global_3d():
    w = synth.ellipsoids(20, 24, 28, seed=4)
    w.labels0 = synth.cube_grid_labels(20, 24, 28, 12, 6)
    ctx, run = pair(w, gradient="sobolev_global")
    for it in range(8):
        compare_step(ctx, run, f"global 3d it{it}")
    ctx.close()


def test_global_job_in_a_batch_equals_solo():
    a = synth.disks(96, 112, seed=31)
    b = synth.disks(80, 64, seed=32)
    solo = []
    for w, grad in ((a, "sobolev_global"), (b, "sobolev")):
        c = seg.Context.from_workload(w, gradient=grad)
        c.step(10)
        solo.append(c.labels().copy())
        c.close()
    ca = seg.Context.from_workload(a, gradient="sobolev_global")
    cb = seg.Context.from_workload(b, gradient="sobolev")
    batch = seg.Batch()
    batch.add(ca)
    batch.add(cb)
    batch.step(10)
    assert np.array_equal(ca.labels(), solo[0]) and np.array_equal(cb.labels(), solo[1])
    batch.close()
    ca.close()
    cb.close()
