"""Region-sum precision modes: FP64 sums and compensated FP32 sums against the exact sums of
the same labels, after several iterations of moves (every move updates two regions' sums). The
errors are measured against each label's sum of magnitudes (the condition-aware scale), and the
labels are compared with the exact-mode run."""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu

# |S - S_exact| / sum|I| and |Q - Q_exact| / sum I^2 after the run
TOL = {"f64": 1e-12, "kahan32": 1e-7}


def _case(name):
    if name == "disks":
        w = synth.disks(160, 144, seed=31)
        w.labels0 = synth.square_grid_labels(160, 144, 32, 16)
        return w
    w = synth.ellipsoids(20, 24, 22, seed=32)
    w.labels0 = synth.cube_grid_labels(20, 24, 22, 10, 5)
    return w


@pytest.mark.parametrize("mode", ["f64", "kahan32"])
@pytest.mark.parametrize("case", ["disks", "u16_3d"])
def test_inexact_sums_track_the_exact_ones(mode, case):
    w = _case(case)
    ctx = seg.Context.from_workload(w, stats=mode)
    ref = seg.Context.from_workload(w)
    moved = 0
    for _ in range(15):
        moved += ctx.step(1)["n_accepted"]
        ref.step(1)
    assert moved > 0
    L = ctx.labels()
    n, S, Q = ctx.stats()
    p = oracle.make_params(w.image, L, w.model, w.connectivity, w.lam, w.cutoff, nlabels=ctx.nlabels)
    ne, Se, Qe = oracle.stats(p, w.image, L)
    assert np.array_equal(n, ne)
    v = w.image.astype(np.float64).reshape(-1)
    absS = np.bincount(L.reshape(-1), weights=np.abs(v), minlength=ctx.nlabels)
    sumQ = np.bincount(L.reshape(-1), weights=v * v, minlength=ctx.nlabels)
    m = n > 0
    errS = float((np.abs(S - Se)[m] / np.maximum(absS[m], 1e-300)).max())
    errQ = float((np.abs(Q - Qe)[m] / np.maximum(sumQ[m], 1e-300)).max())
    assert errS <= TOL[mode] and errQ <= TOL[mode], (errS, errQ)
    if w.image.dtype == np.uint16 and mode == "f64":
        assert np.array_equal(S, Se) and np.array_equal(Q, Qe)     # integer sums below 2^53: exact
    # the means differ from the exact ones only in their last bits: the runs agree almost everywhere
    diff = int((L != ref.labels()).sum())
    assert diff <= 1e-3 * L.size, diff
    ctx.close()
    ref.close()


def test_stats_mode_is_checked():
    w = _case("disks")
    with pytest.raises(seg.SegError) as e:
        seg.Context.from_workload(w, stats=3)
    assert e.value.code == seg.SEG_EINVAL
