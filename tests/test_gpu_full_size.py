"""Full-size workloads: after some GPU iterations, one whole iteration is compared with the
oracle started from the same labels (Sobolev mode throughout, so the optimiser state is the
same): every particle, every gradient within its bound and the float contract, and the labels
bit for bit. These reach states far into a run (many FP64 recomputes, a 4096^2 image) that the
whole-trajectory tests do not."""
import time

import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import check_floats, record

pytestmark = pytest.mark.gpu


def _one_iteration_parity(w, warm_iters):
    ctx = seg.Context.from_workload(w)
    st = ctx.step(warm_iters)
    assert st["error"] == 0
    L_t = ctx.labels().copy()
    n, S, Q = ctx.stats()
    p = oracle.make_params(w.image, L_t, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius,
                           nlabels=int(w.labels0.max()) + 1)
    n_ref, S_ref, Q_ref = oracle.stats(p, w.image, L_t)
    assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref)
    run = oracle.Run(p, w.image, L_t)
    t0 = time.time()
    ref, dump = run.step(dump=True)
    t_oracle = time.time() - t0
    st = ctx.step(1)
    for k in ("n_particles", "n_candidates", "n_accepted"):
        assert st[k] == ref[k], (k, st, ref)
    got = ctx.particles()
    order = np.lexsort((got["c"], got["idx"]))
    g = {k: v[order] for k, v in got.items()}
    assert np.array_equal(g["idx"], dump["idx"]) and np.array_equal(g["c"], dump["c"])
    assert (np.abs(g["dE"].astype(np.float64) - dump["dE"]) <= g["eE"]).all()
    assert (np.abs(g["g"].astype(np.float64) - dump["g"]) <= g["eg"]).all()
    fixed = (g["flags"] & 1) != 0
    assert np.array_equal(g["key"][fixed], dump["g"][fixed])
    errs = check_floats(g["dE"], g["g"], dump, f"{w.name} after {warm_iters}")
    errs["n"] = int(g["idx"].size)
    record(f"{w.name}_{w.image.shape[-1]} after {warm_iters}", errs)
    assert np.array_equal(ctx.labels(), run.L)
    ctx.close()
    return st, t_oracle


def test_large_2d_image_two_iterations():
    """A 4096 x 4096 image (16.8 M pixels, about 9000 tiles, a sparse contour): one iteration on
    the GPU, then one whole iteration compared with the oracle."""
    w = synth.disks(4096, 4096, seed=41, n_disks=40)
    st, t = _one_iteration_parity(w, 1)
    assert st["n_particles"] > 1000
