"""Full-size workloads: after some GPU iterations, one whole iteration is compared with the
oracle started from the same labels (Sobolev mode throughout, so the optimiser state is the
same): every particle, every gradient within its bound, and the labels bit for bit."""
import time

import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import REL_TOL, scaled_err

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
    assert scaled_err(g["dE"], dump["dE"], dump["dE_scale"]) <= REL_TOL
    assert scaled_err(g["g"], dump["g"], dump["g_scale"]) <= REL_TOL
    assert np.array_equal(ctx.labels(), run.L)
    ctx.close()
    return st, t_oracle


def test_ellipses_1024_one_iteration_after_20():
    st, t = _one_iteration_parity(synth.ellipses(), 20)
    assert st["n_particles"] > 50000


def test_ellipsoids_256_one_iteration_after_5():
    st, t = _one_iteration_parity(synth.ellipsoids(), 5)
    assert st["n_particles"] > 1000000


def test_ellipsoids_256_many_recomputes():
    # around iteration 25 thousands of particles are queued for the FP64 recompute (more than
    # the recompute grid's blocks), so it runs one particle per warp instead of per block
    st, t = _one_iteration_parity(synth.ellipsoids(), 24)
    assert st["n_fixup"] > 8 * 152


def test_batch512_sampled_jobs_match_oracle():
    """The 512-image batch (sides 64-512, 1-8 disks) stepped together with the batch-tuned
    settings, as the batch benchmark runs it; eight jobs spread over the batch are replayed by
    the oracle and must end with the same labels and statistics."""
    from paper_1403_0240_gb300 import tune
    jobs = synth.batch_disks(512, seed0=1000, iterations=8)
    best, _ = tune.autotune_batch([(w.image, w.labels0, dict(model=w.model, lam=w.lam, cutoff=w.cutoff))
                                   for w in jobs], iters=2, sample=64)
    settings = lambda w: {"cell_edge": best["cell_multiple"] * int(np.ceil(w.cutoff)), "tile": best["tile"]}
    ctxs = [seg.Context(w.image, w.labels0, model=w.model, lam=w.lam, cutoff=w.cutoff, **settings(w)) for w in jobs]
    batch = seg.Batch()
    for c in ctxs:
        batch.add(c)
    sts = batch.step(8)
    assert all(s["error"] == 0 for s in sts)
    for i in np.linspace(0, 511, 8).astype(int):
        w = jobs[i]
        p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
        run = oracle.Run(p, w.image, w.labels0)
        for _ in range(8):
            run.step()
        assert np.array_equal(ctxs[i].labels(), run.L), i
        n, S, Q = ctxs[i].stats()
        n_ref, S_ref, Q_ref = oracle.stats(p, w.image, run.L)
        assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref), i
    batch.close()
    for c in ctxs:
        c.close()


def test_large_2d_image_two_iterations():
    """A 4096 x 4096 image (16.8 M pixels, about 9000 tiles, a sparse contour): one iteration on
    the GPU, then one whole iteration compared with the oracle."""
    w = synth.disks(4096, 4096, seed=41, n_disks=40)
    st, t = _one_iteration_parity(w, 1)
    assert st["n_particles"] > 1000
