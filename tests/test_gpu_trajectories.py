"""Whole trajectories of the standard workloads against the oracle.

- 1024^2 piecewise smooth: all 200 iterations from the initial labels, every iteration
  compared element by element (particles, dE and g within the float contract, FP64
  recomputes, labels bit for bit).
- 256^3 uint16 piecewise constant: the first 30 iterations from the initial labels, compared
  the same way.
- The 512-image batch in the batch benchmark's launch configuration (batch-tuned cell edge
  and tile): all 512 jobs for all 50 iterations, stepped together; every job's status counts
  and label image (by digest) after every iteration, and its final statistics, against the
  oracle's run of that job.
- The served stream: jobs that overlap in the continuous-batching server; a sample of 16
  distinct jobs of every kind against the oracle (final labels bit for bit and the
  particle-iterations of the whole run).
"""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step
from oracle_pool import labels_digest, run_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield
    torch.cuda.synchronize()


def _whole(w, iterations, label):
    ctx = seg.Context.from_workload(w)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
    run = oracle.Run(p, w.image, w.labels0)
    most_fixed = 0
    for it in range(iterations):
        st, stats = compare_step(ctx, run, f"{label} it{it}")
        most_fixed = max(most_fixed, st["n_fixup"])
    n, S, Q = ctx.stats()
    n_ref, S_ref, Q_ref = oracle.stats(p, w.image, run.L)
    assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref)
    ctx.close()
    return most_fixed


def test_ellipses1024_all_200_iterations():
    w = synth.ellipses()
    assert w.iterations == 200
    _whole(w, 200, "ellipses1024")


def test_ellipsoids256_first_30_iterations():
    w = synth.ellipsoids()
    _whole(w, 30, "ellipsoids256")


def test_batch512_every_job_every_iteration():
    from paper_1403_0240_gb300 import tune
    iters = 50
    jobs = synth.batch_disks(512, seed0=1000, iterations=iters)
    # oracle trajectories first (worker processes), largest images first
    order = sorted(range(512), key=lambda i: -jobs[i].image.size)
    res = run_all([("batch", i, 1000) for i in order], iters)
    ref = {i: r for i, r in zip(order, res)}
    best, _ = tune.autotune_batch([(w.image, w.labels0, dict(model=w.model, lam=w.lam, cutoff=w.cutoff))
                                   for w in jobs], iters=3, sample=128)
    settings = {"tile": best["tile"]}
    ctxs = [seg.Context(w.image, w.labels0, model=w.model, lam=w.lam, cutoff=w.cutoff,
                        cell_edge=best["cell_multiple"] * int(np.ceil(w.cutoff)), **settings) for w in jobs]
    batch = seg.Batch()
    for c in ctxs:
        batch.add(c)
    for t in range(iters):
        sts = batch.step(1)
        for i, (c, st) in enumerate(zip(ctxs, sts)):
            n_p, n_c, n_a, mode, conv, dig = ref[i][0][t]
            assert (st["n_particles"], st["n_candidates"], st["n_accepted"], st["mode_used"], st["converged"]) == \
                (n_p, n_c, n_a, mode, conv), (i, t, st, ref[i][0][t])
            assert labels_digest(c.labels()) == dig, (i, t)
    for i, c in enumerate(ctxs):
        _, n_ref, S_ref, Q_ref = ref[i]
        n, S, Q = c.stats()
        assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref), i
    batch.close()
    for c in ctxs:
        c.close()


def test_served_sample_matches_oracle():
    import torch
    from paper_1403_0240_gb300.serve import Request, SegBackend, Server
    iters = 100
    arrivals = synth.arrival_stream(64, seed=42)
    keys = [synth.served_job_key(a) for a in arrivals]
    cache = {k: synth.served_job(k, iters) for k in set(keys)}
    reqs = []
    for i, (a, k) in enumerate(zip(arrivals, keys)):
        w = cache[k]
        reqs.append(Request(i, a.t, w.image, w.labels0, iters,
                            dict(model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                                 ps_radius=w.ps_radius), nlabels=int(w.labels0.max()) + 1))
    dev = torch.device("cuda", 0)
    be = SegBackend(stream=torch.cuda.current_stream(dev), init_stream=torch.cuda.Stream(dev), keep_labels=True)
    free, _ = torch.cuda.mem_get_info(dev)
    srv = Server(be, int(0.5 * free), max_jobs=512, max_iters_per_step=4)
    res = srv.run(reqs)
    be.close()
    assert len(res) == len(reqs)
    overlapped = sum(1 for r in res for q in res if q is not r and q.admitted < r.completed and r.admitted < q.completed)
    assert overlapped > 0, "the jobs of the stream should share the GPU"
    # 16 distinct jobs of every kind whose oracle runs are bounded (3D sides up to 128)
    first = {}
    for r, k in zip(sorted(res, key=lambda r: r.job_id), keys):
        if k not in first and (k[0] != "pc3d" or k[1] <= 128):
            first[k] = r
    pick = sorted(first, key=lambda k: (k[0], k[1]))
    by_kind = {kind: [k for k in pick if k[0] == kind] for kind in ("pc2d", "ps2d", "pc3d")}
    sample = by_kind["pc3d"][:4] + by_kind["ps2d"][-6:] + by_kind["pc2d"][-6:]
    assert len({k[0] for k in sample}) == 3 and len(sample) >= 12
    specs = sorted(sample, key=lambda k: -cache[k].image.size)
    out = run_all([("served", k, iters) for k in specs], iters)
    for k, (traj, n_ref, S_ref, Q_ref) in zip(specs, out):
        r = first[k]
        assert labels_digest(r.labels) == traj[-1][5], k
        assert r.particles == sum(t[0] for t in traj), k
