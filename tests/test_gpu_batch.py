"""Batched stepping: each job of a batch gives exactly what it gives alone.

A batch runs one launch per stage for all of its jobs; jobs never share data, so labels,
statistics and every particle array must be identical (bit for bit) to a solo run of the
same job. Jobs joining and leaving between steps (continuous batching) must not change
anything either."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu


def _jobs():
    a = synth.disks(128, 128, seed=0)
    b = synth.disks(97, 151, seed=5)
    b.labels0 = synth.square_grid_labels(97, 151, 32, 12)
    c = synth.ellipses(160, 192, seed=7)
    c.labels0 = synth.square_grid_labels(160, 192, 32, 16)
    d = synth.ellipsoids(24, 28, 32, seed=8)
    d.labels0 = synth.cube_grid_labels(24, 28, 32, 12, 6)
    e = synth.disks(5, 3, seed=9)
    e.labels0 = np.zeros((5, 3), np.int32)
    e.labels0[1:3, 1] = 1
    f = synth.ellipsoids(16, 16, 16, seed=10)
    g = synth.deconv_scene(72, 88, seed=12, sigma=2.5)
    return [a, b, c, d, e, f, g]


def _solo(w, iters):
    ctx = seg.Context.from_workload(w)
    for _ in range(iters):
        ctx.step(1)
    out = {"labels": ctx.labels().copy(), "stats": ctx.stats(), "particles": ctx.particles(),
           "state": ctx.get_state()}
    ctx.close()
    return out


def _sorted(p):
    # tiles take their ranges of the particle arrays in completion order: compare in key order
    order = np.lexsort((p["c"], p["idx"]))
    return {k: v[order] for k, v in p.items()}


def _same(got_ctx, ref):
    assert np.array_equal(got_ctx.labels(), ref["labels"])
    n, S, Q = got_ctx.stats()
    assert np.array_equal(n, ref["stats"][0]) and np.array_equal(S, ref["stats"][1])
    p, r = _sorted(got_ctx.particles()), _sorted(ref["particles"])
    for k in ("idx", "l", "c", "dE", "eE", "g", "eg", "key", "flags"):
        assert np.array_equal(p[k], r[k]), k
    assert got_ctx.get_state() == ref["state"]


def test_batch_equals_solo():
    jobs = _jobs()
    iters = 12
    refs = [_solo(w, iters) for w in jobs]
    batch = seg.Batch()
    ctxs = [seg.Context.from_workload(w) for w in jobs]
    for c in ctxs:
        batch.add(c)
    for _ in range(iters):
        sts = batch.step(1)
        assert all(s["error"] == 0 for s in sts)
    for c, r in zip(ctxs, refs):
        _same(c, r)
    batch.close()
    for c in ctxs:
        c.close()


def test_continuous_batching_equals_solo():
    jobs = _jobs()
    refs = {i: _solo(w, 10) for i, w in enumerate(jobs)}
    batch = seg.Batch()
    ctxs = {}
    done = {}
    pending = list(range(len(jobs)))
    step = 0
    # admit two jobs at a time, remove a job once it has run 10 iterations
    while pending or ctxs:
        while pending and len(ctxs) < 3:
            i = pending.pop(0)
            ctxs[i] = seg.Context.from_workload(jobs[i])
            batch.add(ctxs[i])
        batch.step(1)
        step += 1
        for i in list(ctxs):
            if ctxs[i].get_state()["t"] == 10:
                batch.remove(ctxs[i])
                _same(ctxs[i], refs[i])
                ctxs[i].close()
                done[i] = True
                del ctxs[i]
    assert len(done) == len(jobs)
    batch.close()


def test_batch_rejects_double_membership():
    w = _jobs()[0]
    c = seg.Context.from_workload(w)
    b1, b2 = seg.Batch(), seg.Batch()
    b1.add(c)
    with pytest.raises(seg.SegError):
        b2.add(c)
    with pytest.raises(seg.SegError):
        c.step(1)                         # a context in a batch is stepped by its batch
    b1.remove(c)
    c.step(1)
    b1.close()
    b2.close()
    c.close()


def test_served_jobs_equal_solo():
    from paper_1403_0240_gb300.serve import Request, SegBackend, Server
    jobs = _jobs()
    iters = [8, 12, 10, 6, 9, 11, 7]
    refs = [_solo(w, n) for w, n in zip(jobs, iters)]

    def params(w):
        return dict(model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff, ps_radius=w.ps_radius,
                    psf=w.psf)

    backend = SegBackend()
    reqs = [Request(i, 0.0, w.image, w.labels0, n, params(w)) for i, (w, n) in enumerate(zip(jobs, iters))]
    biggest = max(backend.estimate(r) for r in reqs)
    srv = Server(backend, budget_bytes=int(2.5 * biggest), max_jobs=4, max_iters_per_step=3)
    for r in reqs:
        srv.submit(r)
    while not srv.idle():
        srv.step()
    assert len(srv.results) == len(jobs)
    for r in srv.results:
        assert r.iterations == iters[r.job_id]
        assert np.array_equal(r.labels, refs[r.job_id]["labels"])
    backend.close()


def test_batch_of_large_images_equals_solo():
    # four 1024^2 images: the batch's candidate count per iteration spans the ranges where the
    # selection rounds run in one block with and without their shared-memory neighbour rows,
    # and (above 32768 candidates) on the whole grid
    jobs = [synth.ellipses(seed=s) for s in range(1, 5)]
    iters = 8
    refs = [_solo(w, iters) for w in jobs]
    batch = seg.Batch()
    ctxs = [seg.Context.from_workload(w) for w in jobs]
    for c in ctxs:
        batch.add(c)
    cands = []
    for _ in range(iters):
        sts = batch.step(1)
        cands.append(sum(s["n_candidates"] for s in sts))
    assert max(cands) > 20000
    for c, r in zip(ctxs, refs):
        assert np.array_equal(c.labels(), r["labels"])
        assert c.get_state() == r["state"]
    batch.close()
    for c in ctxs:
        c.close()
