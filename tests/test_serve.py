"""Scheduling of the continuous-batching server, with a fake device backend (no GPU)."""
import numpy as np
import pytest

from paper_1403_0240_gb300.serve import Request, Server, latency_summary


class FakeCtx:
    def __init__(self, req):
        self.req = req
        self.t = 0
        self.parts = 0
        self.in_batch = False
        self.closed = False


class FakeBackend:
    """Each context gains `rate` particles per iteration and converges at `converge_at`."""

    def __init__(self, clock):
        self.members = []
        self.clock = clock
        self.steps = []

    def estimate(self, req):
        return req.params["bytes"]

    def create(self, req):
        return FakeCtx(req)

    def add(self, ctx):
        assert not ctx.in_batch
        ctx.in_batch = True
        self.members.append(ctx)

    def remove(self, ctx):
        assert ctx.in_batch
        ctx.in_batch = False
        self.members.remove(ctx)

    def step_async(self, k):
        self.steps.append((k, len(self.members)))
        for c in self.members:
            for _ in range(k):
                if c.t >= c.req.params.get("converge_at", 10 ** 9):
                    break
                c.t += 1
                c.parts += c.req.params["rate"]
        self.clock.advance(0.001 * k)

    def poll(self):
        return [{"particles_total": c.parts, "converged": int(c.t >= c.req.params.get("converge_at", 10 ** 9))}
                for c in self.members]

    def finish(self, ctx):
        ctx.closed = True
        return np.full((2, 2), ctx.req.job_id, np.int32)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-6
        return self.t

    def advance(self, dt):
        self.t += dt


def _req(i, arrival=0.0, iters=10, nbytes=100, rate=7, **extra):
    return Request(i, arrival, np.zeros((2, 2), np.float32), np.zeros((2, 2), np.int32), iters,
                   dict(bytes=nbytes, rate=rate, **extra))


def test_budget_and_fifo_and_iterations():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, budget_bytes=350, max_jobs=10, max_iters_per_step=3, clock=clock)
    for i in range(8):
        srv.submit(_req(i, iters=5 + i, nbytes=100 + 10 * i))
    admitted_order = []
    while not srv.idle():
        srv.step()
        assert srv.used <= 350
        for jid in srv.order:
            if jid not in admitted_order:
                admitted_order.append(jid)
    assert admitted_order == sorted(admitted_order)           # first come, first served
    res = {r.job_id: r for r in srv.results}
    assert sorted(res) == list(range(8))
    for i, r in res.items():
        assert r.iterations == 5 + i and r.particles == 7 * (5 + i)
        assert r.completed >= r.admitted >= r.arrival
        assert (r.labels == i).all()


def test_slot_limit_and_early_convergence():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, budget_bytes=10 ** 9, max_jobs=2, max_iters_per_step=4, clock=clock)
    for i in range(5):
        srv.submit(_req(i, iters=20, converge_at=6 if i % 2 else 10 ** 9))
    while not srv.idle():
        srv.step()
        assert len(srv.resident) <= 2
    res = {r.job_id: r for r in srv.results}
    for i, r in res.items():
        if i % 2:
            assert r.converged and r.particles == 7 * 6
        else:
            assert not r.converged and r.iterations == 20
    assert all(n <= 2 for _, n in be.steps)


def test_job_larger_than_budget_is_refused():
    clock = FakeClock()
    srv = Server(FakeBackend(clock), budget_bytes=50, clock=clock)
    srv.submit(_req(0, nbytes=51))
    with pytest.raises(ValueError):
        srv.step()


def test_real_time_replay_and_latency_summary():
    clock = FakeClock()
    srv = Server(FakeBackend(clock), budget_bytes=10 ** 6, max_jobs=8, max_iters_per_step=2, clock=clock)
    reqs = [_req(i, arrival=0.002 * i, iters=6) for i in range(20)]
    res = srv.run(reqs)
    assert len(res) == 20
    s = latency_summary(res)
    assert 0.0 < s["p50_s"] <= s["p99_s"]


def test_request_options_reach_the_library_parameters():
    # every option a request may carry ends up in seg_params (topology events, curvature
    # regulariser, statistics mode), and the device-memory estimate sees the split capacity
    import ctypes as C
    from paper_1403_0240_gb300 import seg
    from paper_1403_0240_gb300.serve import Request, _param_kwargs
    img = np.zeros((64, 48), np.float32)
    req = Request(0, 0.0, img, np.zeros(img.shape, np.int32), 10,
                  params={"model": "pc", "lam": 0.5, "cutoff": 3.0, "stats": "exact", "topology": "vanish+split+fuse",
                          "max_labels": 64, "curv_radius": 4.0, "psf": None})
    p = seg.make_params(img, **_param_kwargs(req, with_psf=False))
    assert p.topology == 7 and p.max_labels == 64
    assert p.regulariser == seg.SEG_REG_CURVATURE and p.curv_radius == 4.0
    assert p.stats_mode == seg.STATS_MODES["exact"]
    out = C.c_size_t(0)
    assert seg.lib().seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_OK
    big = out.value
    p.topology = 0
    assert seg.lib().seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_OK and out.value < big
