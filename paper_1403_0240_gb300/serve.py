"""Continuous-batching segmentation server on one GPU.

Requests arrive with an image, initial labels, parameters and an iteration count. The
server admits a request when its estimated device memory fits the budget and a batch slot
is free, keeps every admitted job's labels, particles and statistics resident on the
device, and steps all resident jobs together (one launch per stage for all of them). A job
leaves the batch when it has run its iterations or converged; its labels are copied to the
host and its latency (completion time minus arrival time) recorded. Initialising a newly
admitted job (host checks, host-to-device copies) overlaps the batch step in flight.

The device work goes through a backend (``SegBackend`` wraps libseg); tests can substitute
a fake backend to check the scheduling on the CPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    job_id: int
    arrival: float                 # seconds, on the server's clock
    image: np.ndarray
    labels0: np.ndarray
    iterations: int
    params: dict = field(default_factory=dict)   # model, connectivity, lam, cutoff, ps_radius, psf, ...
    nlabels: int | None = None     # largest initial label + 1 (found from labels0 when None)


@dataclass
class Result:
    job_id: int
    arrival: float
    admitted: float
    completed: float
    iterations: int
    particles: int                 # particle-iterations processed for this job
    converged: bool
    labels: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


class SegBackend:
    """libseg on the current CUDA device: contexts in one batch. New contexts are set up on
    their own stream (init_stream) so that this overlaps the batch step in flight."""

    def __init__(self, stream=None, init_stream=None, keep_labels: bool = True, time_steps: bool = False):
        from . import seg
        self.seg = seg
        self.stream = stream
        self.init_stream = init_stream
        self.batch = seg.Batch(stream=stream)
        self.keep_labels = keep_labels
        # CUDA events around every batch step on the batch stream (device time of the step)
        self.time_steps = time_steps and stream is not None
        self._ev = None
        self.last_step_ms = None

    def launches(self) -> int:
        """Kernels libseg has launched in this process so far."""
        return self.seg.kernel_launches()

    def estimate(self, req: Request) -> int:
        if req.nlabels is None:
            req.nlabels = int(req.labels0.max()) + 1
        p = self.seg.make_params(req.image, **_param_kwargs(req, with_psf=False))
        return self.seg.estimate_bytes(p, req.nlabels)

    def create(self, req: Request):
        return self.seg.Context(req.image, req.labels0, stream=self.init_stream, **_param_kwargs(req))

    def add(self, ctx):
        self.batch.add(ctx)

    def remove(self, ctx):
        self.batch.remove(ctx)

    def step_async(self, iters: int):
        if self.time_steps:
            import torch
            self._ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            self._ev[0].record(self.stream)
        self.batch.step_async(iters)
        if self._ev is not None:
            self._ev[1].record(self.stream)

    def poll(self) -> list[dict]:
        out = self.batch.poll()
        if self._ev is not None:
            self.last_step_ms = self._ev[0].elapsed_time(self._ev[1])
            self._ev = None
        return out

    def finish(self, ctx):
        labels = ctx.labels() if self.keep_labels else None
        ctx.close()
        return labels

    def close(self):
        self.batch.close()


def _param_kwargs(req: Request, with_psf: bool = True) -> dict:
    keys = ("model", "connectivity", "lam", "cutoff", "ps_radius", "gradient", "osc_window", "cell_edge", "tile",
            "stats", "topology", "max_labels", "curv_radius")
    out = {k: req.params[k] for k in keys if k in req.params}
    if with_psf and req.params.get("psf") is not None:
        out["psf"] = req.params["psf"]          # deconvolving model: set after seg_init
    return out


class Server:
    def __init__(self, backend, budget_bytes: int, max_jobs: int = 512, max_iters_per_step: int = 4,
                 clock=time.perf_counter):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_jobs = int(max_jobs)
        self.max_iters = int(max_iters_per_step)
        self.clock = clock
        self.queue: deque[Request] = deque()
        self.resident: dict[int, dict] = {}      # job_id -> {req, ctx, bytes, admitted, done}
        self.order: list[int] = []               # batch member order (matches poll())
        self.used = 0
        self.results: list[Result] = []
        self.steps = 0
        # host seconds spent per phase of step(): setting up admitted jobs, waiting for the batch
        # step to finish, retiring finished jobs (label read-back), adding joined jobs
        self.timing = {"admit_s": 0.0, "wait_s": 0.0, "retire_s": 0.0, "join_s": 0.0, "member_steps": 0}
        # one entry per batch step: start and end (server clock), iterations, members, jobs
        # waiting in the queue when it started, particle-iterations it processed, and the
        # device time of the step when the backend measures it
        self.log: list[dict] = []

    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self) -> list[int]:
        """Set up the queued jobs that fit (memory and slots); they join the batch later."""
        joined = []
        while self.queue and len(self.resident) < self.max_jobs:
            req = self.queue[0]
            need = self.backend.estimate(req)
            if need > self.budget:
                raise ValueError(f"job {req.job_id} needs {need} bytes, more than the whole budget {self.budget}")
            if self.used + need > self.budget:
                break                             # first-come first-served: wait for memory
            self.queue.popleft()
            ctx = self.backend.create(req)
            self.used += need
            self.resident[req.job_id] = {"req": req, "ctx": ctx, "bytes": need, "admitted": self.clock(),
                                         "done": 0, "particles": 0, "converged": False}
            joined.append(req.job_id)
        return joined

    def _iters_for(self, members) -> int:
        left = [self.resident[j]["req"].iterations - self.resident[j]["done"] for j in members]
        return max(1, min(self.max_iters, min(left))) if left else 0

    def step(self) -> int:
        """Run one batch step while admitting what fits, then retire finished jobs and let
        the admitted ones join; returns the iterations run (0 when nothing was resident)."""
        members = list(self.order)
        k = self._iters_for(members)
        queued = len(self.queue)
        count = getattr(self.backend, "launches", None)
        l0 = count() if count else None
        t0 = self.clock()
        if k:
            self.backend.step_async(k)
        joined = self._admit()                    # host work overlaps the step in flight
        t1 = self.clock()
        statuses = self.backend.poll() if k else []
        t2 = self.clock()
        self.timing["admit_s"] += t1 - t0
        self.timing["wait_s"] += t2 - t1
        self.timing["member_steps"] += len(members)
        step_particles = 0
        for jid, st in zip(members, statuses):
            r = self.resident[jid]
            r["done"] += k
            step_particles += int(st["particles_total"]) - r["particles"]
            r["particles"] = int(st["particles_total"])
            r["converged"] = bool(st["converged"])
        now = self.clock()
        for jid in members:
            r = self.resident[jid]
            if r["done"] >= r["req"].iterations or r["converged"]:
                self.backend.remove(r["ctx"])
                labels = self.backend.finish(r["ctx"])
                self.used -= r["bytes"]
                self.order.remove(jid)
                del self.resident[jid]
                self.results.append(Result(jid, r["req"].arrival, r["admitted"], now, r["done"], r["particles"],
                                           r["converged"], labels))
        t3 = self.clock()
        for jid in joined:                        # membership changes only between steps
            self.backend.add(self.resident[jid]["ctx"])
            self.order.append(jid)
        t4 = self.clock()
        self.timing["retire_s"] += t3 - t2
        self.timing["join_s"] += t4 - t3
        if k:
            self.steps += 1
            self.log.append({"t0": t0, "t1": t4, "iters": k, "members": len(members), "queued": queued,
                             "particles": step_particles,
                             "device_ms": getattr(self.backend, "last_step_ms", None),
                             "launches": (count() - l0) if count else None})
        return k

    def idle(self) -> bool:
        return not self.queue and not self.resident

    def run(self, requests: list[Request], t0: float | None = None) -> list[Result]:
        """Replay requests in real time (arrival seconds after t0) until all are served."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        t0 = self.clock() if t0 is None else t0
        while pending or not self.idle():
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                req = pending.popleft()
                req.arrival = t0 + req.arrival
                self.submit(req)
            if self.idle():
                if pending:
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - (self.clock() - t0))))
                continue
            self.step()
        return self.results


def latency_summary(results: list[Result]) -> dict:
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    return {"jobs": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}
