"""Oracle runs in worker processes, for the whole-trajectory GPU tests.

The pool is started with the spawn method (the test process has a CUDA context, and a
process forked from it would hang). A worker rebuilds its job from the seeded input
generators, iterates the oracle and returns, per iteration, the status counts and a digest
of the label image, then the final statistics."""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np


def labels_digest(L) -> str:
    return hashlib.sha256(np.ascontiguousarray(L, np.int32).tobytes()).hexdigest()


def build(spec):
    from paper_1403_0240_gb300 import synth
    kind = spec[0]
    if kind == "batch":
        return synth.batch_disk(spec[1], seed0=spec[2])
    if kind == "served":
        return synth.served_job(spec[1], iterations=spec[2])
    raise ValueError(spec)


def trajectory(spec, iterations: int):
    """(per-iteration [(n_particles, n_candidates, n_accepted, mode_used, converged, digest)],
    final n, S, Q) of the oracle on the job `spec`."""
    import oracle
    w = build(spec)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius,
                           psf=getattr(w, "psf", None))
    run = oracle.Run(p, w.image, w.labels0)
    out = []
    for _ in range(iterations):
        s, _ = run.step()
        out.append((s["n_particles"], s["n_candidates"], s["n_accepted"], s["mode_used"], s["converged"],
                    labels_digest(run.L)))
    n, S, Q = oracle.stats(p, w.image, run.L)
    return out, n, S, Q


def _job(args):
    return trajectory(*args)


def pool():
    procs = max(1, min(len(os.sched_getaffinity(0)), 32))
    return mp.get_context("spawn").Pool(processes=procs)


def run_all(specs, iterations):
    """Trajectories of all jobs, in the order of specs (the largest jobs should come first)."""
    with pool() as p:
        return p.map(_job, [(s, iterations) for s in specs], chunksize=1)
