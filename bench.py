#!/usr/bin/env python
"""Throughput of the particle region-competition iteration with Sobolev gradients.

The metric counts particles processed per second (particle-iterations/s), one iteration of
the whole hot path (extraction, energy differences, Eq. 6 interaction, certified selection,
moves, exact statistics) over every particle of a job.

Default workload (served): a Poisson arrival stream of segmentation jobs (200 jobs/s; 80% 2D
of sides 128-1024, half piecewise-constant disk scenes and half piecewise-smooth ellipse scenes,
20% 3D uint16 ellipsoid volumes of sides 64-256; 100 iterations each) through the continuous-
batching server. A step is one server step (up to --iters-per-step iterations of every resident
job); after the ramp-up, K steps are timed with CUDA events. The same stream is also run one
job at a time (the plain loop), and the line reports both, with p50/p99 job latency and the
arrival rate the server sustains.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Other workloads step one job per iteration (ellipses1024, ellipsoids256, disks128, ...), a
512-image batch (batch512), the region-sum precision study (precision) or the L2/Sobolev
convergence study (convergence).

Under torchrun (N > 1) every rank runs its own independent stream or job (replicas: the
method has no exchange step), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sobolev particle-iterations/s"
UNIT = "particle-iterations/s"
STAGES = ("psf", "extract", "sobolev", "select", "lists", "fixup", "rounds", "moves", "finish")
L2_FLUSH_BYTES = 256 << 20

# Algorithmic bytes per unit (one particle, or one accepted move) of each stage: the
# method's own traffic, band-only (a full-image rescan is implementation overhead).
#   extract = particle write (idx, l, c: 12 B) + amortised label-band reads (8 B)
#           + image value (4 B) + energy difference out (4 B)
#   sobolev = particle in (idx, l, c, dE: 16 B) + gradient out (4 B), plus the candidate
#           selection fused into it (12 B: a particle read per decision stage)
#   select (E = |Gamma| only), lists, fixup, rounds = 12 B per particle (a particle read per
#           decision stage);
#   moves = 24 B per accepted move (label write and statistics); finish = 12 B per particle
ALG_BYTES = {"extract": (28, 0), "sobolev": (32, 0), "fixup": (12, 0),
             "select": (12, 0), "lists": (12, 0), "rounds": (12, 0), "moves": (0, 24), "finish": (12, 0)}


def workloads():
    from paper_1403_0240_gb300 import synth
    return {
        "ellipses1024": (lambda seed: synth.ellipses(seed=1 + seed),
                         "2D 1024x1024 float32 piecewise smooth: 40 ellipses, bias field, Poisson noise (20 photons); "
                         "32x32 squares on a 64 px pitch; local-mean radius 8, cutoff 5, lambda 0.04, 200 iterations"),
        "disks128": (lambda seed: synth.disks(seed=seed) if seed == 0 else synth.disks(128, 128, seed=seed),
                     "2D 128x128 float32 piecewise constant: two disks, Gaussian noise 0.3; centred 64x64 square; "
                     "cutoff 3, lambda 0.04, 50 iterations"),
        "ellipses4096": (lambda seed: synth.ellipses(4096, 4096, seed=1 + seed),
                         "2D 4096x4096 float32 piecewise smooth: the ellipses1024 recipe at 16x the area (640 "
                         "ellipses, same density, bias field and noise); 32x32 squares on a 64 px pitch"),
        "ellipses8192": (lambda seed: synth.ellipses(8192, 8192, seed=1 + seed),
                         "2D 8192x8192 float32 piecewise smooth: the ellipses1024 recipe at 64x the area (2560 "
                         "ellipses); 32x32 squares on a 64 px pitch"),
        "deconv512": (lambda seed: synth.deconv_scene(seed=11 + seed),
                      "2D 512x512 float32, deconvolving piecewise-constant model (Eq. 8): four objects over a faint "
                      "background blurred by a Gaussian PSF sigma 15 px (r = 45, as in Figure 3), Poisson noise (10 "
                      "photons); 64x64 squares on a 128 px pitch; cutoff 5, lambda 0.04, 200 iterations"),
        "ellipsoids256": (lambda seed: synth.ellipsoids(seed=2 + seed),
                          "3D 256^3 uint16 piecewise constant: 200 ellipsoids, blur 1.5, Poisson noise; 16^3 cubes on a "
                          "32 pitch; cutoff 4, lambda 1600, 100 iterations"),
    }


FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64, nominal
# kernels of one iteration's graph: extract, sobolev (with the candidate selection), lists, fixup,
# rounds, moves, finish (plus the deconvolving model's field passes); poll() adds one
KERNELS_PER_ITERATION = 7
# opt-in events and regulariser: kernels each adds to an iteration (the connected-component
# relabelling of splits with its statistics rebuild; the fusion pairs, matching and relabelling;
# the curvature term)
TOPOLOGY_BITS = {"vanish": 1, "split": 2, "fuse": 4}
EXTRA_KERNELS = {"split": 8, "fuse": 3, "curvature": 1}


def topology_code(name: str) -> int:
    """'vanish+split' -> 3; '' -> 0."""
    return sum(TOPOLOGY_BITS[part] for part in name.split("+")) if name else 0


def extra_kernels(args) -> int:
    t = topology_code(args.topology)
    return ((EXTRA_KERNELS["split"] if t & 2 else 0) + (EXTRA_KERNELS["fuse"] if t & 4 else 0) +
            (EXTRA_KERNELS["curvature"] if args.curv_radius > 0 else 0))


def psf_passes(w) -> int:
    """Field passes the deconvolving model adds to an iteration (2D: 3, 3D: 5)."""
    if w.model != "pcd":
        return 0
    return 3 if w.image.ndim == 2 else 5


def psf_pass_flops(w) -> float:
    """FP64 flops (2 per fused multiply-add) of one iteration's field passes: every pixel of
    a pass takes the taps whose offset stays inside the image along the pass's axis."""
    import numpy as np
    r = (w.psf.size - 1) // 2
    shape = w.image.shape
    npix = float(np.prod(shape))

    def taps(n):
        t = np.arange(n)
        return float((np.minimum(r, n - 1 - t) + np.minimum(r, t) + 1).sum())

    per_axis = [taps(n) * npix / n for n in shape[::-1]]       # x, y[, z]
    fmas = per_axis[0] + per_axis[1] + per_axis[0] if len(shape) == 2 else \
        per_axis[0] + per_axis[1] + per_axis[2] + per_axis[0] + per_axis[1]
    return 2.0 * fmas


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_digest(texts) -> str:
    """sha256 (16 hex digits) of C/CUDA sources without their comments and blank lines."""
    h = hashlib.sha256()
    for src in texts:
        text = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code.strip():
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def kernel_sources_digest() -> str:
    """A digest of the profiled kernels' code: the sources without their comments and blank lines, so
    that a change of wording leaves the committed ncu figures valid and a change of code does not."""
    texts = []
    for f in ("k_tile.cu", "k_select.cu", "seg_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1403_0240_gb300", "csrc", f), encoding="utf-8") as fh:
            texts.append(fh.read())
    return _code_digest(texts)


def traffic_from_profile(stage: str, workload: str, units: float):
    """DRAM bytes per launch from the committed ncu summary (bytes per particle of the captured
    launch, scaled to this launch's particles), or None when there is no capture of this stage on
    this workload or the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("sources") != kernel_sources_digest():
        return None
    for e in d.get("entries", []):
        if e.get("stage") == stage and e.get("workload") == workload:
            return float(e["dram_bytes_per_unit"]) * units
    return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.lines: list[str] = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0:
            time.sleep(0.02)
        self.mark = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(", ") for r in self.lines[max(0, getattr(self, "mark", 0) - 1):] if r]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend: str | None = None):
    """One process per GPU (torchrun): NCCL on GPUs, gloo otherwise. Replicas only: the ranks
    exchange nothing but the barrier and the two scalar reductions of the timing."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def _reduce(pg, x: float, op) -> float:
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=op)
    return float(t.item())


def allmax(pg, x: float) -> float:
    return x if pg is None else _reduce(pg, x, pg.ReduceOp.MAX)


def allsum(pg, x: float) -> float:
    return x if pg is None else _reduce(pg, x, pg.ReduceOp.SUM)


def aggregate(pg, units: float, seconds: float) -> tuple[float, float, float]:
    """Whole-job throughput of replicas: the units of all ranks over the slowest rank's time.
    Returns (value, total units, max seconds)."""
    t_max = allmax(pg, seconds)
    total = allsum(pg, units)
    return total / t_max, total, t_max


def oracle_sample(w, seconds: float = 12.0, max_iters: int = 400, topology: int = 0, curv_radius: float = 0.0):
    """The CPU oracle as it stands, single-threaded, on the first iterations of the job."""
    import oracle
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius, psf=w.psf,
                           topology=topology, curv_radius=curv_radius)
    run = oracle.Run(p, w.image, w.labels0)
    t0 = time.perf_counter()
    parts, its = 0, 0
    while its < max_iters and (time.perf_counter() - t0) < seconds:
        s, _ = run.step()
        parts += s["n_particles"]
        its += 1
    dt = time.perf_counter() - t0
    return parts / dt, its, dt


def run_batch(args, world, rank, local, pg):
    """512 uneven 2D images (sides 64-512, 1-8 disks): one batch stepped together, against
    the plain loop that steps each image alone."""
    import torch

    from paper_1403_0240_gb300 import seg, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    jobs = synth.batch_disks(args.images, seed0=1000 + 100000 * rank, iterations=args.steps)
    dev_jobs = [(torch.from_numpy(w.image).to(dev), torch.from_numpy(w.labels0).to(dev), w) for w in jobs]

    # cell edge and tile shape for the batch, tuned by timing candidate settings on a sample of
    # the batch stepped together; both the batch and the per-image loop use the tuned settings
    from paper_1403_0240_gb300 import tune
    tuned, tune_table = {}, []
    if not args.no_tune:
        best, tune_table = tune.autotune_batch(
            [(i, l, dict(model=w.model, lam=w.lam, cutoff=w.cutoff)) for i, l, w in dev_jobs], iters=5,
            sample=128, stream=stream)
        tuned = {"cell_mult": best["cell_multiple"], "tile": best["tile"]}

    def settings(w):
        if not tuned:
            return {}
        return {"cell_edge": tuned["cell_mult"] * max(1, math.ceil(w.cutoff)), "tile": tuned["tile"]}

    def contexts(n=None):
        return [seg.Context(i, l, model=w.model, lam=w.lam, cutoff=w.cutoff, stream=stream, **settings(w))
                for i, l, w in dev_jobs[:n]]

    # warm-up: graph capture and code paths on a few jobs
    warm = contexts(8)
    b = seg.Batch(stream=stream)
    for c in warm:
        b.add(c)
    b.step(args.warmup)
    b.close()
    for c in warm:
        c.step(1)
        c.close()

    plain_ctx = contexts()
    torch.cuda.synchronize(dev)
    barrier(pg)
    t0 = time.perf_counter()
    plain_parts = 0
    for c in plain_ctx:
        plain_parts += c.step(args.steps)["particles_total"]
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    for c in plain_ctx:
        c.close()

    batch_ctx = contexts()
    b = seg.Batch(stream=stream)
    for c in batch_ctx:
        b.add(c)
    b.poll()
    torch.cuda.synchronize(dev)
    barrier(pg)
    t0 = time.perf_counter()
    st = b.step(args.steps)
    torch.cuda.synchronize(dev)
    t_batch = time.perf_counter() - t0
    barrier(pg)
    batch_parts = sum(x["particles_total"] for x in st)
    b.close()
    for c in batch_ctx:
        c.close()
    t_b = allmax(pg, t_batch)
    t_p = allmax(pg, t_plain)
    parts_b = allsum(pg, float(batch_parts))
    parts_p = allsum(pg, float(plain_parts))
    if rank != 0:
        return
    value = parts_b / t_b
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch512", "description": f"{args.images} 2D float32 disk images, sides U{{64..512}}, "
                       "1-8 disks, piecewise constant, cutoff 3, one batch stepped together",
                       "plain_value": parts_p / t_p, "batched_over_plain": (parts_b / t_b) / (parts_p / t_p),
                       "plain_s": t_p, "batched_s": t_b, "images": args.images,
                       "tuned": tuned, "tune_table_s_per_iter": [list(t) for t in tune_table],
                       "timing": "wall clock around whole-batch steps (synchronised)"}}
    print(json.dumps(line), flush=True)


def run_precision(args, world, rank, local, pg):
    """Region-sum precision study on the 512-image batch (50 iterations): the batch stepped with
    exact, FP64 and compensated-FP32 region sums. Per mode: throughput, the largest relative
    error of S, Q and the variance Q/n - mu^2 against the exact sums of the same final labels,
    and the pixels whose final label differs from the exact-mode run."""
    import numpy as np
    import torch

    from paper_1403_0240_gb300 import seg, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    iters = args.steps
    jobs = synth.batch_disks(args.images, seed0=1000 + 100000 * rank, iterations=iters)
    dev_jobs = [(torch.from_numpy(w.image).to(dev), torch.from_numpy(w.labels0).to(dev), w) for w in jobs]

    def run(mode, n=None, steps=iters):
        ctxs = [seg.Context(i, l, model=w.model, lam=w.lam, cutoff=w.cutoff, stream=stream, stats=mode)
                for i, l, w in dev_jobs[:n]]
        b = seg.Batch(stream=stream)
        for c in ctxs:
            b.add(c)
        b.poll()
        torch.cuda.synchronize(dev)
        barrier(pg)
        t0 = time.perf_counter()
        st = b.step(steps)
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        parts = sum(x["particles_total"] for x in st)
        b.close()
        return ctxs, parts, t

    for mode in ("exact", "f64", "kahan32"):            # warm-up: graph capture and code paths
        ctxs, _, _ = run(mode, 8, args.warmup)
        for c in ctxs:
            c.close()
    out, ref_labels = {}, None
    for mode in ("exact", "f64", "kahan32"):
        ctxs, parts, t = run(mode)
        labels = [c.labels() for c in ctxs]
        err = {"S": 0.0, "Q": 0.0, "var": 0.0}
        for c, (img, _, w), L in zip(ctxs, dev_jobs, labels):
            n, S, Q = c.stats()
            ne, Se, Qe = (x.cpu().numpy() for x in seg.region_stats_noalloc(
                img, torch.from_numpy(L).to(dev), c.nlabels, stream=stream))
            assert np.array_equal(n, ne)
            m = n > 0
            for key, a, e in (("S", S, Se), ("Q", Q, Qe)):
                err[key] = max(err[key], float((np.abs(a[m] - e[m]) / np.maximum(np.abs(e[m]), 1e-300)).max()))
            var = Q[m] / n[m] - (S[m] / n[m]) ** 2
            var_e = Qe[m] / n[m] - (Se[m] / n[m]) ** 2
            err["var"] = max(err["var"], float((np.abs(var - var_e) / np.maximum(np.abs(var_e), 1e-300)).max()))
        for c in ctxs:
            c.close()
        if ref_labels is None:
            ref_labels = labels
        diff = sum(int((a != b).sum()) for a, b in zip(labels, ref_labels))
        same = sum(int(np.array_equal(a, b)) for a, b in zip(labels, ref_labels))
        parts_all, t_all = allsum(pg, float(parts)), allmax(pg, t)
        out[mode] = {"value": parts_all / t_all, "seconds": t_all, "max_rel_err_S": err["S"],
                     "max_rel_err_Q": err["Q"], "max_rel_err_variance": err["var"],
                     "label_pixels_differing_from_exact": diff, "jobs_with_labels_equal_to_exact": same}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": out["exact"]["value"], "unit": UNIT, "n_gpus": world, "steps": iters,
            "warmup": args.warmup, "ms_per_step": 1000 * out["exact"]["seconds"] / iters, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "precision", "description": f"{args.images} 2D float32 disk images (the batch512 "
                       "set), one batch stepped together per region-sum mode; errors against the exact sums of "
                       "each run's final labels", "images": args.images, "modes": out,
                       "timing": "wall clock around whole-batch steps (synchronised)"}}
    print(json.dumps(line), flush=True)


def _served_jobs(args, rank):
    """The arrival stream and its pooled job images (generated in worker processes, largest
    first; spawn, so that no worker inherits a CUDA context)."""
    import multiprocessing as mp

    from paper_1403_0240_gb300 import synth
    arrivals = synth.arrival_stream(args.jobs, rate=args.rate, seed=42 + rank)
    keys = [synth.served_job_key(a) for a in arrivals]
    distinct = sorted(set(keys), key=lambda k: -(k[1] ** (3 if k[0] == "pc3d" else 2)))
    procs = max(1, min(len(os.sched_getaffinity(0)), len(distinct), 16))
    with mp.get_context("spawn").Pool(procs) as pool:
        made = pool.starmap(synth.served_job, [(k, args.job_iters) for k in distinct], chunksize=1)
    return arrivals, keys, dict(zip(distinct, made))


def _served_params(w) -> dict:
    return dict(model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff, ps_radius=w.ps_radius)


def _plain_stream(reqs, dev):
    """One job at a time, first come first served, in real time over the same arrivals: each
    job is set up from its host buffers, stepped through all its iterations and its labels read
    back before the next one starts. Returns (results, makespan from the first arrival)."""
    import torch

    from paper_1403_0240_gb300 import seg
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    out = []
    for r in sorted(reqs, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        start = time.perf_counter() - t0
        c = seg.Context(r.image, r.labels0, **r.params)
        st = c.step(r.iterations)
        c.labels()
        c.close()
        done = time.perf_counter() - t0
        out.append({"job": r.job_id, "arrival": r.arrival, "start": start, "done": done,
                    "latency": done - r.arrival, "service": done - start, "particles": st["particles_total"]})
    return out, max(x["done"] for x in out) - min(x["arrival"] for x in out)


def _serve_stream(reqs, dev, budget, iters_per_step, keep_labels=False):
    """The continuous-batching server over the arrivals in real time; returns (server, results)."""
    import torch

    from paper_1403_0240_gb300.serve import SegBackend, Server
    be = SegBackend(stream=torch.cuda.current_stream(dev), init_stream=torch.cuda.Stream(dev, priority=-1),
                    keep_labels=keep_labels, time_steps=True)
    srv = Server(be, budget, max_jobs=512, max_iters_per_step=iters_per_step)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = srv.run(reqs, t0=t0)
    torch.cuda.synchronize(dev)
    srv.t_start = t0
    be.close()
    return srv, res


def _requests(arrivals, keys, cache, pinned, iters, scale_rate=1.0):
    from paper_1403_0240_gb300.serve import Request
    out = []
    for i, (a, k) in enumerate(zip(arrivals, keys)):
        img_h, lab_h, nl = pinned[k]
        out.append(Request(i, a.t * scale_rate, img_h, lab_h, iters, _served_params(cache[k]), nlabels=nl))
    return out


def _oracle_stream_sample(arrivals, keys, cache, seconds, iters_each=5):
    """The oracle, single-threaded, on the first iterations of the stream's jobs in arrival
    order (iters_each per job) until `seconds` have passed; returns (particle-iterations/s,
    seconds, [(key, seconds of that job)])."""
    import oracle
    total, parts, sample = 0.0, 0, []
    for k in keys:
        if total >= seconds:
            break
        w = cache[k]
        p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
        run = oracle.Run(p, w.image, w.labels0)
        t0 = time.perf_counter()
        for _ in range(iters_each):
            s, _ = run.step()
            parts += s["n_particles"]
        dt = time.perf_counter() - t0
        total += dt
        sample.append((k, dt))
    return parts / total, total, sample


def _oracle_worker(keys, iters, iters_each, barrier, out):
    """One host core: set up the oracle runs of its jobs, wait for the others, run them."""
    import oracle
    from paper_1403_0240_gb300 import synth
    runs = []
    for k in keys:
        w = synth.served_job(k, iters)
        p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
        runs.append(oracle.Run(p, w.image, w.labels0))
    barrier.wait()
    parts = 0
    for r in runs:
        for _ in range(iters_each):
            s, _ = r.step()
            parts += s["n_particles"]
    out.put(parts)


def _oracle_all_cores(sample, iters, iters_each):
    """The same sample with one single-threaded oracle process per host core: jobs assigned
    longest first to the least loaded core (by their single-core times), set up before the
    clock starts; returns (particle-iterations/s, processes, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = max(1, min(len(os.sched_getaffinity(0)), len(sample)))
    load = [0.0] * cores
    share = [[] for _ in range(cores)]
    for k, dt in sorted(sample, key=lambda x: -x[1]):
        c = load.index(min(load))
        share[c].append(k)
        load[c] += dt
    barrier = ctx.Barrier(cores + 1)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(share[c], iters, iters_each, barrier, out)) for c in range(cores)]
    for pr in procs:
        pr.start()
    barrier.wait()
    t0 = time.perf_counter()
    parts = sum(out.get() for _ in procs)
    dt = time.perf_counter() - t0
    for pr in procs:
        pr.join()
    return parts / dt, cores, dt


def run_served(args, world, rank, local, pg):
    """Served workload: Poisson arrivals (200 jobs/s; 80% 2D of sides 128-1024, half piecewise
    constant disks and half piecewise smooth ellipses, 20% 3D ellipsoid volumes of sides
    64-256; 100 iterations each) through the continuous-batching server, against the same
    stream run one job at a time."""
    import torch

    from paper_1403_0240_gb300 import seg

    arrivals, keys, cache = _served_jobs(args, rank)     # worker processes before any CUDA work
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pinned = {}
    for k, w in cache.items():      # request payloads sit in pinned host memory, as a server's would
        pinned[k] = (torch.from_numpy(w.image).pin_memory(), torch.from_numpy(w.labels0).pin_memory(),
                     int(w.labels0.max()) + 1)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(0.6 * free)
    iters = args.job_iters

    # warm-up: graph capture and first launches on one job of every kind, then one of each
    # distinct pooled job through the server (untimed)
    warm_keys = []
    for kind in ("pc2d", "ps2d", "pc3d"):
        ks = [k for k in cache if k[0] == kind]
        if ks:
            warm_keys.append(min(ks, key=lambda k: k[1]))
    from paper_1403_0240_gb300.serve import Request
    warm = [Request(i, 0.0, pinned[k][0], pinned[k][1], 3, _served_params(cache[k]), pinned[k][2])
            for i, k in enumerate(warm_keys)]
    _serve_stream(warm, dev, budget, args.iters_per_step)

    # the served stream (timed): per-step device time from CUDA events on the batch stream
    reqs = _requests(arrivals, keys, cache, pinned, iters)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(pg)
    launches0 = seg.kernel_launches()
    srv, res = _serve_stream(reqs, dev, budget, args.iters_per_step)
    launches_stream = seg.kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    log = srv.log
    # the timed window: K server steps from the first step, at or after the W-th, that starts
    # once the whole stream has arrived (every remaining job is resident or queued: the server
    # works on its full backlog); earlier steps are the ramp-up. When fewer than K steps remain
    # the window ends with the last step.
    last_arrival = max(r.arrival for r in res)
    s0 = next((i for i, e in enumerate(log) if i >= args.warmup and e["t0"] >= last_arrival), len(log))
    s0 = max(min(args.warmup, len(log) - 1), min(s0, len(log) - args.steps))
    win = log[s0:s0 + args.steps]
    win_ms = sum(e["device_ms"] for e in win)
    win_parts = sum(e["particles"] for e in win)
    win_wall = win[-1]["t1"] - win[0]["t0"]
    value, _, t_max = aggregate(pg, float(win_parts), win_ms / 1000.0)
    # kernels launched inside the window: each step's graph replays plus the set-up of the jobs
    # admitted meanwhile (counted by the library)
    win_launches = sum(e["launches"] for e in win)
    t_first = min(r.arrival for r in res)
    makespan = max(r.completed for r in res) - t_first
    stream_parts = sum(r.particles for r in res)
    served_lat = np.array([r.latency for r in res])

    # the same stream, one job at a time (real run, real time)
    plain, plain_makespan = _plain_stream(_requests(arrivals, keys, cache, pinned, iters), dev)
    plain_parts = sum(x["particles"] for x in plain)
    plain_busy = sum(x["service"] for x in plain)
    plain_lat = np.array([x["latency"] for x in plain])
    plain_kind = {}
    for x in plain:
        d = plain_kind.setdefault(keys[x["job"]][0], {"jobs": 0, "busy_s": 0.0, "particle_iterations": 0})
        d["jobs"] += 1
        d["busy_s"] += x["service"]
        d["particle_iterations"] += x["particles"]

    # the arrival rate the server sustains: its throughput under overload over the mean job
    # size; then a shorter stream at 80% of that rate, whose latencies must stay bounded
    capacity = stream_parts / makespan
    mean_job = stream_parts / len(res)
    rate_star = capacity / mean_job
    n_sus = min(len(reqs), args.sustain_jobs)
    sus_reqs = _requests(arrivals[:n_sus], keys[:n_sus], cache, pinned, iters,
                         scale_rate=args.rate / (0.8 * rate_star))
    srv2, res2 = _serve_stream(sus_reqs, dev, budget, args.iters_per_step)
    sus_lat = np.array([r.latency for r in res2])
    sus_first = min(r.arrival for r in res2)
    sus_span = max(r.arrival for r in res2) - sus_first

    # stage breakdown of a batch of the stream's first jobs (per-stage events inside the graph)
    prof_jobs = [cache[k] for k in keys[:args.profile_jobs]]
    ctxs = [seg.Context(pinned[k][0], pinned[k][1], **_served_params(cache[k])) for k in keys[:args.profile_jobs]]
    b = seg.Batch(stream=torch.cuda.current_stream(dev))
    for c in ctxs:
        b.add(c)
    b.step(2)
    b.profile(True)
    b.step(2)
    stage_ms = {k: 0.0 for k in STAGES}
    stage_parts, n_prof = 0.0, 5
    for _ in range(n_prof):
        sts = b.step(1)
        st_ms = b.stage_times()
        for k in STAGES:
            stage_ms[k] += st_ms[k] / n_prof
        stage_parts += sum(x["n_particles"] for x in sts) / n_prof
    b.close()
    for c in ctxs:
        c.close()

    if rank != 0:
        return
    dom = max(stage_ms, key=stage_ms.get)
    per_p, _ = ALG_BYTES[dom]
    alg_bytes = per_p * stage_parts
    peak, peak_kind = read_peaks()
    achieved = alg_bytes / (stage_ms[dom] / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(dom, "served", stage_parts), "kernel": dom, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes, "mean_launch_ms": stage_ms[dom],
                "measured_on": f"a batch of the stream's first {len(prof_jobs)} jobs, per-stage CUDA events"}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v1, secs, sample = _oracle_stream_sample(arrivals, keys, cache, args.cpu_seconds, iters_each=2)
        njobs = len(sample)
        vN, cores, secsN = _oracle_all_cores(sample, iters, 2)
        cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"iterations 0-1 of the stream's first {njobs} jobs in arrival order ({secs:.1f} s), "
                         "single-threaded FP64 C oracle",
               "all_cores": {"value": vN, "cores": cores, "seconds": secsN,
                             "sample": "the same jobs and iterations, one single-threaded oracle process per "
                                       "host core (os.sched_getaffinity), jobs set up before the clock"}}
    in_bytes = sum(r.image.numel() * r.image.element_size() + r.labels0.numel() * 4 for r in reqs)
    out_bytes = sum(r.labels0.numel() * 4 for r in reqs)
    n_steps = max(1, srv.steps)
    e2e = {"value": stream_parts / makespan, "unit": UNIT, "h2d_bytes_per_step": int(in_bytes / n_steps),
           "d2h_bytes_per_step": int(out_bytes / n_steps) + 200 * int(np.mean([e["members"] for e in log])),
           "what": "the whole served stream: request payloads from pinned host memory, set-up, all "
                   "iterations, labels back to the host; first arrival to last completion"}
    by_kind = {}
    for r, k in zip(sorted(res, key=lambda r: r.job_id), keys):
        d = by_kind.setdefault(k[0], {"jobs": 0, "particle_iterations": 0})
        d["jobs"] += 1
        d["particle_iterations"] += r.particles
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(win),
            "warmup": s0, "ms_per_step": win_ms / len(win), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served", "jobs": len(res), "arrival_rate_per_s": args.rate,
                       "description": "Poisson arrivals, 80% 2D (half piecewise-constant disks, half piecewise-"
                                      "smooth ellipses, sides 128-1024), 20% 3D uint16 ellipsoids (sides 64-256); "
                                      f"{iters} iterations per job; images pooled by size bucket",
                       "step": "one server step: up to {0} iterations of every resident job, one graph replay "
                               "per iteration for all of them".format(args.iters_per_step),
                       "timed_window": f"server steps {s0}..{s0 + len(win) - 1} of {len(log)} (from the first step "
                                       f"at or after step {args.warmup} that starts after the last arrival), CUDA "
                                       "events on the batch stream; value = their particle-iterations / their "
                                       "device time",
                       "window_mean_jobs": float(np.mean([e["members"] for e in win])),
                       "window_wall_value": win_parts / win_wall,
                       "l2": "not flushed: every step walks all resident jobs (the working set exceeds L2)",
                       "served_value": stream_parts / makespan, "served_makespan_s": makespan,
                       "served_p50_s": float(np.percentile(served_lat, 50)),
                       "served_p99_s": float(np.percentile(served_lat, 99)),
                       "plain_value": plain_parts / plain_makespan, "plain_makespan_s": plain_makespan,
                       "plain_busy_value": plain_parts / plain_busy,
                       "plain_by_kind": {k: {"jobs": v["jobs"], "busy_s": round(v["busy_s"], 3),
                                             "particle_iterations": v["particle_iterations"]}
                                         for k, v in plain_kind.items()},
                       "plain_p50_s": float(np.percentile(plain_lat, 50)),
                       "plain_p99_s": float(np.percentile(plain_lat, 99)),
                       "served_over_plain": (stream_parts / makespan) / (plain_parts / plain_makespan),
                       "plain": "the same arrivals one job at a time in real time (set-up from host buffers, "
                                "all iterations, labels back), first come first served",
                       "offered_particle_iterations_per_s": stream_parts / max(1e-9, arrivals[-1].t - arrivals[0].t),
                       "sustainable_rate_jobs_per_s": rate_star,
                       "at_80pct_of_sustainable": {"rate_jobs_per_s": 0.8 * rate_star, "jobs": len(res2),
                                                   "p50_s": float(np.percentile(sus_lat, 50)),
                                                   "p99_s": float(np.percentile(sus_lat, 99)),
                                                   "arrival_span_s": sus_span,
                                                   "makespan_s": max(r.completed for r in res2) - sus_first},
                       "budget_bytes": budget, "server_steps": len(log),
                       "by_kind": by_kind,
                       "stages_ms": {k: round(v, 5) for k, v in stage_ms.items()},
                       "stage_particles": stage_parts},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": win_launches, "gpu_launches_stream": launches_stream,
            "clocks": clocks, "wall_s": makespan}
    print(json.dumps(line), flush=True)


def _contour_length(L: np.ndarray) -> int:
    """Adjacent pixel pairs (4/6-neighbours) with different labels: the length prior's P."""
    return int(sum(np.count_nonzero(np.diff(L, axis=a)) for a in range(L.ndim)))


def _pc_energy(I: np.ndarray, L: np.ndarray, lam: float) -> float:
    """Piecewise-constant energy: squared deviations from the region means plus lambda * P."""
    I64 = I.astype(np.float64).ravel()
    lab = L.ravel()
    n = np.bincount(lab)
    S = np.bincount(lab, weights=I64)
    mu = np.divide(S, n, out=np.zeros_like(S), where=n > 0)
    return float(np.sum((I64 - mu[lab]) ** 2) + lam * _contour_length(L))


def _deconv_energy(I: np.ndarray, L: np.ndarray, psf: np.ndarray, lam: float) -> float:
    """sum (I - K * s)^2 + lam |Gamma| for the deconvolving model (theta = region means, K the
    separable PSF, zero outside the image), evaluated in FP64 on the host for the report."""
    Id = I.astype(np.float64)
    M = int(L.max()) + 1
    n = np.bincount(L.ravel(), minlength=M)
    S = np.bincount(L.ravel(), weights=Id.ravel(), minlength=M)
    theta = np.where(n > 0, S / np.maximum(n, 1), 0.0)
    J = theta[L]
    r = (psf.size - 1) // 2
    for axis in range(L.ndim):
        pad = [(0, 0)] * L.ndim
        pad[axis] = (r, r)
        Jp = np.pad(J, pad)
        acc = np.zeros_like(J)
        for u, k in enumerate(psf):
            acc += k * np.take(Jp, np.arange(u, u + J.shape[axis]), axis=axis)
        J = acc
    return float(((Id - J) ** 2).sum()) + lam * _contour_length(L)


def run_convergence(args, world, rank, local, pg):
    """Iterations to convergence of the L2 flow and of the Sobolev flow with the oscillation
    switch live, on the 128^2 and 1024^2 workloads and the 512^2 deconvolution scene (one job at
    a time, status read every iteration)."""
    import torch

    from paper_1403_0240_gb300 import seg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = []
    for name in ("disks128", "ellipses1024", "deconv512"):
        make, _ = workloads()[name]
        w = make(rank)
        runs = {}
        for flow in ("l2", "sobolev", "sobolev_global"):
            ctx = seg.Context(torch.from_numpy(w.image).to(dev), torch.from_numpy(w.labels0).to(dev), model=w.model,
                              connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff, ps_radius=w.ps_radius,
                              gradient=flow, osc_window=args.osc_window if flow != "l2" else 0, psf=w.psf)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            switch, accepted, it = None, [], 0
            # a flow also stops when its labels repeat with period 2 (the deconvolving model's
            # re-estimated means can make a few pixels flip back and forth for ever)
            hist, cycle_at = [], None
            while it < args.max_iters:
                st = ctx.step(1)
                it += 1
                accepted.append(st["n_accepted"])
                if flow != "l2" and switch is None and st["mode_used"] == seg.SEG_L2:
                    switch = st["iteration"]
                if st["converged"]:
                    break
                if w.model == "pcd":
                    hist = (hist + [ctx.labels().copy()])[-3:]
                    if len(hist) == 3 and np.array_equal(hist[0], hist[2]):
                        cycle_at = it
                        break
            torch.cuda.synchronize(dev)
            secs = time.perf_counter() - t0
            L = ctx.labels().copy()
            runs[flow] = {"iterations": it, "converged": bool(st["converged"]), "switch_to_l2_at": switch,
                          "period2_at": cycle_at, "moves_last_iteration": accepted[-1] if accepted else 0,
                          "seconds": round(secs, 4), "particle_iterations": int(st["particles_total"]),
                          "moves": int(sum(accepted)), "contour_length": _contour_length(L),
                          "energy": (_pc_energy(w.image, L, w.lam) if w.model == "pc" else
                                     _deconv_energy(w.image, L, w.psf, w.lam) if w.model == "pcd" else None),
                          "labels": L}
            ctx.close()
        agree = float(np.mean(runs["l2"]["labels"] == runs["sobolev"]["labels"]))
        agree_g = float(np.mean(runs["sobolev_global"]["labels"] == runs["sobolev"]["labels"]))
        for r in runs.values():
            r.pop("labels")
        out.append({"workload": name, "l2": runs["l2"], "sobolev": runs["sobolev"],
                    "sobolev_global": runs["sobolev_global"], "final_label_agreement": agree,
                    "global_vs_local_agreement": agree_g})
    if rank != 0:
        return
    tot_p = sum(r[f]["particle_iterations"] for r in out for f in ("l2", "sobolev", "sobolev_global"))
    tot_s = sum(r[f]["seconds"] for r in out for f in ("l2", "sobolev", "sobolev_global"))
    line = {"metric": METRIC, "value": tot_p / tot_s, "unit": UNIT, "n_gpus": world, "steps": None,
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "convergence", "osc_window": args.osc_window, "max_iters": args.max_iters,
                       "timing": "wall clock, status read after every iteration", "runs": out}}
    print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """Reference arm: the oracle, timed on this host's cores, on the same workload. For the
    served workload a step is one oracle iteration of a stream job: iterations 0-4 of each job
    in arrival order (W warm-up steps, then K timed)."""
    if rank != 0:
        return
    import oracle
    name = args.workload
    if name == "served":
        from paper_1403_0240_gb300 import synth
        arrivals = synth.arrival_stream(args.jobs, rate=args.rate, seed=42)
        keys = [synth.served_job_key(a) for a in arrivals]
        n_jobs = (args.warmup + args.steps + 4) // 5
        runs = []
        for k in keys[:n_jobs]:
            w = synth.served_job(k, args.job_iters)
            p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
            runs.append(oracle.Run(p, w.image, w.labels0))
        seq = [runs[i // 5] for i in range(args.warmup + args.steps)]
        desc = (f"the served stream's first {n_jobs} jobs in arrival order, iterations 0-4 of each, one oracle "
                "iteration per step")
    else:
        make, desc = workloads()[name]
        w = make(0)
        p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius, psf=w.psf,
                               topology=topology_code(args.topology), curv_radius=args.curv_radius)
        run = oracle.Run(p, w.image, w.labels0)
        seq = [run] * (args.warmup + args.steps)
    for r in seq[:args.warmup]:
        r.step()
    parts, times = 0, []
    for r in seq[args.warmup:]:
        t0 = time.perf_counter()
        s, _ = r.step()
        times.append(time.perf_counter() - t0)
        parts += s["n_particles"]
    total = sum(times)
    value = parts / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "description": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"steps {args.warmup}..{args.warmup + args.steps - 1} ({desc}), "
                                       "single-threaded FP64 C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local, pg):
    import numpy as np
    import torch

    from paper_1403_0240_gb300 import seg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    name = args.workload
    make, desc = workloads()[name]
    w = make(rank)
    iters_per_job = w.iterations
    img_d = torch.from_numpy(w.image).to(dev)
    lab_d = torch.from_numpy(w.labels0).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    settings = {}
    if args.tile:
        settings["tile"] = tuple(int(v) for v in args.tile.split("x"))
    if args.cell_edge:
        settings["cell_edge"] = args.cell_edge
    tune_table = None
    if args.autotune:
        best, tune_table = seg.autotune(img_d, lab_d, iters=20, stream=stream, model=w.model,
                                        connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                                        ps_radius=w.ps_radius)
        settings = {"cell_edge": best["cell_edge"], "tile": best["tile"]}
    if args.topology:
        settings["topology"] = topology_code(args.topology)
        if topology_code(args.topology) & 2:
            # split pieces take new labels: room for the job's iterations (the 1024^2 scene gains
            # 12-20 labels per iteration at its lambda)
            m0 = int(w.labels0.max()) + 1
            settings["max_labels"] = args.max_labels or 4 * m0 + 4096
    if args.curv_radius > 0:
        settings["curv_radius"] = args.curv_radius

    def new_ctx(profile):
        c = seg.Context(img_d, lab_d, model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                        ps_radius=w.ps_radius, osc_window=0, stream=stream, psf=w.psf, **settings)
        c.profile(profile)
        return c

    iter_log = open(args.iter_log, "w") if args.iter_log else None
    job = {"ctx": new_ctx(False), "done": 0, "before": 0, "profile": False}

    def step_job(phase):
        """One iteration of the current job (a fresh job every iters_per_job iterations); returns
        the CUDA-event time of the iteration, its status and the finished jobs' particles."""
        finished = 0
        if job["done"] == iters_per_job:
            finished = job["ctx"].poll()["particles_total"] - job["before"]
            job["ctx"].close()
            job.update(ctx=new_ctx(job["profile"]), done=0, before=0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        job["ctx"].step_async(1)
        e1.record(stream)
        job["done"] += 1
        sp = job["ctx"].poll()
        if iter_log:
            iter_log.write(json.dumps({"phase": phase, **sp}) + "\n")
        return e0, e1, sp, finished

    def pass_particles(parts_done):
        return parts_done + job["ctx"].poll()["particles_total"] - job["before"]

    for _ in range(args.warmup):
        step_job("warmup")
    torch.cuda.synchronize(dev)

    # pass 1 (the reported value): no events inside the iteration graph, so the stage kernels'
    # launches overlap (programmatic dependent launch)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(pg)
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    job["before"] = job["ctx"].poll()["particles_total"]
    evs, parts_done = [], 0
    accepted = fixups = rounds = 0
    for k in range(args.steps):
        e0, e1, sp, fin = step_job("timed")
        evs.append((e0, e1))
        parts_done += fin
        accepted += sp["n_accepted"]
        fixups += sp["n_fixup"]
        rounds += sp["mis_rounds"]
    particles = float(pass_particles(parts_done))
    torch.cuda.synchronize(dev)
    barrier(pg)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    if job["ctx"].poll()["error"]:
        raise RuntimeError(f"device error {job['ctx'].poll()['error']}")
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, total_particles, t_max = aggregate(pg, particles, dev_ms / 1000.0)

    # pass 2 (the stage breakdown and the roofline kernel time): CUDA events recorded between
    # the stages inside the graph; these serialise the launches, so this pass runs slower
    job["profile"] = True
    job["ctx"].profile(True)
    for _ in range(2):
        step_job("warmup")
    n_stage = min(args.steps, 200)
    stage_ms = {k: 0.0 for k in STAGES}
    stage_parts, stage_dev_ms = 0, 0.0
    job["before"] = job["ctx"].poll()["particles_total"]
    for k in range(n_stage):
        e0, e1, sp, fin = step_job("stages")
        st = job["ctx"].stage_times()
        for s_ in STAGES:
            stage_ms[s_] += st[s_]
        stage_dev_ms += e0.elapsed_time(e1)
        stage_parts += fin
    stage_parts = float(pass_particles(stage_parts))
    job["ctx"].close()

    # end to end through the public API: host (pinned) inputs, a status read every step,
    # the label image back to the host at the end; one job of K' iterations
    img_h = torch.from_numpy(w.image).pin_memory()
    lab_h = torch.from_numpy(w.labels0).pin_memory()
    out_h = torch.empty(w.labels0.shape, dtype=torch.int32).pin_memory()
    k_e2e = min(args.steps, iters_per_job)
    barrier(pg)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    c2 = seg.Context(img_h, lab_h, model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                     ps_radius=w.ps_radius, osc_window=0, stream=stream, psf=w.psf, **settings)
    for _ in range(k_e2e):
        s2 = c2.step(1)
    c2.labels(out=out_h)
    e2e_t = time.perf_counter() - t0
    barrier(pg)
    e2e_parts = allsum(pg, float(s2["particles_total"]))
    e2e_t = allmax(pg, e2e_t)
    c2.close()
    in_bytes = w.image.nbytes + w.labels0.nbytes + (w.psf.nbytes if w.psf is not None else 0)
    status_bytes = 200     # the per-step counter record read back by seg_step
    e2e = {"value": e2e_parts / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": int(math.ceil(in_bytes / k_e2e)),
           "d2h_bytes_per_step": int(math.ceil(w.labels0.nbytes / k_e2e)) + status_bytes,
           "iterations": k_e2e}

    if rank != 0:
        return
    mean_stage = {k: v / n_stage for k, v in stage_ms.items()}
    dom = max(mean_stage, key=mean_stage.get)
    mean_parts = particles / args.steps
    stage_mean_parts = stage_parts / n_stage
    if dom == "psf":
        # the deconvolving model's FP64 field passes: bound by the FP64 pipe
        flops = psf_pass_flops(w)
        achieved = flops / (mean_stage[dom] / 1000.0) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None, "kernel": "psf (k_psf_pass x3)",
                    "peak_source": "nominal FP64 (no measured FP64 figure)", "algorithmic_flops_per_launch": flops,
                    "mean_launch_ms": mean_stage[dom]}
    else:
        per_p, per_move = ALG_BYTES[dom]
        alg_bytes = per_p * stage_mean_parts + per_move * (accepted / args.steps)
        peak, peak_kind = read_peaks()
        achieved = alg_bytes / (mean_stage[dom] / 1000.0) / 1e9
        traffic = traffic_from_profile(dom, name, stage_mean_parts)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "kernel": dom, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": alg_bytes, "mean_launch_ms": mean_stage[dom]}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, its, secs = oracle_sample(w, seconds=args.cpu_seconds, topology=topology_code(args.topology),
                                     curv_radius=args.curv_radius)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {its} iterations of the same job ({secs:.1f} s), single-threaded FP64 C oracle"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if w.model == "pcd" else "f32",
            "data": "synthetic",
            "config": {"workload": name, "description": desc, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between timed iterations (256 MiB write)",
                       "iterations_per_job": iters_per_job, "mean_particles": mean_parts,
                       "settings": {k: list(v) if isinstance(v, tuple) else v for k, v in settings.items()} or "default",
                       "autotune_ms_per_iter": tune_table,
                       "mean_accepted": accepted / args.steps, "mean_fp64_recomputes": fixups / args.steps,
                       "mean_selection_rounds": rounds / args.steps,
                       "precision": "float32 gradients with certified bounds, FP64 recompute of uncertified "
                                    "decisions, exact region sums"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            # per step: the kernels of the iteration graph plus the status gather of poll()
            "gpu_launches": (KERNELS_PER_ITERATION + 1 + psf_passes(w) + extra_kernels(args)) * args.steps,
            "clocks": clocks,
            "stages_ms": {k: round(v, 5) for k, v in mean_stage.items()},
            "stage_pass": {"steps": n_stage, "ms_per_step": stage_dev_ms / n_stage,
                           "note": "per-stage CUDA events inside the iteration graph (serialises the "
                                   "stage launches); roofline.mean_launch_ms comes from this pass"},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: served 40, per-image 1000)")
    ap.add_argument("--warmup", type=int, default=None, help="warm-up steps (default: served 5, per-image 20)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="served", choices=sorted(list(workloads().keys()) + ["batch512", "served", "convergence", "precision"]))
    ap.add_argument("--images", type=int, default=512, help="batch512: images in the batch")
    ap.add_argument("--jobs", type=int, default=600, help="served: jobs in the arrival stream")
    ap.add_argument("--rate", type=float, default=200.0, help="served: arrivals per second")
    ap.add_argument("--sustain-jobs", type=int, default=150,
                    help="served: jobs of the stream replayed at 80%% of the sustainable rate")
    ap.add_argument("--profile-jobs", type=int, default=48,
                    help="served: jobs of the batch whose stages are timed for the roofline")
    ap.add_argument("--job-iters", type=int, default=100, help="served: iterations per job")
    ap.add_argument("--iters-per-step", type=int, default=4, help="served: most iterations per batch step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="batch512: default cell edge and tile shape")
    ap.add_argument("--tile", default="", help="tile shape in pixels, e.g. 30x64 (2D: y x x) or 8x8x32")
    ap.add_argument("--cell-edge", type=int, default=0)
    ap.add_argument("--topology", default="", choices=["", "vanish", "split", "fuse", "vanish+split", "vanish+fuse",
                                                         "split+fuse", "vanish+split+fuse"],
                    help="opt-in topology events (fusion: piecewise-constant workloads)")
    ap.add_argument("--max-labels", type=int, default=0,
                    help="label capacity with splits (default 4 M + 4096 for M initial labels)")
    ap.add_argument("--curv-radius", type=float, default=0.0,
                    help="curvature regulariser with this ball radius instead of the length prior")
    ap.add_argument("--autotune", action="store_true", help="time seg_autotune's candidates first and use the fastest")
    ap.add_argument("--osc-window", type=int, default=10, help="convergence: oscillation window of the Sobolev flow")
    ap.add_argument("--max-iters", type=int, default=3000, help="convergence: iteration cap per run")
    ap.add_argument("--iter-log", default="", help="write every warm-up and timed iteration's status here "
                    "(JSON lines), to relate profiler launches to their particle counts")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 40 if args.workload == "served" else 1000
    if args.warmup is None:
        args.warmup = 5 if args.workload == "served" else 20
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, pg = dist_setup() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0, None)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch512":
        run_batch(args, world, rank, local, pg)
    elif args.workload == "served":
        run_served(args, world, rank, local, pg)
    elif args.workload == "convergence":
        run_convergence(args, world, rank, local, pg)
    elif args.workload == "precision":
        run_precision(args, world, rank, local, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
