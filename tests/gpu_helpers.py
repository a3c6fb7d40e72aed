"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle side by side."""
import numpy as np

import oracle
from paper_1403_0240_gb300 import seg

# Float tolerance of the FP32 gradients against the FP64 oracle: relative 1e-5 of the
# larger of |reference| and a cancellation floor (1e-3 of the largest |reference| of the
# iteration), besides the per-particle rigorous bound the library reports.
REL_TOL = 1e-5
FLOOR = 1e-3


def pair(w, gradient="sobolev", osc_window=0, cell_edge=0, lam=None, cutoff=None):
    lam = w.lam if lam is None else lam
    cutoff = w.cutoff if cutoff is None else cutoff
    ctx = seg.Context(w.image, w.labels0, model=w.model, connectivity=w.connectivity, lam=lam, cutoff=cutoff,
                      ps_radius=w.ps_radius, gradient=gradient, osc_window=osc_window, cell_edge=cell_edge)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, lam, cutoff, w.ps_radius,
                           gradient=gradient, osc_window=osc_window)
    return ctx, oracle.Run(p, w.image, w.labels0)


def rel_err(x, ref):
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    floor = FLOOR * float(np.abs(ref).max())
    return float((np.abs(np.asarray(x, np.float64) - ref) / np.maximum(np.abs(ref), max(floor, 1e-300))).max())


def compare_step(ctx, run, label=""):
    """Advance both sides one iteration and compare everything the iteration produced."""
    st = ctx.step(1)
    ref, dump = run.step(dump=True)
    where = f"{label} iteration {ref.get('n_particles')}"
    for k in ("n_particles", "n_candidates", "n_accepted", "mode_used", "converged"):
        assert st[k] == ref[k], (label, k, st, ref)
    if ref["converged"] and ref["n_particles"] == 0:
        assert np.array_equal(ctx.labels(), run.L)
        return st, {}
    got = ctx.particles()
    order = np.lexsort((got["c"], got["idx"]))
    g = {k: v[order] for k, v in got.items()}
    assert np.array_equal(g["idx"], dump["idx"]), where
    assert np.array_equal(g["l"], dump["l"]), where
    assert np.array_equal(g["c"], dump["c"]), where
    dE_err = np.abs(g["dE"].astype(np.float64) - dump["dE"])
    assert (dE_err <= g["eE"].astype(np.float64)).all(), (where, "dE outside its bound", float(dE_err.max()))
    g_err = np.abs(g["g"].astype(np.float64) - dump["g"])
    assert (g_err <= g["eg"].astype(np.float64)).all(), (where, "g outside its bound", float(g_err.max()))
    fixed = (g["flags"] & 1) != 0
    assert np.array_equal(g["key"][fixed], dump["g"][fixed]), (where, "FP64 recompute differs from the oracle")
    stats = {"rel_dE": rel_err(g["dE"], dump["dE"]), "rel_g": rel_err(g["g"], dump["g"]),
             "fixed": int(fixed.sum()), "n": int(g["idx"].size)}
    assert stats["rel_dE"] <= REL_TOL and stats["rel_g"] <= REL_TOL, (where, stats)
    assert np.array_equal(ctx.labels(), run.L), (where, "labels differ")
    return st, stats
