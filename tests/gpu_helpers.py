"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle side by side."""
import numpy as np

import oracle
from paper_1403_0240_gb300 import seg

# Float tolerance of the FP32 path against the FP64 oracle: 1e-5 of each value's first-order
# magnitude scale from the oracle (dE: every deviation v - mu weighted by the magnitudes it is
# formed from, plus the data and length terms; g: the Eq. 6 sums of K times those scales,
# plus |A| + |B|), because both are differences of nearly equal quantities. Each value must
# also lie within the rigorous bound the library reports for it.
REL_TOL = 1e-5


def pair(w, gradient="sobolev", osc_window=0, cell_edge=0, lam=None, cutoff=None):
    lam = w.lam if lam is None else lam
    cutoff = w.cutoff if cutoff is None else cutoff
    psf = getattr(w, "psf", None)
    ctx = seg.Context(w.image, w.labels0, model=w.model, connectivity=w.connectivity, lam=lam, cutoff=cutoff,
                      ps_radius=w.ps_radius, gradient=gradient, osc_window=osc_window, cell_edge=cell_edge, psf=psf)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, lam, cutoff, w.ps_radius,
                           gradient=gradient, osc_window=osc_window, psf=psf)
    return ctx, oracle.Run(p, w.image, w.labels0)


def scaled_err(x, ref, scale):
    """max |x - ref| / scale, the scale being the sum of term magnitudes (0 where scale is 0)."""
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    err = np.abs(np.asarray(x, np.float64) - ref)
    scale = np.asarray(scale, np.float64)
    assert (err[scale == 0] == 0).all()
    nz = scale > 0
    return float((err[nz] / scale[nz]).max()) if nz.any() else 0.0


def plain_rel_err(x, ref, scale):
    """Plain relative error where |ref| > 1e-3 of its scale (reported, not asserted)."""
    ref = np.asarray(ref, np.float64)
    m = np.abs(ref) > 1e-3 * np.asarray(scale, np.float64)
    if not m.any():
        return 0.0
    return float((np.abs(np.asarray(x, np.float64)[m] - ref[m]) / np.abs(ref[m])).max())


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
    stats = {"rel_dE": scaled_err(g["dE"], dump["dE"], dump["dE_scale"]),
             "rel_g": scaled_err(g["g"], dump["g"], dump["g_scale"]),
             "plain_rel_g": plain_rel_err(g["g"], dump["g"], dump["g_scale"]),
             "fixed": int(fixed.sum()), "n": int(g["idx"].size)}
    assert stats["rel_dE"] <= REL_TOL and stats["rel_g"] <= REL_TOL, (where, stats)
    assert np.array_equal(ctx.labels(), run.L), (where, "labels differ")
    return st, stats
