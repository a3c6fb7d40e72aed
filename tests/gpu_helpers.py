"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle side by side."""
import json
import os

import numpy as np

import oracle
from paper_1403_0240_gb300 import seg

# Float tolerance of the FP32 path against the FP64 oracle. Both dE and g are sums of terms
# that can cancel (t1 - t2, A - B), so the contract is |x - x_ref| <= REL_TOL * T, with T the
# value's sum of term magnitudes computed by the oracle (orc_energy / orc_sobolev). Where the
# value is not dominated by cancellation, |x_ref| >= PLAIN_FLOOR * T, the plain relative error
# |x - x_ref| / |x_ref| must also stay within REL_TOL. The library keeps each dE as its FP64
# value in a float pair and sums Eq. 6 with compensated products, so both hold down to values a
# thousandth of their term sums; the plain relative error is also recorded at 1e-6 of T.
# Each value must also lie within the rigorous bound the library reports for it.
REL_TOL = 1e-5
PLAIN_FLOOR = 1e-3
REPORT_FLOORS = (1e-6, PLAIN_FLOOR)

# largest errors seen per test label (written out at the end of the session when
# SEG_PARITY_REPORT names a file)
ERRORS: dict = {}


def pair(w, gradient="sobolev", osc_window=0, cell_edge=0, lam=None, cutoff=None):
    lam = w.lam if lam is None else lam
    cutoff = w.cutoff if cutoff is None else cutoff
    psf = getattr(w, "psf", None)
    ctx = seg.Context(w.image, w.labels0, model=w.model, connectivity=w.connectivity, lam=lam, cutoff=cutoff,
                      ps_radius=w.ps_radius, gradient=gradient, osc_window=osc_window, cell_edge=cell_edge, psf=psf)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, lam, cutoff, w.ps_radius,
                           gradient=gradient, osc_window=osc_window, psf=psf)
    return ctx, oracle.Run(p, w.image, w.labels0)


def scaled_err(x, ref, terms):
    """max |x - ref| / T over the values, T the sum of term magnitudes; a value whose terms are
    all zero must be exact."""
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    err = np.abs(np.asarray(x, np.float64) - ref)
    terms = np.asarray(terms, np.float64)
    assert (err[terms == 0] == 0).all(), "a value with no non-zero term is not exact"
    nz = terms > 0
    return float((err[nz] / terms[nz]).max()) if nz.any() else 0.0


def plain_rel_err(x, ref, terms, floor):
    """max |x - ref| / |ref| over the values with |ref| >= floor * T."""
    ref = np.asarray(ref, np.float64)
    m = np.abs(ref) >= floor * np.asarray(terms, np.float64)
    m &= ref != 0
    if not m.any():
        return 0.0
    return float((np.abs(np.asarray(x, np.float64)[m] - ref[m]) / np.abs(ref[m])).max())


def float_errors(x, ref, terms, name):
    """The contract's errors of one float output: scaled, and plain relative at each floor."""
    out = {f"{name}_scaled": scaled_err(x, ref, terms)}
    for f in REPORT_FLOORS:
        out[f"{name}_plain@{f:g}"] = plain_rel_err(x, ref, terms, f)
    return out


def check_floats(got_dE, got_g, dump, where):
    """Assert the float contract on dE and g against the oracle's dump; returns the errors."""
    e = float_errors(got_dE, dump["dE"], dump["dE_terms"], "dE")
    e.update(float_errors(got_g, dump["g"], dump["g_terms"], "g"))
    for name in ("dE", "g"):
        assert e[f"{name}_scaled"] <= REL_TOL, (where, name, "outside 1e-5 of its term sum", e)
        assert e[f"{name}_plain@{PLAIN_FLOOR:g}"] <= REL_TOL, (where, name, "plain relative error", e)
    return e


def record(label, errors):
    """Keep the largest error of each kind per label (the test's workload)."""
    cur = ERRORS.setdefault(label, {"values": 0})
    for k, v in errors.items():
        if k == "n":
            cur["values"] += int(v)
        elif isinstance(v, float):
            cur[k] = max(cur.get(k, 0.0), v)


def write_report():
    path = os.environ.get("SEG_PARITY_REPORT")
    if path and ERRORS:
        with open(path, "w") as f:
            json.dump(ERRORS, f, indent=1, sort_keys=True)


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
    stats = check_floats(g["dE"], g["g"], dump, where)
    stats.update(fixed=int(fixed.sum()), n=int(g["idx"].size))
    record(label.split(" it")[0], stats)
    assert np.array_equal(ctx.labels(), run.L), (where, "labels differ")
    return st, stats
