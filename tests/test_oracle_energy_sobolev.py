"""Pins of the oracle's particle extraction, energy differences and Eq. 6 sums."""
import math
import os

import numpy as np
import pytest
from scipy import ndimage

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _nbr_shifts(ndim):
    if ndim == 2:
        return [(-1, 0), (1, 0), (0, -1), (0, 1)]
    return [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def _shifted(L, off):
    """L moved by -off with -1 outside: out[x] = L[x + off]."""
    out = np.full(L.shape, -1, np.int64)
    src = tuple(slice(max(0, o), L.shape[i] + min(0, o)) for i, o in enumerate(off))
    dst = tuple(slice(max(0, -o), L.shape[i] + min(0, -o)) for i, o in enumerate(off))
    out[dst] = L[src]
    return out


def _brute_particles(L):
    keys = set()
    flat = L.reshape(-1)
    for off in _nbr_shifts(L.ndim):
        nb = _shifted(L, off).reshape(-1)
        m = (nb >= 0) & (nb != flat)
        for i in np.nonzero(m)[0]:
            keys.add((int(i), int(flat[i]), int(nb[i])))
    return sorted(keys)


def test_square_start_has_508_particles(orc):
    L = np.zeros((128, 128), np.int32)
    L[32:96, 32:96] = 1
    I = np.zeros(L.shape, np.float32)
    idx, l, c = orc.extract(orc.make_params(I, L), L)
    assert idx.size == 508
    assert (l == 1).sum() == 4 * 64 - 4 and (l == 0).sum() == 4 * 64


@pytest.mark.parametrize("shape,labels", [((23, 31), 4), ((7, 9, 11), 5), ((1, 13), 3), ((5, 1, 6), 2)])
def test_extract_matches_brute_force(orc, shape, labels):
    rng = np.random.default_rng(sum(shape))
    L = rng.integers(0, labels, shape).astype(np.int32)
    I = np.zeros(shape, np.float32)
    p = orc.make_params(I, L)
    idx, l, c = orc.extract(p, L)
    got = list(zip(idx.tolist(), l.tolist(), c.tolist()))
    assert got == _brute_particles(L)          # same set, ascending (pixel, candidate) order


def _perimeter(L):
    P = 0
    for ax in range(L.ndim):
        a = np.swapaxes(L, 0, ax)
        P += int((a[1:] != a[:-1]).sum())
    return P


def _sse(I, L, M):
    tot = 0.0
    for m in range(M):
        v = I[L == m].astype(np.float64)
        if v.size:
            tot += float(((v - v.mean()) ** 2).sum())
    return tot


@pytest.mark.parametrize("dtype,shape", [(np.float32, (12, 15)), (np.uint16, (12, 15)), (np.float32, (5, 6, 7))])
def test_pc_energy_is_brute_force_sse_change(orc, dtype, shape):
    rng = np.random.default_rng(7)
    if dtype == np.float32:
        I = rng.normal(1.0, 0.5, shape).astype(np.float32)
    else:
        I = rng.integers(50, 400, shape).astype(np.uint16)
    L = rng.integers(0, 3, shape).astype(np.int32)
    M = 3
    p = orc.make_params(I, L, "pc", lam=0.0, nlabels=M)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    base = _sse(I, L, M)
    scale = float((I.astype(np.float64) ** 2).sum()) + 1.0
    for k in range(0, idx.size, 3):
        L2 = L.copy().reshape(-1)
        L2[idx[k]] = c[k]
        ref = _sse(I, L2.reshape(shape), M) - base
        assert abs(dE[k] - ref) <= 1e-11 * scale, (k, dE[k], ref)


@pytest.mark.parametrize("shape", [(14, 17), (6, 7, 8)])
def test_length_term_is_perimeter_recount(orc, shape):
    rng = np.random.default_rng(8)
    I = rng.normal(0, 1, shape).astype(np.float32)
    L = rng.integers(0, 3, shape).astype(np.int32)
    p0 = orc.make_params(I, L, "pc", lam=0.0)
    p1 = orc.make_params(I, L, "pc", lam=1.0)
    idx, l, c = orc.extract(p0, L)
    d0 = orc.energy(p0, I, L, idx, l, c)
    d1 = orc.energy(p1, I, L, idx, l, c)
    P = _perimeter(L)
    for k in range(idx.size):
        L2 = L.copy().reshape(-1)
        L2[idx[k]] = c[k]
        dP = _perimeter(L2.reshape(shape)) - P
        assert orc.delta_perimeter(p0, L, int(idx[k]), int(l[k]), int(c[k])) == dP
        assert d1[k] - d0[k] == pytest.approx(dP, abs=1e-9)


def _ball(R, ndim):
    r = int(math.floor(R))
    grids = np.mgrid[tuple(slice(-r, r + 1) for _ in range(ndim))]
    return (sum(g.astype(np.int64) ** 2 for g in grids) <= R * R).astype(np.float64)


@pytest.mark.parametrize("shape,R", [((20, 23), 3.0), ((20, 23), 8.0), ((7, 8, 9), 2.5)])
def test_ps_energy_matches_convolution(orc, shape, R):
    # local means over a ball via scipy convolutions of the label indicators
    rng = np.random.default_rng(9)
    I = rng.uniform(0.2, 2.0, shape).astype(np.float32)
    L = rng.integers(0, 3, shape).astype(np.int32)
    p = orc.make_params(I, L, "ps", lam=0.0, ps_radius=R)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    fp = _ball(R, I.ndim)
    Id = I.astype(np.float64)
    sums, cnts = {}, {}
    for m in range(3):
        ind = (L == m).astype(np.float64)
        sums[m] = ndimage.convolve(ind * Id, fp, mode="constant", cval=0.0).reshape(-1)
        cnts[m] = ndimage.convolve(ind, fp, mode="constant", cval=0.0).reshape(-1)
    v = Id.reshape(-1)
    for k in range(idx.size):
        x = idx[k]
        mc = sums[int(c[k])][x] / cnts[int(c[k])][x]
        ml = sums[int(l[k])][x] / cnts[int(l[k])][x]
        ref = (v[x] - mc) ** 2 - (v[x] - ml) ** 2
        assert dE[k] == pytest.approx(ref, rel=1e-10, abs=1e-10)


def test_ps_large_radius_is_region_mean_difference(orc):
    rng = np.random.default_rng(10)
    I = rng.uniform(0.0, 3.0, (9, 11)).astype(np.float32)
    L = rng.integers(0, 3, I.shape).astype(np.int32)
    p = orc.make_params(I, L, "ps", lam=0.0, ps_radius=50.0)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    means = [I[L == m].astype(np.float64).mean() for m in range(3)]
    v = I.astype(np.float64).reshape(-1)
    ref = (v[idx] - np.take(means, c)) ** 2 - (v[idx] - np.take(means, l)) ** 2
    assert np.allclose(dE, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape,cutoff,labels", [((19, 23), 3.0, 3), ((19, 23), 5.0, 4), ((9, 10, 11), 2.5, 3),
                                                 ((9, 10, 11), 4.0, 5), ((1, 40), 3.0, 2)])
def test_sobolev_cell_list_equals_all_pairs(orc, shape, cutoff, labels):
    rng = np.random.default_rng(int(cutoff * 10) + len(shape))
    L = rng.integers(0, labels, shape).astype(np.int32)
    I = np.zeros(shape, np.float32)
    p = orc.make_params(I, L, cutoff=cutoff)
    idx, l, c = orc.extract(p, L)
    dE = rng.normal(0, 1, idx.size)
    g1, A1, B1, n1, m1 = orc.sobolev(p, idx, l, c, dE, all_pairs=False)
    g2, A2, B2, n2, m2 = orc.sobolev(p, idx, l, c, dE, all_pairs=True)
    assert np.array_equal(g1, g2) and np.array_equal(n1, n2) and np.array_equal(m1, m2)
    # every particle sees itself in its own set
    assert (n1 >= 1).all()


def test_sobolev_set_sizes_by_brute_force(orc):
    rng = np.random.default_rng(12)
    L = rng.integers(0, 3, (15, 16)).astype(np.int32)
    p = orc.make_params(np.zeros(L.shape, np.float32), L, cutoff=3.5)
    idx, l, c = orc.extract(p, L)
    dE = np.ones(idx.size)
    _, _, _, nQ, nQp = orc.sobolev(p, idx, l, c, dE)
    y, x = np.divmod(idx.astype(np.int64), L.shape[1])
    d2 = (y[:, None] - y[None, :]) ** 2 + (x[:, None] - x[None, :]) ** 2
    near = d2 < 3.5 ** 2
    assert np.array_equal(nQ, (near & (l[None, :] == l[:, None])).sum(1))
    assert np.array_equal(nQp, (near & (c[None, :] == l[:, None])).sum(1))


def test_sobolev_straight_line_golden(orc):
    vals = {}
    for line in open(os.path.join(GOLD, "sobolev_line.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    L = np.zeros((12, 40), np.int32)
    L[:6] = 1                       # inner row 5 (label 1), outer row 6 (label 0)
    p = orc.make_params(np.zeros(L.shape, np.float32), L, cutoff=3.0)
    idx, l, c = orc.extract(p, L)
    g, A, B, nQ, nQp = orc.sobolev(p, idx, l, c, np.ones(idx.size))
    k = int(np.nonzero(idx == 5 * 40 + 20)[0][0])
    assert nQ[k] == vals["nQ"] and nQp[k] == vals["nQp"]
    assert A[k] == pytest.approx(vals["A"], abs=1e-15)
    assert B[k] == pytest.approx(vals["B"], abs=1e-15)
    assert g[k] == pytest.approx(vals["g"], abs=1e-15)


@pytest.mark.parametrize("cutoff", [1.0, 0.75])
def test_degenerate_cutoff_is_rescaled_l2(orc, cutoff):
    # cutoff <= 1: only the particle itself lies closer than E/2 (two labels: one particle per pixel),
    # so Eq. 6 gives K(0) dE = (3/E) dE.
    rng = np.random.default_rng(13)
    I = rng.normal(0.5, 0.4, (24, 26)).astype(np.float32)
    L = np.zeros(I.shape, np.int32)
    L[6:18, 5:20] = 1
    p = orc.make_params(I, L, "pc", lam=0.04, cutoff=cutoff)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    g, A, B, nQ, nQp = orc.sobolev(p, idx, l, c, dE)
    assert (nQ == 1).all() and (nQp == 0).all()
    E = 2 * cutoff
    assert np.allclose(g, (3.0 / E) * dE, rtol=1e-15, atol=0)


# ---- the tolerance scale: sums of term magnitudes ----

def _region_sse(v):
    v = np.asarray(v, np.float64)
    return float(((v - v.mean()) ** 2).sum()) if v.size else 0.0


@pytest.mark.parametrize("dtype,shape,lam", [(np.float32, (11, 13), 0.3), (np.uint16, (10, 12), 40.0),
                                             (np.float32, (5, 6, 7), 0.2)])
def test_pc_terms_are_brute_force_region_changes(orc, dtype, shape, lam):
    # The PC energy difference adds two region terms and the length term: the increase of
    # region c's squared deviations when v joins it, minus the decrease of region l's when v
    # leaves it, plus lambda * dP. Each is recomputed here by brute force from the pixels.
    rng = np.random.default_rng(17)
    I = (rng.normal(1.0, 0.5, shape).astype(np.float32) if dtype == np.float32
         else rng.integers(50, 400, shape).astype(np.uint16))
    L = rng.integers(0, 3, shape).astype(np.int32)
    p = orc.make_params(I, L, "pc", lam=lam, nlabels=3)
    idx, l, c = orc.extract(p, L)
    dE, terms = orc.energy(p, I, L, idx, l, c, with_terms=True)
    flat_I = I.reshape(-1).astype(np.float64)
    flat_L = L.reshape(-1)
    P = _perimeter(L)
    for k in range(0, idx.size, 2):
        x, lk, ck = int(idx[k]), int(l[k]), int(c[k])
        in_c, in_l = flat_I[flat_L == ck], flat_I[flat_L == lk]
        t1 = _region_sse(np.append(in_c, flat_I[x])) - _region_sse(in_c)
        rest = flat_I[(flat_L == lk) & (np.arange(flat_L.size) != x)]
        t2 = _region_sse(in_l) - _region_sse(rest)
        L2 = flat_L.copy()
        L2[x] = ck
        dP = _perimeter(L2.reshape(shape)) - P
        ref = abs(t1) + abs(t2) + abs(lam * dP)
        tol = 1e-10 * (float((flat_I ** 2).sum()) + 1.0)
        assert terms[k] == pytest.approx(ref, abs=tol), (k, terms[k], ref)
        assert terms[k] >= abs(dE[k]) - tol


@pytest.mark.parametrize("model", ["ps", "psp"])
def test_ps_terms_from_convolved_local_means(orc, model):
    # PS: (v - m_c)^2 + (v - m_l)^2; Poisson: m_c + |v ln m_c| + m_l + |v ln m_l| (means floored),
    # with the local means from scipy convolutions of the label indicators; plus lambda |dP|
    rng = np.random.default_rng(19)
    shape, R, lam = (18, 21), 3.0, 0.05
    I = rng.uniform(0.2, 2.0, shape).astype(np.float32)
    L = rng.integers(0, 3, shape).astype(np.int32)
    p = orc.make_params(I, L, model, lam=lam, ps_radius=R)
    idx, l, c = orc.extract(p, L)
    dE, terms = orc.energy(p, I, L, idx, l, c, with_terms=True)
    fp = _ball(R, 2)
    Id = I.astype(np.float64)
    sums = {m: ndimage.convolve((L == m) * Id, fp, mode="constant").reshape(-1) for m in range(3)}
    cnts = {m: ndimage.convolve((L == m).astype(np.float64), fp, mode="constant").reshape(-1) for m in range(3)}
    v = Id.reshape(-1)
    P = _perimeter(L)
    for k in range(idx.size):
        x = int(idx[k])
        mc = sums[int(c[k])][x] / cnts[int(c[k])][x]
        ml = sums[int(l[k])][x] / cnts[int(l[k])][x]
        if model == "ps":
            data_terms = (v[x] - mc) ** 2 + (v[x] - ml) ** 2
        else:
            mc, ml = max(mc, p.mu_floor), max(ml, p.mu_floor)
            data_terms = mc + abs(v[x] * math.log(mc)) + ml + abs(v[x] * math.log(ml))
        L2 = L.copy().reshape(-1)
        L2[x] = c[k]
        dP = _perimeter(L2.reshape(shape)) - P
        assert terms[k] == pytest.approx(data_terms + abs(lam * dP), rel=1e-9, abs=1e-12)


def test_sobolev_terms_straight_line_golden(orc):
    # every dE = 1 on the straight contour: no term cancels, so the term sum is A + B of the
    # hand-worked golden values
    vals = {}
    for line in open(os.path.join(GOLD, "sobolev_line.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, val = line.split()
            vals[k] = float(val)
    L = np.zeros((12, 40), np.int32)
    L[:6] = 1
    p = orc.make_params(np.zeros(L.shape, np.float32), L, cutoff=3.0)
    idx, l, c = orc.extract(p, L)
    *_, terms = orc.sobolev(p, idx, l, c, np.ones(idx.size), with_terms=True)
    k = int(np.nonzero(idx == 5 * 40 + 20)[0][0])
    assert terms[k] == pytest.approx(vals["A"] + vals["B"], abs=1e-15)


def test_sobolev_terms_by_brute_force_sets(orc):
    # sum over Q of |K dE_q| / |Q| plus the same over Q', the sets and K found here by brute
    # force over all particle pairs with numpy; signed energy differences so that terms cancel
    rng = np.random.default_rng(23)
    L = rng.integers(0, 3, (17, 19)).astype(np.int32)
    cutoff = 3.5
    p = orc.make_params(np.zeros(L.shape, np.float32), L, cutoff=cutoff)
    idx, l, c = orc.extract(p, L)
    dE = rng.normal(0, 1, idx.size)
    g, A, B, nQ, nQp, terms = orc.sobolev(p, idx, l, c, dE, with_terms=True)
    y, x = np.divmod(idx.astype(np.int64), L.shape[1])
    d2 = (y[:, None] - y[None, :]) ** 2 + (x[:, None] - x[None, :]) ** 2
    near = d2 < cutoff ** 2
    E = 2 * cutoff
    K = (3.0 / E) * (1.0 - 2.0 * np.sqrt(d2) / E) ** 2
    inQ = near & (l[None, :] == l[:, None])
    inQp = near & (c[None, :] == l[:, None])
    w = np.abs(K * dE[None, :])
    ref = (w * inQ).sum(1) / inQ.sum(1) + np.where(inQp.sum(1) > 0, (w * inQp).sum(1) / np.maximum(inQp.sum(1), 1), 0)
    assert np.allclose(terms, ref, rtol=1e-12, atol=0)
    assert (terms >= np.abs(g) * (1 - 1e-12)).all()
    assert (terms > 2 * np.abs(g)).any(), "the case should contain cancelling terms"


def test_oscillation_rule_golden(orc):
    # hand-worked accepted-move sequences (tests/golden/osc_switch.txt)
    n = 0
    for line in open(os.path.join(GOLD, "osc_switch.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, grad, window, acc, modes, conv = line.split()
        acc = [int(t) for t in acc.split(",")]
        want = list(zip([int(t) for t in modes.split(",")], [int(t) for t in conv.split(",")]))
        got = orc.mode_sequence(int(window), acc, gradient=int(grad))
        assert got == want, (name, got, want)
        n += 1
    assert n >= 7
