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
