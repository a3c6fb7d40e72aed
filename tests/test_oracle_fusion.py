"""The oracle's fusion event (topology bit 4, piecewise-constant model): touching foreground
regions a < b fuse after the moves when dE = n_a n_b/(n_a + n_b) (mu_a - mu_b)^2 - lambda B_ab < 0,
greedily in ascending (dE, a, b), each label at most once per iteration.

Pins: the pair list and B_ab against a perimeter recount (P before minus P after renaming b to a),
dE against a brute-force recompute of the total energy (sum of squared deviations about the
region means plus lambda times the perimeter) before and after the fusion, the pass against a
greedy matching over brute-force energies (a matching, maximal, the global minimum taken first),
and the total energy falling."""
import numpy as np
import pytest


def _blocks(H=48, W=64, pitch=16, border=True, seed=0, sigma=0.05, levels=None):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[:H, :W]
    ncol = (W + pitch - 1) // pitch
    L = (1 + (yy // pitch) * ncol + (xx // pitch)).astype(np.int32)
    if border:
        L[:2], L[-2:], L[:, :2], L[:, -2:] = 0, 0, 0, 0
    M = int(L.max()) + 1
    lev = rng.uniform(0.0, 1.0, M) if levels is None else np.asarray(levels, np.float64)
    I = (lev[L] + rng.normal(0.0, sigma, L.shape)).astype(np.float32)
    return I, L


def _energy(I, L, lam, orc, p):
    I = I.astype(np.float64)
    E = 0.0
    for m in np.unique(L):
        v = I[L == m]
        E += float(((v - v.mean()) ** 2).sum())
    return E + lam * orc.perimeter(p, L)


def test_pairs_and_shared_boundary_by_perimeter_recount(orc):
    I, L = _blocks(seed=1)
    L[20:30, 30:40] = 0                               # a background hole breaks some contacts
    p = orc.make_params(I, L, "pc", lam=0.1, topology=4)
    a, b, B = orc.fuse_pairs(p, L)
    assert (a < b).all() and (a > 0).all()
    keys = list(zip(a.tolist(), b.tolist()))
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    ref = set()
    for ax in range(L.ndim):
        u = np.moveaxis(L, ax, 0)
        x, y = u[:-1].ravel(), u[1:].ravel()
        m = (x != y) & (x > 0) & (y > 0)
        ref |= {(min(s, t), max(s, t)) for s, t in zip(x[m].tolist(), y[m].tolist())}
    assert set(keys) == ref
    P0 = orc.perimeter(p, L)
    for (s, t), Bst in zip(keys, B.tolist()):
        L2 = np.where(L == t, s, L).astype(np.int32)
        assert P0 - orc.perimeter(p, L2) == Bst


@pytest.mark.parametrize("lam", [0.0, 0.05, 2.0])
def test_fuse_energy_matches_brute_force(orc, lam):
    I, L = _blocks(seed=2, sigma=0.2)
    p = orc.make_params(I, L, "pc", lam=lam, topology=4)
    n, S, _ = orc.stats(p, I, L)
    E0 = _energy(I, L, lam, orc, p)
    a, b, B = orc.fuse_pairs(p, L)
    for s, t, Bst in zip(a.tolist(), b.tolist(), B.tolist()):
        dE = orc.fuse_energy(p, n, S, s, t, Bst)
        L2 = np.where(L == t, s, L).astype(np.int32)
        ref = _energy(I, L2, lam, orc, p) - E0
        assert abs(dE - ref) <= 1e-9 * (abs(E0) + 1.0), (s, t, dE, ref)


def test_fusion_pass_is_the_greedy_matching(orc):
    # half the blocks share a level with a neighbour: those pairs fuse, contrasted ones do not
    I, L = _blocks(H=64, W=80, seed=3, sigma=0.05, levels=[0.0] + [0.2 * (k // 2) for k in range(40)])
    lam = 0.02
    p = orc.make_params(I, L, "pc", lam=lam, topology=4)
    n, S, _ = orc.stats(p, I, L)
    a, b, B = orc.fuse_pairs(p, L)
    E0 = _energy(I, L, lam, orc, p)
    cand = []
    for s, t, Bst in zip(a.tolist(), b.tolist(), B.tolist()):
        L2 = np.where(L == t, s, L).astype(np.int32)
        dE = _energy(I, L2, lam, orc, p) - E0
        if dE < -1e-9:
            cand.append((dE, s, t))
    cand.sort()
    used, want = set(), {}
    for dE, s, t in cand:
        if s in used or t in used:
            continue
        used |= {s, t}
        want[t] = s
    assert len(want) >= 5
    L1, nf = orc.fuse(p, I, L)
    assert nf == len(want)
    ref = L.copy()
    for t, s in want.items():
        ref[L == t] = s
    assert np.array_equal(L1, ref)
    assert _energy(I, L1, lam, orc, p) < E0
    # maximal: no negative pair is left between two untouched labels
    for dE, s, t in cand:
        assert s in used or t in used


def test_contrasted_regions_do_not_fuse(orc):
    I, L = _blocks(seed=4, sigma=0.01, levels=np.arange(40) * 1.0)
    p = orc.make_params(I, L, "pc", lam=0.01, topology=4)
    L1, nf = orc.fuse(p, I, L)
    assert nf == 0 and np.array_equal(L1, L)


def test_fusion_in_3d(orc):
    rng = np.random.default_rng(5)
    zz, yy, xx = np.mgrid[:12, :16, :16]
    L = (1 + (zz // 6) * 4 + (yy // 8) * 2 + (xx // 8)).astype(np.int32)
    lev = np.array([0.0] + [1.0, 1.0, 5.0, 5.0, 1.0, 1.0, 5.0, 5.0])
    I = (lev[L] + rng.normal(0, 0.05, L.shape)).astype(np.float32)
    p = orc.make_params(I, L, "pc", 6, lam=0.01, topology=4)
    n, S, _ = orc.stats(p, I, L)
    a, b, B = orc.fuse_pairs(p, L)
    P0 = orc.perimeter(p, L)
    for s, t, Bst in zip(a.tolist(), b.tolist(), B.tolist()):
        assert P0 - orc.perimeter(p, np.where(L == t, s, L).astype(np.int32)) == Bst
    L1, nf = orc.fuse(p, I, L)
    assert nf >= 2
    assert _energy(I, L1, 0.01, orc, p) < _energy(I, L, 0.01, orc, p)


@pytest.mark.parametrize("topology", [4, 7])
def test_iterations_with_fusion_keep_one_component_per_label(orc, topology):
    from scipy import ndimage
    I, L = _blocks(H=64, W=80, seed=6, sigma=0.1, levels=[0.0] + [0.5 * (k // 2) for k in range(40)])
    p = orc.make_params(I, L, "pc", lam=0.05, cutoff=3.0, topology=topology)
    run = orc.Run(p, I, L)
    labels0 = len(np.unique(L))
    for _ in range(10):
        run.step()
        for m in np.unique(run.L):
            if m == 0:
                continue
            assert ndimage.label(run.L == m)[1] == 1
    assert len(np.unique(run.L)) < labels0
