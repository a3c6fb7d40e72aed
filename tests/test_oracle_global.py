"""The oracle's Sobolev step with the length scale set to the contour length (E = |Gamma|,
Length scale section; all particle pairs considered), pinned against an independent numpy
evaluation of Eq. 6, and |Gamma| against perimeter counts."""
import numpy as np
import pytest

import oracle


def _perimeter_np(L):
    return int(sum(np.count_nonzero(np.diff(L, axis=a)) for a in range(L.ndim)))


def test_perimeter_of_square_cube_and_random(orc):
    L = np.zeros((20, 30), np.int32)
    L[4:11, 5:14] = 1
    p = oracle.make_params(np.zeros(L.shape, np.float32), L)
    assert oracle.perimeter(p, L) == 2 * (7 + 9)
    V = np.zeros((9, 10, 11), np.int32)
    V[2:6, 3:6, 1:8] = 2
    p3 = oracle.make_params(np.zeros(V.shape, np.uint16), V, nlabels=3)
    assert oracle.perimeter(p3, V) == 2 * (3 * 7 + 4 * 7 + 4 * 3)
    rng = np.random.default_rng(5)
    R = rng.integers(0, 4, size=(13, 17)).astype(np.int32)
    assert oracle.perimeter(oracle.make_params(np.zeros(R.shape, np.float32), R), R) == _perimeter_np(R)


def _eq6_global_np(idx, l, c, dE, shape, E):
    """Eq. 6 over all pairs with |d| < E/2 and the eps = 1/24 kernel in closed form,
    K(r) = (3/E)(1 - 2r/E)^2, in plain numpy."""
    H, W = shape
    y, x = np.divmod(idx.astype(np.int64), W)
    d = np.sqrt((y[:, None] - y[None, :]) ** 2 + (x[:, None] - x[None, :]) ** 2)
    inside = d < E / 2
    K = 3.0 / E * (1.0 - 2.0 * d / E) ** 2
    same = (l[None, :] == l[:, None]) & inside
    other = (c[None, :] == l[:, None]) & inside
    nA, nB = same.sum(1), other.sum(1)
    A = np.where(nA > 0, (K * same * dE[None, :]).sum(1) / np.maximum(nA, 1), 0.0)
    B = np.where(nB > 0, (K * other * dE[None, :]).sum(1) / np.maximum(nB, 1), 0.0)
    return A - B, nA, nB


@pytest.mark.parametrize("seed", [0, 1])
def test_global_length_scale_step_is_eq6_over_all_pairs(orc, seed):
    rng = np.random.default_rng(seed)
    H, W = 26, 31
    I = rng.normal(0.0, 0.3, (H, W)).astype(np.float32)
    I[5:15, 6:20] += 1.0
    L = np.zeros((H, W), np.int32)
    L[7:13, 8:16] = 1
    L[16:22, 20:27] = 2
    p = oracle.make_params(I, L, "pc", lam=0.04, gradient="sobolev_global")
    run = oracle.Run(p, I, L)
    E = float(oracle.perimeter(p, L))
    st, dump = run.step(dump=True)
    assert st["mode_used"] == oracle.SOBOLEV_GLOBAL
    g_np, nA, nB = _eq6_global_np(dump["idx"], dump["l"], dump["c"], dump["dE"], (H, W), E)
    scale = np.abs(dump["g"]) + np.abs(g_np) + 1e-300
    assert np.max(np.abs(dump["g"] - g_np) / scale) < 1e-12
    # E/2 here exceeds most pair distances: far more partners than a local cutoff gives
    assert nA.mean() > 20


def test_global_mode_switches_to_l2(orc):
    rng = np.random.default_rng(3)
    I = rng.normal(0.0, 0.3, (24, 24)).astype(np.float32)
    I[6:18, 6:18] += 1.0
    L = np.zeros((24, 24), np.int32)
    L[9:15, 9:15] = 1
    p = oracle.make_params(I, L, "pc", lam=0.04, gradient="sobolev_global", osc_window=2)
    run = oracle.Run(p, I, L)
    modes = [run.step()[0]["mode_used"] for _ in range(8)]
    assert modes[0] == oracle.SOBOLEV_GLOBAL and oracle.L2 in modes
    assert modes.index(oracle.L2) > 0 and all(m == oracle.L2 for m in modes[modes.index(oracle.L2):])
