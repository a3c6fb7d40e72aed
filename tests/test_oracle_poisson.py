"""The oracle's Poisson-noise piecewise-smooth model (Methods: Poisson likelihood with the
local means as the model): its logarithm against the C library's, and its energy change
against an evaluation with scipy convolutions and numpy logarithms."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle


def test_log_matches_libm_within_4_ulp(orc):
    rng = np.random.default_rng(1)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 4000)), rng.uniform(0.5, 2.0, 4000),
                         [1.0, 2.0, 0.5, math.sqrt(0.5), math.sqrt(2.0), 1e-300, 5e-324, 1.7e308,
                          1.0 + 2 ** -52, 1.0 - 2 ** -53, 3.0, 10.0]])
    for x in xs:
        ref = math.log(float(x))
        got = oracle.log(float(x))
        assert abs(got - ref) <= 4 * math.ulp(ref) + 1e-300, (x, got, ref)
    assert oracle.log(1.0) == 0.0


def _ball(R, ndim):
    r = int(math.floor(R))
    grids = np.mgrid[tuple(slice(-r, r + 1) for _ in range(ndim))]
    return (sum(g.astype(np.int64) ** 2 for g in grids) <= R * R).astype(np.float64)


@pytest.mark.parametrize("shape,R", [((20, 23), 3.0), ((20, 23), 8.0), ((7, 8, 9), 2.5)])
def test_poisson_energy_matches_convolution(orc, shape, R):
    rng = np.random.default_rng(19)
    # Poisson counts with zero patches, so that floored means occur
    I = rng.poisson(rng.uniform(0.0, 6.0, shape)).astype(np.float32)
    I[: shape[0] // 3] = 0.0
    L = rng.integers(0, 3, shape).astype(np.int32)
    lam = 0.3
    p = orc.make_params(I, L, "psp", lam=lam, ps_radius=R)
    floor = math.ldexp(max(1.0, float(I.max())), -20)
    assert p.mu_floor == floor
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

    def f(vx, mu):
        m = max(mu, floor)
        return m - vx * np.log(m)

    for k in range(idx.size):
        x = int(idx[k])
        mc = sums[int(c[k])][x] / cnts[int(c[k])][x]
        ml = sums[int(l[k])][x] / cnts[int(l[k])][x]
        dP = orc.delta_perimeter(p, L, x, int(l[k]), int(c[k]))
        ref = f(v[x], mc) - f(v[x], ml) + lam * dP
        assert dE[k] == pytest.approx(ref, rel=1e-10, abs=1e-9)


def test_poisson_prefers_the_region_whose_mean_fits(orc):
    # a pixel of value 9 between a region of mean ~9 and one of mean ~1 gains by joining the first
    I = np.ones((10, 10), np.float32)
    I[:, 5:] = 9.0
    L = np.zeros((10, 10), np.int32)
    L[:, 5:] = 1
    L[4, 5] = 0                     # a bright pixel held by the dark region
    p = orc.make_params(I, L, "psp", lam=0.0, ps_radius=3.0)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    k = [i for i in range(idx.size) if idx[i] == 4 * 10 + 5 and c[i] == 1]
    assert len(k) == 1 and dE[k[0]] < 0
