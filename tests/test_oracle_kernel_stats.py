"""Pins of the oracle's Sobolev kernel (Eq. 5) and exact region statistics."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            out.append(line.split())
    return out


def test_kernel_closed_form_at_eps_1_24(orc):
    # Eq. 5 with eps = 1/24 equals (3/E)(1 - 2|r|/E)^2 on [-E/2, E/2].
    for E in (2.0, 6.0, 8.0, 10.0, 12.0):
        for r in np.linspace(-E / 2, E / 2, 41):
            k = orc.kernel_eq5(float(r), E, 1.0 / 24.0)
            ref = (3.0 / E) * (1.0 - 2.0 * abs(r) / E) ** 2
            assert abs(k - ref) <= 1e-14 * (3.0 / E)


def test_kernel_figure2_ticks(orc):
    # Figure 2: K*E vs r/E for eps = 1/24, 0.06, 0.08 (values worked from Eq. 5 by hand).
    for eps, rE, KE in _rows("kernel_fig2.txt"):
        eps, rE, KE = float(eps), float(rE), float(KE)
        E = 10.0
        got = orc.kernel_eq5(rE * E, E, eps) * E
        assert abs(got - KE) < 1e-13, (eps, rE, got, KE)


@pytest.mark.parametrize("eps", [1.0 / 24.0, 0.06, 0.08, 0.2])
def test_kernel_unit_mass(orc, eps):
    # the integral of (x^2 - |x| + 1/6) over [-1/2, 1/2] vanishes, so K has unit mass for any eps
    E = 8.0
    mass, _ = integrate.quad(lambda r: orc.kernel_eq5(r, E, eps), -E / 2, E / 2, points=[0.0])
    assert abs(mass - 1.0) < 1e-12


def test_kernel_symmetric_and_decreasing(orc):
    E = 10.0
    prev = None
    for r in np.linspace(0, E / 2, 51):
        k = orc.kernel_eq5(float(r), E, 1.0 / 24.0)
        assert k == orc.kernel_eq5(-float(r), E, 1.0 / 24.0)
        if prev is not None:
            assert k <= prev
        prev = k


def _wide_f32(rng, n):
    mant = rng.uniform(-1, 1, n)
    expo = rng.integers(-40, 40, n)
    v = (mant * np.exp2(expo)).astype(np.float32)
    v[::17] = 0.0
    v[::29] = np.float32(1e-42)      # subnormal
    return v


@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_matches_fsum(orc, seed):
    rng = np.random.default_rng(seed)
    v = _wide_f32(rng, 3000)
    # cancellation-heavy tail
    v = np.concatenate([v, -v[:1000], np.float32([3.0e30, 1.0, -3.0e30])])
    rng.shuffle(v)
    got = orc.exact_sum_f32(v)
    assert got == math.fsum(float(x) for x in v)
    exact = sum((Fraction(float(x)) for x in v), Fraction(0))
    assert got == float(exact)
    # squares: float64 products of float32 values are exact, fsum rounds their sum correctly
    got2 = orc.exact_sum_f32(v, squares=True)
    assert got2 == math.fsum(float(x) * float(x) for x in v)


def test_exact_sum_ties_round_to_even(orc):
    # 2^53 + 1 is a tie between 2^53 and 2^53 + 2: round half to even gives 2^53
    big = np.float32(2.0 ** 53)
    assert orc.exact_sum_f32(np.array([big, 1.0], np.float32)) == 2.0 ** 53
    assert orc.exact_sum_f32(np.array([big, 1.0, 1.0, 1.0], np.float32)) == 2.0 ** 53 + 4
    assert orc.exact_sum_f32(np.array([big, 2.0, 1.0], np.float32)) == 2.0 ** 53 + 4


def test_stats_partition_invariants(orc):
    rng = np.random.default_rng(3)
    I = rng.normal(0, 1, (37, 53)).astype(np.float32)
    L = rng.integers(0, 5, I.shape).astype(np.int32)
    p = orc.make_params(I, L)
    n, S, Q = orc.stats(p, I, L)
    assert n.sum() == I.size
    for m in range(5):
        vals = I[L == m].astype(np.float64)
        assert n[m] == vals.size
        assert S[m] == math.fsum(vals)
        assert Q[m] == math.fsum(vals * vals)
    assert math.fsum(S) == pytest.approx(math.fsum(I.astype(np.float64).ravel()), abs=1e-12)


def test_stats_u16_exact_integers(orc):
    rng = np.random.default_rng(4)
    I = rng.integers(0, 65536, (6, 17, 19)).astype(np.uint16)
    L = rng.integers(0, 4, I.shape).astype(np.int32)
    p = orc.make_params(I, L)
    n, S, Q = orc.stats(p, I, L)
    for m in range(4):
        v = I[L == m].astype(np.int64)
        assert S[m] == float(int(v.sum()))
        q = int((v * v).sum())
        assert Q[m] == float(Fraction(q))   # correctly rounded when above 2^53
