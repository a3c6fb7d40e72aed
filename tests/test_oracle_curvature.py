"""The oracle's curvature regulariser (ball counts A_l - A_c with weight lambda 3/(2 rho^3) in 2D,
lambda 4/(pi rho^4) in 3D, from the integral invariants of a ball centred on a boundary).

Pins: the exact count on a straight edge (half-plane / half-space: only the ball's central row
or plane is unbalanced), the curvature of digital disks and spheres recovered from the energy
differences of the inner and outer boundary particles (a wrong constant, power or sign in the
weight fails), the image border (pixels outside count for neither label), and a brute-force
count on random label images."""
import math

import numpy as np
import pytest


def _const_image(shape):
    return np.zeros(shape, np.float32)       # the data term vanishes: dE is the regulariser alone


@pytest.mark.parametrize("rho", [4.0, 5.5, 7.0])
def test_straight_edge_counts_the_central_row(orc, rho):
    H, W = 48, 48
    L = np.zeros((H, W), np.int32)
    L[:24] = 1
    p = orc.make_params(_const_image((H, W)), L, "pc", lam=1.0, curv_radius=rho)
    row = sum(1 for dx in range(-10, 11) if dx * dx <= rho * rho)
    assert row == 2 * int(math.floor(rho)) + 1
    for x in (16, 24, 31):
        assert orc.ball_balance(p, L, 23 * W + x, 1, 0) == row      # inside, towards the background
        assert orc.ball_balance(p, L, 24 * W + x, 0, 1) == row      # outside, towards the region


def test_straight_plane_counts_the_central_disk(orc):
    rho = 4.5
    D = H = W = 24
    L = np.zeros((D, H, W), np.int32)
    L[:12] = 1
    p = orc.make_params(_const_image((D, H, W)), L, "pc", lam=1.0, curv_radius=rho)
    disk = sum(1 for dy in range(-5, 6) for dx in range(-5, 6) if dy * dy + dx * dx <= rho * rho)
    for (y, x) in [(12, 12), (9, 14)]:
        assert orc.ball_balance(p, L, (11 * H + y) * W + x, 1, 0) == disk
        assert orc.ball_balance(p, L, (12 * H + y) * W + x, 0, 1) == disk


def _boundary_curvature(orc, L, rho, lam=0.5):
    """(mean dE of the outer particles - mean dE of the inner ones) / (2 lambda): the straight-edge
    offset of both sides cancels, leaving the curvature of the region at its boundary."""
    p = orc.make_params(_const_image(L.shape), L, "pc", lam=lam, curv_radius=rho)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, _const_image(L.shape), L, idx, l, c)
    inner = dE[l == 1]
    outer = dE[l == 0]
    assert inner.size > 50 and outer.size > 50
    return (outer.mean() - inner.mean()) / (2.0 * lam)


@pytest.mark.parametrize("R0", [25.0, 50.0])
def test_disk_curvature_is_one_over_the_radius(orc, R0):
    n = int(2 * R0 + 40)
    yy, xx = np.mgrid[:n, :n]
    L = (((yy - n / 2 + 0.5) ** 2 + (xx - n / 2 + 0.5) ** 2) <= R0 * R0).astype(np.int32)
    kappa = _boundary_curvature(orc, L, rho=8.0)
    assert abs(kappa - 1.0 / R0) <= 0.12 / R0, (kappa, 1.0 / R0)


def test_sphere_curvature_is_two_over_the_radius(orc):
    R0 = 14.0
    n = 40
    zz, yy, xx = np.mgrid[:n, :n, :n]
    c = n / 2 - 0.5
    L = (((zz - c) ** 2 + (yy - c) ** 2 + (xx - c) ** 2) <= R0 * R0).astype(np.int32)
    H = _boundary_curvature(orc, L, rho=5.0)
    assert abs(H - 2.0 / R0) <= 0.15 * 2.0 / R0, (H, 2.0 / R0)


def test_weight_scales_with_lambda_and_radius(orc):
    L = np.zeros((30, 30), np.int32)
    L[:15] = 1
    I = _const_image(L.shape)
    w = [orc.curvature_weight(orc.make_params(I, L, "pc", lam=lam, curv_radius=r))
         for lam, r in [(1.0, 4.0), (2.0, 4.0), (1.0, 8.0)]]
    assert w[1] == 2.0 * w[0]
    assert abs(w[0] / w[2] - 8.0) <= 1e-15 * 8.0                  # rho^-3 in 2D
    L3 = np.zeros((12, 12, 12), np.int32)
    L3[:6] = 1
    w3 = [orc.curvature_weight(orc.make_params(_const_image(L3.shape), L3, "pc", lam=1.0, curv_radius=r))
          for r in (2.0, 4.0)]
    assert abs(w3[0] / w3[1] - 16.0) <= 1e-15 * 16.0              # rho^-4 in 3D


def test_balance_matches_brute_force_with_borders(orc):
    rng = np.random.default_rng(4)
    for shape, rho in [((17, 23), 3.3), ((7, 9, 8), 2.5)]:
        L = rng.integers(0, 4, shape).astype(np.int32)
        p = orc.make_params(_const_image(shape), L, "pc", lam=1.0, curv_radius=rho)
        R = int(rho)
        for xi in range(0, L.size, 7):
            pos = np.unravel_index(xi, shape)
            l = int(L[pos])
            c = (l + 1 + xi % 3) % 4
            bal = 0
            for d in np.ndindex(*([2 * R + 1] * len(shape))):
                off = np.array(d) - R
                if (off ** 2).sum() > rho * rho:
                    continue
                q = np.array(pos) + off
                if (q < 0).any() or (q >= np.array(shape)).any():
                    continue
                m = L[tuple(q)]
                bal += int(m == l) - int(m == c)
            assert orc.ball_balance(p, L, xi, l, c) == bal


def test_energy_is_data_plus_weighted_balance(orc):
    rng = np.random.default_rng(6)
    I = rng.normal(1.0, 0.5, (32, 40)).astype(np.float32)
    L = np.zeros(I.shape, np.int32)
    L[8:24, 10:30] = 1
    p0 = orc.make_params(I, L, "pc", lam=0.0)
    p1 = orc.make_params(I, L, "pc", lam=0.3, curv_radius=4.0)
    idx, l, c = orc.extract(p0, L)
    d0 = orc.energy(p0, I, L, idx, l, c)
    d1 = orc.energy(p1, I, L, idx, l, c)
    w = orc.curvature_weight(p1)
    for k in range(idx.size):
        b = orc.ball_balance(p1, L, int(idx[k]), int(l[k]), int(c[k]))
        assert d1[k] == d0[k] + w * b
