"""The oracle's deconvolving piecewise-constant model (Eq. 8, J = s_theta(Gamma) * K): the
separable PSF correlation against scipy and its exact impulse response, the per-pixel
|K_x|^2 against a brute-force sum, and the energy change of every particle against a
brute-force recompute of sum (I - K * s)^2 before and after the flip (theta held), which a
dropped term, a wrong sign, a wrong factor or a wrong border norm would all fail."""
import numpy as np
import pytest
from scipy import ndimage

from paper_1403_0240_gb300 import synth


def _outer(k, ndim):
    K = k
    for _ in range(ndim - 1):
        K = np.multiply.outer(K, k)
    return K


def _sym_profile(rng, r):
    h = rng.uniform(0.05, 1.0, r + 1)
    k = np.concatenate([h[:0:-1], h])
    return k / k.sum()


@pytest.mark.parametrize("shape,r", [((37, 53), 6), ((9, 11, 13), 3), ((5, 40), 7)])
def test_psf_correlate_matches_scipy(orc, shape, r):
    rng = np.random.default_rng(3)
    f = rng.normal(0.0, 2.0, shape)
    k = _sym_profile(rng, r)
    I = np.zeros(shape, np.float32)
    p = orc.make_params(I, np.zeros(shape, np.int32), "pcd", psf=k, nlabels=1)
    got = orc.psf_correlate(p, f)
    K = _outer(k, len(shape))
    ref = ndimage.correlate(f, K, mode="constant", cval=0.0)
    mag = ndimage.correlate(np.abs(f), np.abs(K), mode="constant", cval=0.0)
    assert np.all(np.abs(got - ref) <= 1e-13 * mag + 1e-300)


@pytest.mark.parametrize("pos", [(20, 30), (0, 0), (39, 2)])
def test_impulse_response_is_the_outer_product(orc, pos):
    k = synth.gaussian_psf(1.7)
    r = (k.size - 1) // 2
    shape = (40, 45)
    f = np.zeros(shape)
    f[pos] = 1.0
    p = orc.make_params(np.zeros(shape, np.float32), np.zeros(shape, np.int32), "pcd", psf=k, nlabels=1)
    got = orc.psf_correlate(p, f)
    ref = np.zeros(shape)
    K = np.multiply.outer(k, k)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            y, x = pos[0] - dy, pos[1] - dx
            if 0 <= y < shape[0] and 0 <= x < shape[1]:
                ref[y, x] = K[dy + r, dx + r]
    assert np.array_equal(got, ref)


def test_norm2_matches_brute_force(orc):
    rng = np.random.default_rng(5)
    k = _sym_profile(rng, 4)
    for shape in [(12, 15), (6, 7, 9)]:
        p = orc.make_params(np.zeros(shape, np.float32), np.zeros(shape, np.int32), "pcd", psf=k, nlabels=1)
        K2 = _outer(k, len(shape)) ** 2
        for pos in np.ndindex(*shape):
            f = np.zeros(shape)
            f[pos] = 1.0
            ref = ndimage.correlate(f, K2, mode="constant", cval=0.0).sum()
            z, y, x = (0,) + pos if len(shape) == 2 else pos
            assert abs(orc.psf_norm2(p, z, y, x) - ref) <= 1e-14 * ref


def _brute_energy(I, s, K):
    J = ndimage.correlate(s, K, mode="constant", cval=0.0)
    return float(((I - J) ** 2).sum())


def _perimeter(L):
    return sum(int((np.diff(L, axis=a) != 0).sum()) for a in range(L.ndim))


@pytest.mark.parametrize("shape,sigma,lam", [((24, 30), 1.5, 0.0), ((24, 30), 1.5, 0.3), ((20, 17), 4.0, 0.1),
                                             ((7, 8, 9), 1.0, 0.2)])
def test_energy_change_matches_brute_force(orc, shape, sigma, lam):
    rng = np.random.default_rng(11)
    I = rng.uniform(0.0, 3.0, shape).astype(np.float32)
    L = rng.integers(0, 3, shape).astype(np.int32)
    k = synth.gaussian_psf(sigma)
    p = orc.make_params(I, L, "pcd", lam=lam, psf=k)
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    theta = np.array([I[L == m].astype(np.float64).mean() for m in range(3)])
    K = _outer(k, len(shape))
    Id = I.astype(np.float64)
    s = theta[L]
    E0 = _brute_energy(Id, s, K)
    P0 = _perimeter(L)
    tol = 1e-10 * max(E0, 1.0)
    checked = 0
    for q in range(0, idx.size, max(1, idx.size // 150)):
        x = int(idx[q])
        pos = np.unravel_index(x, shape)
        s1 = s.copy()
        s1[pos] = theta[int(c[q])]
        L1 = L.copy()
        L1[pos] = int(c[q])
        ref = _brute_energy(Id, s1, K) - E0 + lam * (_perimeter(L1) - P0)
        assert abs(dE[q] - ref) <= tol, (q, dE[q], ref)
        checked += 1
    assert checked > 50


def test_delta_psf_gives_the_fixed_mean_sse_change(orc):
    rng = np.random.default_rng(12)
    shape = (30, 31)
    I = rng.normal(1.0, 1.0, shape).astype(np.float32)
    L = rng.integers(0, 4, shape).astype(np.int32)
    p = orc.make_params(I, L, "pcd", lam=0.0, psf=np.array([1.0]))
    idx, l, c = orc.extract(p, L)
    dE = orc.energy(p, I, L, idx, l, c)
    n, S, _ = orc.stats(p, I, L)
    theta = S / n
    v = I.reshape(-1).astype(np.float64)[idx]
    ref = (v - theta[c]) ** 2 - (v - theta[l]) ** 2
    assert np.all(np.abs(dE - ref) <= 1e-12 * (1.0 + np.abs(v) + np.abs(theta[c])) ** 2)
    J, R, G = orc.deconv_fields(p, I, L)
    assert np.array_equal(J, theta[L]) and np.array_equal(G, R)


def test_iterations_keep_invariants(orc):
    w = synth.deconv_scene(64, 64, seed=3, sigma=3.0)
    p = orc.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, psf=w.psf)
    run = orc.Run(p, w.image, w.labels0)
    M = int(w.labels0.max()) + 1
    counts0 = np.bincount(run.L.ravel(), minlength=M)
    accepted = 0
    for _ in range(8):
        before = run.L.copy()
        s, _ = run.step()
        accepted += s["n_accepted"]
        assert (before != run.L).sum() == s["n_accepted"]
        counts = np.bincount(run.L.ravel(), minlength=M)
        assert counts.sum() == counts0.sum() and (counts[1:] > 0).all()
    assert accepted > 0
