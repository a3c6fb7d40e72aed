"""Seeded synthetic workloads: determinism and the shapes the configurations call for."""
import numpy as np

from paper_1403_0240_gb300 import synth


def test_stream_is_deterministic_and_uniform():
    a = synth.Stream(7, 3).uniform(100000)
    b = synth.Stream(7, 3).uniform(100000)
    assert np.array_equal(a, b)
    assert abs(a.mean() - 0.5) < 0.01 and a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, synth.Stream(7, 4).uniform(100000))


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    z = np.array([0x9E3779B97F4A7C15, 2 * 0x9E3779B97F4A7C15 % 2**64], dtype=np.uint64)
    out = synth.splitmix64_mix(z)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_normal_and_poisson_moments():
    s = synth.Stream(1, 1)
    z = s.normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    for lam in (0.7, 4.0, 20.0, 150.0):
        k = synth.Stream(2, int(lam * 10)).poisson(np.full(100000, lam))
        assert abs(k.mean() - lam) < 0.05 * max(1.0, np.sqrt(lam))
        assert abs(k.var() - lam) < 0.1 * lam + 0.05


def test_disks_config():
    w = synth.disks()
    assert w.image.shape == (128, 128) and w.image.dtype == np.float32
    assert (w.labels0 == 1).sum() == 64 * 64
    assert np.array_equal(w.image, synth.disks().image)


def test_ellipses_and_ellipsoid_initial_grids():
    assert synth.square_grid_labels(1024, 1024).max() == 256
    L = synth.cube_grid_labels(64, 64, 64)
    assert L.max() == 8 and (L == 3).sum() == 16 ** 3
    w = synth.ellipses(256, 256, seed=3)
    assert w.image.dtype == np.float32 and w.labels0.max() == 16
    v = synth.ellipsoids(32, 32, 32, seed=4)
    assert v.image.dtype == np.uint16 and v.labels0.max() == 1


def test_arrival_stream_mix():
    arr = synth.arrival_stream(2000)
    kinds = [a.kind for a in arr]
    assert 0.75 < kinds.count("pc2d") / 1000 + kinds.count("ps2d") / 1000 < 0.85 * 2
    assert all(arr[i].t < arr[i + 1].t for i in range(len(arr) - 1))
    rate = len(arr) / arr[-1].t
    assert 180 < rate < 220
