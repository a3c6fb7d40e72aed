"""The piecewise-smooth model with Poisson noise against the oracle, iteration by iteration:
the staged 2D path, the generic path (3D, and 2D with a ball wider than the staged halo), and
the rejection of negative intensities."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step, pair

pytestmark = pytest.mark.gpu


def test_poisson_2d_staged():
    w = synth.ellipses(192, 160, seed=51, iterations=15)
    w.model = "psp"
    w.labels0 = synth.square_grid_labels(192, 160, 32, 16)
    ctx, run = pair(w)
    for it in range(15):
        compare_step(ctx, run, f"psp2d it{it}")
    ctx.close()


def test_poisson_2d_wide_ball():
    w = synth.ellipses(96, 80, seed=52, iterations=5)
    w.model, w.ps_radius = "psp", 36.0
    w.labels0 = synth.square_grid_labels(96, 80, 32, 16)
    ctx, run = pair(w)
    for it in range(5):
        compare_step(ctx, run, f"psp2d-wide it{it}")
    ctx.close()


def test_poisson_3d_u16():
    w = synth.ellipsoids(20, 22, 24, seed=53)
    w.model, w.ps_radius, w.lam = "psp", 2.5, 40.0
    w.labels0 = synth.cube_grid_labels(20, 22, 24, 10, 5)
    ctx, run = pair(w)
    for it in range(6):
        compare_step(ctx, run, f"psp3d it{it}")
    ctx.close()


def test_poisson_rejects_negative_intensities():
    I = np.ones((16, 16), np.float32)
    I[3, 4] = -0.5
    L = np.zeros((16, 16), np.int32)
    L[4:10, 4:10] = 1
    with pytest.raises(seg.SegError) as e:
        seg.Context(I, L, model="psp", ps_radius=3.0)
    assert e.value.code == seg.SEG_EINVAL
    seg.Context(I, L, model="ps", ps_radius=3.0).close()     # the Gaussian model accepts them
