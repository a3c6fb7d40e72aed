"""The deconvolving piecewise-constant model (Eq. 8, J = s_theta(Gamma) * K) against the
oracle, iteration by iteration: particle sets, energy differences within their bounds, FP64
recomputes and labels bit for bit. Cases: a small 2D scene, the 512 x 512 scene with the
sigma = 15 px PSF of Figure 3, 3D, a PSF wider than the image, a PSF changed between steps,
and the argument checks of seg_set_psf."""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step, pair

pytestmark = pytest.mark.gpu


def test_deconv_2d_small():
    w = synth.deconv_scene(96, 80, seed=21, sigma=3.0)
    ctx, run = pair(w)
    for it in range(12):
        compare_step(ctx, run, f"pcd2d it{it}")
    ctx.close()


def test_deconv_2d_sigma15_512():
    w = synth.deconv_scene()                      # 512 x 512, sigma 15 (r = 45)
    ctx, run = pair(w)
    for it in range(3):
        compare_step(ctx, run, f"pcd512 it{it}")
    ctx.close()


def test_deconv_3d_u16():
    w = synth.ellipsoids(18, 20, 22, seed=23)
    w.model, w.lam = "pcd", 40.0
    w.psf = synth.gaussian_psf(1.5)
    w.labels0 = synth.cube_grid_labels(18, 20, 22, 10, 5)
    ctx, run = pair(w)
    for it in range(6):
        compare_step(ctx, run, f"pcd3d it{it}")
    ctx.close()


def test_deconv_odd_extents():
    w = synth.deconv_scene(61, 75, seed=27, sigma=2.5)       # odd rows and columns: unpaired last outputs
    ctx, run = pair(w)
    for it in range(6):
        compare_step(ctx, run, f"pcd-odd2d it{it}")
    ctx.close()
    v = synth.ellipsoids(17, 19, 21, seed=28)
    v.model, v.lam = "pcd", 40.0
    v.psf = synth.gaussian_psf(1.2)
    v.labels0 = synth.cube_grid_labels(17, 19, 21, 10, 5)
    ctx, run = pair(v)
    for it in range(4):
        compare_step(ctx, run, f"pcd-odd3d it{it}")
    ctx.close()


def test_deconv_psf_wider_than_image():
    w = synth.deconv_scene(24, 20, seed=24, sigma=10.0)      # r = 30 > both sides
    ctx, run = pair(w)
    for it in range(5):
        compare_step(ctx, run, f"pcd-wide it{it}")
    ctx.close()


def test_deconv_psf_changed_between_steps():
    w = synth.deconv_scene(64, 72, seed=25, sigma=2.0)
    ctx, run = pair(w)
    for it in range(3):
        compare_step(ctx, run, f"pcd-a it{it}")
    k2 = synth.gaussian_psf(4.0)
    ctx.set_psf(k2)
    oracle.set_psf(run.p, k2)
    for it in range(3):
        compare_step(ctx, run, f"pcd-b it{it}")
    ctx.close()


def test_set_psf_argument_checks():
    w = synth.deconv_scene(32, 32, seed=26, sigma=2.0)
    ctx = seg.Context(w.image, w.labels0, model="pcd", lam=w.lam, cutoff=w.cutoff)
    with pytest.raises(seg.SegError) as e:
        ctx.step(1)                                   # no PSF yet
    assert e.value.code == seg.SEG_ESTATE
    bad = w.psf.copy()
    bad[0] *= 1.5                                     # not symmetric
    for k, code in [(bad, seg.SEG_EINVAL), (np.full(2 * 513 + 1, 1e-3), seg.SEG_EINVAL),
                    (np.array([np.nan]), seg.SEG_EINVAL)]:
        with pytest.raises(seg.SegError) as e:
            ctx.set_psf(k)
        assert e.value.code == code
    ctx.set_psf(w.psf)
    assert ctx.step(2)["error"] == 0
    ctx.close()
    pc = seg.Context(w.image, w.labels0, model="pc")
    with pytest.raises(seg.SegError) as e:
        pc.set_psf(w.psf)
    assert e.value.code == seg.SEG_ESTATE
    pc.close()
