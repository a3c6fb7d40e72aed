"""Curvature regulariser on the GPU (SEG_REG_CURVATURE) against the oracle, iteration by
iteration: particles, energy differences within their bounds and the tolerance, FP64
recomputes bit for bit, labels bit-exact; 2D and 3D, every data model, and in a batch."""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step

pytestmark = pytest.mark.gpu


def _pair(w, rho, lam):
    psf = getattr(w, "psf", None)
    ctx = seg.Context(w.image, w.labels0, model=w.model, connectivity=w.connectivity, lam=lam, cutoff=w.cutoff,
                      ps_radius=w.ps_radius, psf=psf, curv_radius=rho)
    p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, lam, w.cutoff, w.ps_radius, psf=psf,
                           curv_radius=rho)
    return ctx, oracle.Run(p, w.image, w.labels0)


@pytest.mark.parametrize("rho,lam", [(4.0, 4.0), (6.5, 10.0)])
def test_curvature_pc_2d(rho, lam):
    w = synth.disks(128, 144, seed=7)
    ctx, run = _pair(w, rho, lam)
    moved = 0
    for it in range(25):
        st, _ = compare_step(ctx, run, f"curv pc2d it{it}")
        moved += st["n_accepted"]
    assert moved > 0
    ctx.close()


def test_curvature_ps_2d_grid():
    w = synth.ellipses(160, 144, seed=33, iterations=10)
    w.labels0 = synth.square_grid_labels(160, 144, 32, 16)
    ctx, run = _pair(w, 5.0, 2.0)
    for it in range(10):
        compare_step(ctx, run, f"curv ps2d it{it}")
    ctx.close()


def test_curvature_pc_3d_u16():
    w = synth.ellipsoids(32, 30, 36, seed=43)
    w.labels0 = synth.cube_grid_labels(32, 30, 36, 12, 6)
    ctx, run = _pair(w, 3.0, 2000.0)
    for it in range(8):
        compare_step(ctx, run, f"curv pc3d it{it}")
    ctx.close()


def test_curvature_deconv_2d():
    w = synth.deconv_scene(64, 72, seed=5, sigma=2.0)
    ctx, run = _pair(w, 4.0, 1.0)
    for it in range(6):
        compare_step(ctx, run, f"curv deconv it{it}")
    ctx.close()


def test_curvature_job_in_a_batch_equals_solo():
    w1 = synth.disks(96, 112, seed=8)
    w2 = synth.disks(80, 64, seed=9)
    mk1 = lambda: seg.Context(w1.image, w1.labels0, model="pc", lam=3.0, cutoff=w1.cutoff, curv_radius=4.0)
    mk2 = lambda: seg.Context.from_workload(w2)

    def solo(make):
        c = make()
        for _ in range(20):
            c.step(1)
        out = c.labels().copy()
        c.close()
        return out

    r1, r2 = solo(mk1), solo(mk2)
    a, b = mk1(), mk2()
    batch = seg.Batch()
    batch.add(a)
    batch.add(b)
    for _ in range(20):
        batch.step(1)
    assert np.array_equal(a.labels(), r1) and np.array_equal(b.labels(), r2)
    batch.close()
    a.close()
    b.close()


def test_curvature_ball_beyond_the_staged_offsets_3d():
    # rho = 8 in 3D has 2109 ball offsets, more than the 2048 the kernel keeps in shared memory:
    # the rest come from global memory
    w = synth.ellipsoids(18, 20, 22, seed=44)
    w.labels0 = synth.cube_grid_labels(18, 20, 22, 9, 5)
    ctx, run = _pair(w, 8.0, 30000.0)
    for it in range(4):
        compare_step(ctx, run, f"curv rho8 3d it{it}")
    ctx.close()
