"""Region fusion on the GPU (SEG_TOPO_FUSE) against the oracle, iteration by iteration:
particles, energy differences, FP64 recomputes and labels bit-exact, with fusion alone, with
splitting and vanishing, in 3D (uint16), and with E = |Gamma| (which reads the contour length
that fusion shortens)."""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step

pytestmark = pytest.mark.gpu


def _touching_blocks(H, W, pitch, seed, levels_of):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[:H, :W]
    ncol = W // pitch
    L = (1 + (yy // pitch) * ncol + (xx // pitch)).astype(np.int32)
    L[:3], L[-3:], L[:, :3], L[:, -3:] = 0, 0, 0, 0
    M = int(L.max()) + 1
    lev = np.array([0.0] + [levels_of(k) for k in range(M - 1)])
    I = (lev[L] + rng.normal(0.0, 0.15, L.shape)).astype(np.float32)
    return I, L


def _run(I, L, topology, lam, iters, gradient="sobolev", conn=None, cutoff=3.0):
    ctx = seg.Context(I, L, model="pc", connectivity=conn, lam=lam, cutoff=cutoff, topology=topology,
                      gradient=gradient)
    p = oracle.make_params(I, L, "pc", conn, lam, cutoff, topology=topology, gradient=gradient)
    run = oracle.Run(p, I, L)
    for it in range(iters):
        compare_step(ctx, run, f"fuse t{topology} it{it}")
    labels = ctx.labels()
    ctx.close()
    return labels


@pytest.mark.parametrize("topology", [4, 7])
def test_fusion_2d_matches_oracle(topology):
    I, L = _touching_blocks(96, 112, 16, seed=1, levels_of=lambda k: 0.6 * (k // 3 % 3))
    labels = _run(I, L, topology, 0.05, 20)
    assert len(np.unique(labels)) < len(np.unique(L))          # regions have fused


def test_fusion_3d_u16_matches_oracle():
    rng = np.random.default_rng(3)
    zz, yy, xx = np.mgrid[:24, :28, :32]
    L = (1 + (zz // 8) * 16 + (yy // 7) * 4 + (xx // 8)).astype(np.int32)
    L[:2], L[-2:] = 0, 0
    lev = np.array([100.0] + [300.0 if (k // 2) % 2 else 200.0 for k in range(int(L.max()))])
    I = np.clip(rng.poisson(lev[L]), 0, 65535).astype(np.uint16)
    labels = _run(I, L, 4, 800.0, 8, conn=6)
    assert len(np.unique(labels)) < len(np.unique(L))


def test_fusion_with_global_length_scale():
    I, L = _touching_blocks(40, 48, 8, seed=4, levels_of=lambda k: 0.5 * (k // 2 % 2))
    _run(I, L, 4, 0.05, 8, gradient="sobolev_global")


def test_fusion_job_in_a_batch_equals_solo():
    I, L = _touching_blocks(96, 112, 16, seed=1, levels_of=lambda k: 0.6 * (k // 3 % 3))
    w2 = synth.disks(80, 64, seed=9)
    mk1 = lambda: seg.Context(I, L, model="pc", lam=0.05, cutoff=3.0, topology="fuse")
    mk2 = lambda: seg.Context.from_workload(w2)

    def solo(make):
        c = make()
        for _ in range(15):
            c.step(1)
        out = c.labels().copy()
        c.close()
        return out

    r1, r2 = solo(mk1), solo(mk2)
    assert len(np.unique(r1)) < len(np.unique(L))
    a, b = mk1(), mk2()
    batch = seg.Batch()
    batch.add(a)
    batch.add(b)
    for _ in range(15):
        batch.step(1)
    assert np.array_equal(a.labels(), r1) and np.array_equal(b.labels(), r2)
    batch.close()
    a.close()
    b.close()
