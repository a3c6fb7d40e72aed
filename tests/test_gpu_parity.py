"""CUDA path against the oracle, through the C-ABI, element by element."""
import numpy as np
import pytest

import oracle
from paper_1403_0240_gb300 import seg, synth
from gpu_helpers import compare_step, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    yield
    torch.cuda.synchronize()


def _mask_to_nb(mask, ndim):
    n = 8 if ndim == 2 else 26
    bits = [(int(mask) >> k) & 1 for k in range(n)]
    centre = n // 2
    return np.array(bits[:centre] + [1] + bits[centre:], np.uint8)


def test_simple_points_match_oracle():
    m2 = np.arange(256, dtype=np.uint32)
    got2 = seg.debug_simple(2, m2)
    ref2 = np.array([oracle.simple_2d(_mask_to_nb(m, 2)) for m in m2], np.uint8)
    assert np.array_equal(got2, ref2)
    rng = np.random.default_rng(0)
    m3 = np.concatenate([rng.integers(0, 1 << 26, 20000, dtype=np.int64),
                         (rng.random((20000, 26)) < 0.8).dot(1 << np.arange(26)),
                         (rng.random((20000, 26)) < 0.2).dot(1 << np.arange(26))]).astype(np.uint32)
    got3 = seg.debug_simple(3, m3)
    ref3 = np.array([oracle.simple_3d(_mask_to_nb(m, 3)) for m in m3], np.uint8)
    assert np.array_equal(got3, ref3)


def test_disks_128_full_run_bit_exact():
    # 128x128 two-disk scene, 50 Sobolev iterations, every iteration compared
    w = synth.disks()
    ctx, run = pair(w)
    fixed = 0
    for it in range(w.iterations):
        st, stats = compare_step(ctx, run, f"disks it{it}")
        fixed += stats.get("fixed", 0)
    n, S, Q = ctx.stats()
    n_ref, S_ref, Q_ref = oracle.stats(run.p, w.image, run.L)
    assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref)
    ctx.close()


@pytest.mark.parametrize("seed", [11, 12])
def test_disks_uneven_l2_and_switch(seed):
    w = synth.disks(97, 133, seed=seed)
    ctx, run = pair(w, osc_window=3)
    for it in range(40):
        compare_step(ctx, run, f"uneven{seed} it{it}")
    ctx.close()


def test_multilabel_grid_2d_pc():
    w = synth.disks(150, 170, seed=21)
    w.labels0 = synth.square_grid_labels(150, 170, 30, 14)
    ctx, run = pair(w)
    for it in range(15):
        compare_step(ctx, run, f"grid2d it{it}")
    ctx.close()


def test_piecewise_smooth_2d():
    w = synth.ellipses(192, 160, seed=31, iterations=12)
    w.labels0 = synth.square_grid_labels(192, 160, 32, 16)
    ctx, run = pair(w)
    for it in range(12):
        compare_step(ctx, run, f"ps2d it{it}")
    ctx.close()


def test_piecewise_constant_3d_u16():
    w = synth.ellipsoids(40, 36, 44, seed=41)
    w.labels0 = synth.cube_grid_labels(40, 36, 44, 12, 6)
    ctx, run = pair(w)
    for it in range(10):
        compare_step(ctx, run, f"pc3d it{it}")
    ctx.close()


def test_piecewise_smooth_3d():
    w = synth.ellipsoids(20, 22, 24, seed=42)
    w.model, w.ps_radius, w.lam = "ps", 2.5, 400.0
    w.labels0 = synth.cube_grid_labels(20, 22, 24, 10, 5)
    ctx, run = pair(w)
    for it in range(6):
        compare_step(ctx, run, f"ps3d it{it}")
    ctx.close()


@pytest.mark.parametrize("cell_edge", [0, 6])
def test_cell_edge_does_not_change_results(cell_edge):
    w = synth.disks(100, 90, seed=51)
    ctx, run = pair(w, cell_edge=cell_edge)
    for it in range(10):
        compare_step(ctx, run, f"cell{cell_edge} it{it}")
    ctx.close()


@pytest.mark.parametrize("cutoff", [1.0, 0.5])
def test_degenerate_cutoff(cutoff):
    w = synth.disks(64, 64, seed=61)
    ctx, run = pair(w, cutoff=cutoff)
    for it in range(10):
        compare_step(ctx, run, f"cut{cutoff} it{it}")
    ctx.close()


def test_l2_until_convergence():
    w = synth.disks(80, 80, seed=71)
    ctx, run = pair(w, gradient="l2")
    for it in range(200):
        st, _ = compare_step(ctx, run, f"l2 it{it}")
        if st["converged"]:
            break
    assert st["converged"] == 1
    st2, _ = compare_step(ctx, run, "after convergence")
    assert st2["n_accepted"] == 0 and st2["converged"] == 1
    ctx.close()


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (3, 3), (2, 2, 2), (1, 1, 9)])
def test_tiny_images(shape):
    rng = np.random.default_rng(len(shape) * 10 + shape[-1])
    I = (rng.random(shape) * 2).astype(np.float32) if len(shape) == 2 else rng.integers(0, 500, shape).astype(np.uint16)
    L = np.zeros(shape, np.int32)
    L.reshape(-1)[0] = 1
    w = synth.Workload("tiny", I, L, "pc", 4 if len(shape) == 2 else 6, 0.01, 2.0)
    ctx, run = pair(w)
    for it in range(4):
        compare_step(ctx, run, f"tiny{shape} it{it}")
    ctx.close()


def test_no_particles():
    I = np.random.default_rng(0).random((33, 47)).astype(np.float32)
    w = synth.Workload("flat", I, np.zeros(I.shape, np.int32), "pc", 4, 0.04, 3.0)
    ctx, run = pair(w)
    for it in range(3):
        st, _ = compare_step(ctx, run, "flat")
        assert st["n_particles"] == 0
    ctx.close()


@pytest.mark.parametrize("three_d", [False, True])
def test_zero_gradients_drop_every_speculative_candidate(three_d):
    # A flat image and no length prior: every energy difference, hence every gradient, is exactly
    # zero, and the oracle has no candidate. On the GPU each admissible pixel is a possible
    # candidate whose sign the bound cannot certify (|g| <= eg); the FP64 recompute finds 0 and
    # drops it before the rounds, so that the counts and labels match.
    shape = (20, 24, 28) if three_d else (48, 56)
    I = np.full(shape, 5, np.uint16) if three_d else np.full(shape, 5.0, np.float32)
    idx = np.indices(shape)
    r2 = sum((idx[k] - shape[k] // 2) ** 2 for k in range(len(shape)))
    L = np.where(r2 <= 49, 1, 0).astype(np.int32)
    w = synth.Workload("zero", I, L, "pc", 6 if three_d else 4, 0.0, 3.0)
    ctx, run = pair(w)
    for it in range(3):
        st, _ = compare_step(ctx, run, f"zero{len(shape)}d it{it}")
        assert st["n_candidates"] == 0 and st["n_accepted"] == 0
        assert st["n_fixup"] > 0, st                 # the speculative candidates were recomputed
    ctx.close()


def test_checkpoint_resume_repeats_bit_for_bit():
    w = synth.disks(96, 96, seed=81)
    a = seg.Context.from_workload(w, osc_window=4)
    a.step(12)
    saved_L, saved_state = a.labels().copy(), a.get_state()
    a.step(15)
    b = seg.Context(w.image, saved_L, model=w.model, lam=w.lam, cutoff=w.cutoff, osc_window=4)
    b.set_state(saved_state)
    b.step(15)
    assert np.array_equal(a.labels(), b.labels())
    assert a.get_state() == b.get_state()
    a.close()
    b.close()


def test_invalid_inputs_rejected():
    I = np.zeros((8, 8), np.float32)
    L = np.zeros((8, 8), np.int32)
    bad = L.copy()
    bad[0, 0] = -1
    with pytest.raises(seg.SegError):
        seg.Context(I, bad)
    nan = I.copy()
    nan[1, 1] = np.nan
    with pytest.raises(seg.SegError):
        seg.Context(nan, L)
    split = L.copy()
    split[1, 1] = 1
    split[5, 5] = 1
    with pytest.raises(seg.SegError):
        seg.Context(I, split, validate=True)
    with pytest.raises(seg.SegError):
        seg.Context(I, L, cutoff=0.0)
    with pytest.raises(seg.SegError):
        seg.Context(I, L, model="ps", ps_radius=0.5)


def test_region_vanishing_matches_oracle():
    # small seed squares (1x1 and 2x2) over a two-disk image: with SEG_TOPO_VANISH the seeds
    # that lie in the background shrink and vanish, iteration by iteration as in the oracle
    w = synth.disks(96, 96, seed=41)
    L = np.zeros((96, 96), np.int32)
    lab = 1
    for y in range(4, 92, 11):
        for x in range(4, 92, 11):
            s = 1 + (lab % 2)
            L[y:y + s, x:x + s] = lab
            lab += 1
    w.labels0 = L
    import oracle
    ctx = seg.Context(w.image, L, model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                      topology="vanish")
    p = oracle.make_params(w.image, L, w.model, w.connectivity, w.lam, w.cutoff, topology=1)
    run = oracle.Run(p, w.image, L)
    for it in range(12):
        compare_step(ctx, run, f"vanish it{it}")
    counts = np.bincount(ctx.labels().ravel(), minlength=lab)
    assert (counts[1:] == 0).any()          # some seeds have vanished
    ctx.close()


def _two_blobs(shape3d=False):
    rng = np.random.default_rng(5)
    if shape3d:
        I = np.zeros((20, 24, 40), np.float32)
        I[4:16, 6:18, 3:15] = 1.0
        I[4:16, 6:18, 25:37] = 1.0
        L = np.zeros(I.shape, np.int32)
        L[7:13, 9:15, 6:34] = 1                       # one bar across both cubes
    else:
        I = np.zeros((96, 128), np.float32)
        I[20:76, 10:50] = 1.0
        I[20:76, 78:118] = 1.0
        L = np.zeros(I.shape, np.int32)
        L[30:66, 18:110] = 1                          # one rectangle across both blobs
    I += rng.normal(0.0, 0.1, I.shape).astype(np.float32)
    return I, L


@pytest.mark.parametrize("topology,three_d", [(2, False), (3, False), (2, True)])
def test_region_splitting_matches_oracle(topology, three_d):
    # the region loses the pixels between the blobs, splits, and its pieces get new labels,
    # iteration by iteration as in the oracle
    import oracle
    I, L = _two_blobs(three_d)
    conn = 6 if three_d else 4
    lam, cutoff = (0.02, 3.0)
    ctx = seg.Context(I, L, model="pc", connectivity=conn, lam=lam, cutoff=cutoff, topology=topology)
    p = oracle.make_params(I, L, "pc", conn, lam, cutoff, topology=topology, nlabels=2)
    run = oracle.Run(p, I, L)
    for it in range(40 if not three_d else 25):
        compare_step(ctx, run, f"split it{it}")
        assert ctx.nlabels == run.state()["nlabels"]
    assert ctx.nlabels >= 3
    n, S, Q = ctx.stats()
    assert np.array_equal(n, np.bincount(ctx.labels().ravel(), minlength=ctx.nlabels))
    ctx.close()


def test_split_beyond_the_label_capacity_is_reported():
    I, L = _two_blobs()
    ctx = seg.Context(I, L, model="pc", lam=0.02, cutoff=3.0, topology="split", max_labels=2)
    with pytest.raises(seg.SegError) as e:
        for _ in range(40):
            ctx.step(1)
    assert e.value.code == seg.SEG_ENOMEM
    ctx.close()
    with pytest.raises(seg.SegError) as e:
        seg.Context(I, L, model="pc", topology="split", max_labels=1)   # below the initial count
    assert e.value.code == seg.SEG_EINVAL


def test_split_job_in_a_batch_equals_solo():
    I, L = _two_blobs()
    w2 = synth.disks(64, 80, seed=9)

    def solo(make):
        c = make()
        for _ in range(30):
            c.step(1)
        out = (c.labels().copy(), c.nlabels)
        c.close()
        return out

    mk1 = lambda: seg.Context(I, L, model="pc", lam=0.02, cutoff=3.0, topology="split")
    mk2 = lambda: seg.Context.from_workload(w2)
    r1, r2 = solo(mk1), solo(mk2)
    a, b = mk1(), mk2()
    batch = seg.Batch()
    batch.add(a)
    batch.add(b)
    for _ in range(30):
        batch.step(1)
    assert np.array_equal(a.labels(), r1[0]) and a.nlabels == r1[1]
    assert np.array_equal(b.labels(), r2[0])
    batch.close()
    a.close()
    b.close()


def test_exact_ties_take_the_warp_recompute():
    # A noise-free volume: a bright cube (300 on 100) around a smaller label cube. The particles
    # of a flat face have translated neighbourhoods, so their gradients are equal in FP64 as in
    # float32; every such tie is queued for the FP64 recompute, more than the recompute grid has
    # blocks, so the one-warp-per-particle recompute runs, and the ties are broken by pixel index
    # as the oracle breaks them.
    D = H = W = 72
    img = np.full((D, H, W), 100, np.uint16)
    img[12:60, 12:60, 12:60] = 300
    lab = np.zeros((D, H, W), np.int32)
    lab[26:46, 26:46, 26:46] = 1
    w = synth.Workload("ties", img, lab, "pc", 6, 1600.0, 4.0, 0.0, 6)
    ctx, run = pair(w)
    most = 0
    for it in range(6):
        st, _ = compare_step(ctx, run, f"ties it{it}")
        most = max(most, st["n_fixup"])
    assert most > 8 * 152, most
    ctx.close()
