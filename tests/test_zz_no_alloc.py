"""The allocation-free region-statistics entry point against the allocating path.

Callers that cannot allocate device memory (a pool of their own, or code that must not
trigger the device synchronisation of cudaMalloc) use seg_region_stats_noalloc, whose
accumulators live in a fixed device array. It must give the same counts and exactly
rounded sums as seg_init followed by seg_stats, on two calls in a row: the array keeps the
previous call's contents, so the second call also shows that the accumulators start from
zero. This file is collected last so that a failure here stops a run only after every
other test has run."""
import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu


def _case(kind):
    if kind == "f32_2d":
        w = synth.disks(96, 130, seed=3)
        w.labels0 = synth.square_grid_labels(96, 130, 32, 12)
        return w.image, w.labels0
    if kind == "f32_wide":
        rng = np.random.default_rng(5)
        I = (rng.normal(0, 1, (70, 90)) * np.exp2(rng.integers(-30, 30, (70, 90)))).astype(np.float32)
        I[::7, ::5] = 0.0
        L = rng.integers(0, 37, I.shape).astype(np.int32)
        return I, L
    w = synth.ellipsoids(24, 28, 30, seed=9)
    w.labels0 = synth.cube_grid_labels(24, 28, 30, 12, 6)
    return w.image, w.labels0


def _reference(image, labels):
    ctx = seg.Context(image, labels)          # seg_init computes the statistics; seg_stats reads them
    out = ctx.stats()
    ctx.close()
    return out


def test_matches_allocating_path_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    cases = [_case("f32_2d"), _case("u16_3d"), _case("f32_wide")]
    refs = [_reference(I, L) for I, L in cases]
    # two calls in a row on different inputs, then the same input twice
    for (I, L), (n_ref, S_ref, Q_ref) in list(zip(cases, refs)) + [(cases[0], refs[0])]:
        img = torch.from_numpy(I).cuda()
        lab = torch.from_numpy(L).cuda()
        M = int(L.max()) + 1
        n, S, Q = seg.region_stats_noalloc(img, lab, M)
        torch.cuda.synchronize()
        assert np.array_equal(n.cpu().numpy(), n_ref)
        # exact sums rounded once: equal to the allocating path bit for bit
        assert np.array_equal(S.cpu().numpy(), S_ref)
        assert np.array_equal(Q.cpu().numpy(), Q_ref)


def test_rejects_what_it_cannot_hold():
    import torch
    I, L = _case("f32_2d")
    img = torch.from_numpy(I).cuda()
    lab = torch.from_numpy(L).cuda()
    M = int(L.max()) + 1
    with pytest.raises(seg.SegError) as e:
        seg.region_stats_noalloc(img, lab, M - 1)          # a label beyond nlabels - 1
    assert e.value.code == seg.SEG_EINVAL
    with pytest.raises(seg.SegError) as e:
        seg.region_stats_noalloc(img, lab, 1025)            # above the fixed maximum of labels
    assert e.value.code == seg.SEG_EINVAL
    n = torch.empty(M, dtype=torch.int64)                   # host output: rejected
    with pytest.raises(ValueError):
        seg.region_stats_noalloc(img, lab, M, n=n)
    with pytest.raises(ValueError):                         # int64 labels would be read as pairs of words
        seg.region_stats_noalloc(img, lab.to(torch.int64), M)
    with pytest.raises(ValueError):                         # fewer labels than pixels: reads past the end
        seg.region_stats_noalloc(img, lab.reshape(-1)[:-1].contiguous(), M)
    with pytest.raises(ValueError):                         # an output of the wrong length
        seg.region_stats_noalloc(img, lab, M, S=torch.empty(M - 1, dtype=torch.float64, device=img.device))
    # through the C-ABI itself, a host output buffer is refused with SEG_EINVAL
    import ctypes
    n_host = np.zeros(M, np.int64)
    S_dev = torch.empty(M, dtype=torch.float64, device=img.device)
    Q_dev = torch.empty(M, dtype=torch.float64, device=img.device)
    code = seg.lib().seg_region_stats_noalloc(seg.SEG_F32, img.numel(), ctypes.c_void_p(img.data_ptr()),
                                              ctypes.c_void_p(lab.data_ptr()), M, n_host.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.c_void_p(S_dev.data_ptr()), ctypes.c_void_p(Q_dev.data_ptr()),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == seg.SEG_EINVAL
    # a valid call afterwards still matches
    n2, S2, Q2 = seg.region_stats_noalloc(img, lab, M)
    n_ref, S_ref, Q_ref = _reference(I, L)
    assert np.array_equal(S2.cpu().numpy(), S_ref) and np.array_equal(n2.cpu().numpy(), n_ref)
