"""Host helpers of bench.py's convergence study: contour length and piecewise-constant energy."""
import numpy as np

import bench


def test_contour_length_of_a_square_and_a_cube():
    L = np.zeros((10, 12), np.int32)
    L[2:6, 3:8] = 1
    assert bench._contour_length(L) == 2 * (4 + 5)
    V = np.zeros((6, 6, 6), np.int32)
    V[1:3, 1:4, 2:4] = 2
    assert bench._contour_length(V) == 2 * (2 * 3 + 2 * 2 + 3 * 2)


def test_pc_energy_two_regions():
    I = np.array([[1.0, 3.0, 10.0, 14.0]], np.float32)
    L = np.array([[0, 0, 1, 1]], np.int32)
    # means 2 and 12: SSE = 1 + 1 + 4 + 4; one boundary pair
    assert bench._pc_energy(I, L, 0.5) == 10.0 + 0.5


def test_psf_pass_flops_counts_the_in_image_taps():
    from paper_1403_0240_gb300 import synth
    for shape, sigma in [((9, 13), 1.5), ((5, 7, 6), 1.0), ((4, 30), 3.0)]:
        w = synth.disks(8, 8)
        w.model, w.image, w.psf = "pcd", np.zeros(shape, np.float32), synth.gaussian_psf(sigma)
        r = (w.psf.size - 1) // 2
        axes = [len(shape) - 1 - a for a in range(len(shape))]           # numpy axis of x, y[, z]
        passes = [axes[0], axes[1], axes[0]] if len(shape) == 2 else [axes[0], axes[1], axes[2], axes[0], axes[1]]
        brute = 0
        for ax in passes:
            for pos in np.ndindex(*shape):
                brute += sum(1 for u in range(-r, r + 1) if 0 <= pos[ax] + u < shape[ax])
        assert bench.psf_pass_flops(w) == 2.0 * brute
        assert bench.psf_passes(w) == len(passes)


def test_deconv_energy_matches_scipy():
    from scipy import ndimage
    from paper_1403_0240_gb300 import synth
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 2, (20, 23)).astype(np.float32)
    L = rng.integers(0, 3, (20, 23)).astype(np.int32)
    k = synth.gaussian_psf(1.5)
    theta = np.array([I[L == m].astype(np.float64).mean() for m in range(3)])
    J = ndimage.correlate(theta[L], np.multiply.outer(k, k), mode="constant", cval=0.0)
    ref = float(((I.astype(np.float64) - J) ** 2).sum()) + 0.3 * bench._contour_length(L)
    assert abs(bench._deconv_energy(I, L, k, 0.3) - ref) <= 1e-9 * ref


def test_topology_options_and_their_kernel_counts():
    import bench

    class A:
        topology = ""
        curv_radius = 0.0

    assert bench.topology_code("") == 0 and bench.topology_code("vanish+split+fuse") == 7
    assert bench.topology_code("split") == 2 and bench.topology_code("vanish+fuse") == 5
    assert bench.extra_kernels(A) == 0
    A.topology, A.curv_radius = "vanish+split", 5.0
    assert bench.extra_kernels(A) == bench.EXTRA_KERNELS["split"] + bench.EXTRA_KERNELS["curvature"]


def test_profile_digest_covers_code_not_comments():
    a = ["int f(int x) { return x + 1; }  // adds one\n/* a block\n   comment */\n"]
    b = ["// another note\nint f(int x) { return x + 1; }\n\n"]
    c = ["int f(int x) { return x + 2; }\n"]
    assert bench._code_digest(a) == bench._code_digest(b)
    assert bench._code_digest(a) != bench._code_digest(c)
    assert len(bench.kernel_sources_digest()) == 16
