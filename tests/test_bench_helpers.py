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
