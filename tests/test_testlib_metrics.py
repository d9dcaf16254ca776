"""The vector-error measures the GPU parity tests use are the sines of known
angles: a vector rotated by theta in a plane, and a two-dimensional subspace
with principal angles (theta_1, theta_2), at angles from 1e-12 to 1 rad."""
import math

import numpy as np
import pytest

from ssa_testlib import clusters, subspace_sin, vec_sin


def _orthonormal(n, m, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, m)))
    return q


@pytest.mark.parametrize("theta", [1e-12, 1e-9, 1e-6, 1e-3, 0.3, 1.2])
def test_vec_sin_is_the_sine_of_the_angle(theta):
    q = _orthonormal(500, 2, 1)
    a = q[:, 0]
    b = math.cos(theta) * q[:, 0] + math.sin(theta) * q[:, 1]
    want = math.sin(theta)
    for s in (1.0, -1.0):   # either sign of the second vector
        assert abs(vec_sin(a, s * 3.0 * b) - want) <= 1e-9 * want + 1e-15


@pytest.mark.parametrize("t1,t2", [(1e-11, 1e-13), (1e-8, 5e-9), (0.2, 1e-7)])
def test_subspace_sin_is_the_largest_principal_angle(t1, t2):
    q = _orthonormal(400, 4, 2)
    A = q[:, :2]
    B = np.stack([math.cos(t1) * q[:, 0] + math.sin(t1) * q[:, 2],
                  math.cos(t2) * q[:, 1] + math.sin(t2) * q[:, 3]], axis=1)
    B = B @ np.array([[2.0, 1.0], [0.5, -1.0]])    # any basis of the same span
    want = math.sin(max(t1, t2))
    assert abs(subspace_sin(A, B) - want) <= 1e-8 * want + 1e-15


def test_clusters_split_on_relative_gap():
    assert clusters(np.array([10.0, 10.0 - 1e-7, 5.0, 1.0, 1.0])) == [[0, 1], [2], [3, 4]]
