"""Pins of the MP motion-consistency regulariser oracle (Sec. IV-D, Eqs. (23),
(24)): hand-computed values, limits and central differences (no GPU)."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import regular as R


def test_two_gaussians_by_hand():
    means = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 1.0]])
    prev = np.array([[1.0, 2.0, 2.0], [0.5, 0.0, 1.0]])
    mp = np.array([0.25, 0.5])
    L, g = R.mp_consistency(means, mp, prev, lam=2.0)
    # 2 * (0.75 * 1 + 0.5 * 0.25)
    assert L == 2.0 * (0.75 * 1.0 + 0.5 * 0.25)
    np.testing.assert_array_equal(g, [[0.0, 0.0, 2 * 2.0 * 0.75], [2 * 2.0 * 0.5 * -0.5, 0.0, 0.0]])


def test_dynamic_gaussians_are_free_static_ones_fully_weighted():
    rng = np.random.default_rng(0)
    means, prev = rng.normal(size=(50, 3)), rng.normal(size=(50, 3))
    L1, g1 = R.mp_consistency(means, np.ones(50), prev)
    assert L1 == 0.0 and not g1.any()
    L0, _ = R.mp_consistency(means, np.zeros(50), prev)
    assert abs(L0 - np.sum((means - prev) ** 2)) < 1e-12


def test_relative_pose_aligns_the_previous_means():
    rng = np.random.default_rng(1)
    prev = rng.normal(size=(20, 3))
    T = np.hstack([Rotation.from_rotvec([0.1, -0.2, 0.3]).as_matrix(), [[0.5], [-1.0], [2.0]]])
    means = prev @ T[:, :3].T + T[:, 3]
    L, g = R.mp_consistency(means, rng.random(20), prev, lam=500.0, rel_pose=T)
    assert L < 1e-20 and np.abs(g).max() < 1e-12


def test_gradient_central_differences():
    rng = np.random.default_rng(2)
    means, prev, mp = rng.normal(size=(8, 3)), rng.normal(size=(8, 3)), rng.random(8)
    _, g = R.mp_consistency(means, mp, prev, lam=3.0)
    h = 1e-6
    for k in range(8):
        for c in range(3):
            p, m = means.copy(), means.copy()
            p[k, c] += h
            m[k, c] -= h
            fd = (R.mp_consistency(p, mp, prev, 3.0)[0] - R.mp_consistency(m, mp, prev, 3.0)[0]) / (2 * h)
            assert abs(fd - g[k, c]) <= 1e-6 * max(1.0, abs(fd))
