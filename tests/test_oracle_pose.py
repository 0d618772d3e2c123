"""Pins of the FP64 pose-step oracle (no GPU)."""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

from oracle import pose as P


def twist_matrix(xi):
    m = np.zeros((4, 4))
    m[:3, :3] = P.hat(xi[3:])
    m[:3, 3] = xi[:3]
    return m


def test_exp_zero_is_identity():
    R, t = P.se3_exp(np.zeros(6))
    np.testing.assert_array_equal(R, np.eye(3))
    np.testing.assert_array_equal(t, np.zeros(3))


@pytest.mark.parametrize("phi", [[0.3, 0, 0], [0, -1.2, 0], [0, 0, 2.5], [0.2, -0.4, 0.9], [1e-5, 2e-5, -3e-6]])
def test_exp_pure_rotation_matches_rotvec(phi):
    R, t = P.se3_exp(np.r_[0, 0, 0, phi])
    np.testing.assert_allclose(R, Rotation.from_rotvec(phi).as_matrix(), atol=1e-15)
    np.testing.assert_allclose(t, 0, atol=0)


@pytest.mark.parametrize("seed", range(6))
def test_exp_matches_matrix_exponential(seed):
    # The closed form (Rodrigues + left Jacobian V) equals the 4x4 matrix
    # exponential of the twist (scipy.linalg.expm), including the series branch.
    rng = np.random.default_rng(seed)
    scale = [1.0, 1e-3, 1e-5, 3e-5, 0.5, 2.0][seed]
    xi = rng.normal(0, scale, 6)
    R, t = P.se3_exp(xi)
    E = scipy.linalg.expm(twist_matrix(xi))
    np.testing.assert_allclose(R, E[:3, :3], atol=1e-14)
    np.testing.assert_allclose(t, E[:3, 3], atol=1e-14 * max(1, np.abs(xi).max()))


def test_exp_inverse():
    xi = np.array([0.1, -0.2, 0.3, 0.4, -0.1, 0.2])
    pose = np.hstack([Rotation.from_rotvec([0.1, 0.2, 0.3]).as_matrix(), [[1.0], [2.0], [3.0]]])
    back = P.apply_left(-xi, P.apply_left(xi, pose))
    np.testing.assert_allclose(back, pose, atol=1e-14)


def test_series_branch_is_continuous():
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    lo = P.se3_exp(np.r_[1, 2, 3, d * (1e-4 * (1 - 1e-9))])
    hi = P.se3_exp(np.r_[1, 2, 3, d * (1e-4 * (1 + 1e-9))])
    np.testing.assert_allclose(lo[0], hi[0], atol=1e-15)
    np.testing.assert_allclose(lo[1], hi[1], atol=1e-14)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    lr = np.array([1e-3, 1e-3, 1e-3, 2e-3, 2e-3, 2e-3])
    params = [torch.zeros(1, dtype=torch.float64, requires_grad=True) for _ in range(6)]
    opts = [torch.optim.Adam([params[k]], lr=float(lr[k]), betas=(0.9, 0.999), eps=1e-8) for k in range(6)]
    state = np.zeros(13)
    for _ in range(7):
        g = rng.normal(0, 10, 6)
        before = np.array([p.item() for p in params])
        for k in range(6):
            params[k].grad = torch.tensor([g[k]], dtype=torch.float64)
            opts[k].step()
        after = np.array([p.item() for p in params])
        xi, state = P.adam_twist_step(g, state, lr)
        np.testing.assert_allclose(xi, after - before, rtol=1e-12, atol=1e-18)
    assert state[12] == 7
