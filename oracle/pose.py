"""FP64 oracle of the pose step: Adam on the 6-DoF left-perturbation twist of
the world-to-camera pose, followed by T <- exp(xi^) T.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper refines poses jointly with the Gaussians (Eq. (27)) and names
Levenberg-Marquardt for the pose (Sec. V-A(c)); the hot path's step is a
first-order Adam step on the twist in FP64, with the twist reset to zero
after each step (it is a perturbation of the current pose).

Twist order: xi = (rho, phi), translation first. Pose: 3x4 row-major [R | t].

Pins: exp(0) = I; pure rotations against scipy's rotation-vector map; pure
translations; exp(xi) exp(-xi) = I; Adam against torch.optim.Adam.
"""
from __future__ import annotations

import numpy as np


def hat(phi: np.ndarray) -> np.ndarray:
    x, y, z = phi
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def se3_exp(xi: np.ndarray):
    """(R, t) of exp(xi^) for xi = (rho, phi): R by Rodrigues' formula,
    t = V rho with V the left Jacobian of SO(3). Series forms below
    theta = 1e-4 (the next omitted terms are below 1e-17)."""
    xi = np.asarray(xi, dtype=np.float64)
    rho, phi = xi[:3], xi[3:]
    th2 = float(phi @ phi)
    th = np.sqrt(th2)
    K = hat(phi)
    K2 = K @ K
    if th < 1e-4:
        a = 1.0 - th2 / 6.0
        b = 0.5 - th2 / 24.0
        c = 1.0 / 6.0 - th2 / 120.0
    else:
        a = np.sin(th) / th
        b = (1.0 - np.cos(th)) / th2
        c = (th - np.sin(th)) / (th2 * th)
    R = np.eye(3) + a * K + b * K2
    V = np.eye(3) + b * K + c * K2
    return R, V @ rho


def apply_left(xi: np.ndarray, pose: np.ndarray) -> np.ndarray:
    """exp(xi^) composed on the left of a 3x4 pose."""
    pose = np.asarray(pose, dtype=np.float64).reshape(3, 4)
    Re, te = se3_exp(xi)
    out = np.empty((3, 4))
    out[:, :3] = Re @ pose[:, :3]
    out[:, 3] = Re @ pose[:, 3] + te
    return out


def adam_twist_step(grad6, state13, lr6, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on the twist (which is zero before the step).

    state13 = (m[6], v[6], step). Returns (xi, new_state). xi = -lr * m_hat /
    (sqrt(v_hat) + eps) with bias-corrected moments.
    """
    g = np.asarray(grad6, dtype=np.float64)
    st = np.asarray(state13, dtype=np.float64).copy()
    m, v, k = st[0:6], st[6:12], st[12] + 1.0
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** k)
    vh = v / (1.0 - beta2 ** k)
    xi = -np.asarray(lr6, dtype=np.float64) * mh / (np.sqrt(vh) + eps)
    st[0:6], st[6:12], st[12] = m, v, k
    return xi, st


def pose_step(pose, grad6, state13, lr6, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full pose step: returns (new_pose 3x4, new_state13)."""
    xi, st = adam_twist_step(grad6, state13, lr6, beta1, beta2, eps)
    return apply_left(xi, pose), st
