"""Pins of the MP-guided edge-warp regulariser oracle (Sec. IV-D, Eqs. (25),
(26)): invariants, the Huber kernel against scipy, and central differences of
both pose-twist gradients (no GPU)."""
import numpy as np
import pytest
import scipy.special
from scipy.spatial.transform import Rotation

from oracle import edge as E
from oracle import pose as opose

W, H = 48, 36
CAM = (40.0, 40.0, 23.3, 17.6, W, H)


def step_scene(seed, z1=1.5, z2=2.4):
    """Depth of two slanted planes meeting at a vertical step, plus noise-free
    copies for frame j shifted by a sub-pixel amount; a smooth weight map."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    Di = np.where(xx < 20 + 0.3 * yy, z1 + 0.004 * xx, z2 - 0.003 * yy)
    Dj = np.where(xx < 20.6 + 0.3 * yy, z1 + 0.004 * xx + 0.01, z2 - 0.003 * yy - 0.02)
    Di[rng.random((H, W)) < 0.03] = 0.0          # a few invalid observations
    wj = 0.5 + 0.4 * np.sin(0.2 * xx) * np.cos(0.15 * yy)
    return Di.ravel(), Dj.ravel(), wj.ravel()


def poses(seed, scale=0.02):
    rng = np.random.default_rng(seed)
    Ti = opose.apply_left(rng.normal(0, scale, 6), np.hstack([np.eye(3), np.zeros((3, 1))]))
    Tj = opose.apply_left(rng.normal(0, scale, 6), Ti)
    return Ti, Tj


def test_huber_matches_scipy():
    r = np.linspace(-0.3, 0.3, 61)
    rho, drho = E.huber(r, 0.05)
    np.testing.assert_allclose(rho, scipy.special.huber(0.05, r), rtol=1e-15, atol=0)
    np.testing.assert_allclose(drho, np.clip(r, -0.05, 0.05), rtol=1e-15, atol=0)


def test_identical_frames_identity_pose_give_zero():
    Di, _, wj = step_scene(0)
    T = np.hstack([Rotation.from_rotvec([0.1, 0.2, -0.1]).as_matrix(), [[0.3], [0.1], [-0.2]]])
    out = E.edge_warp(CAM, Di, Di, wj, T, T)
    assert out["edges"] > 20 and out["n"] > 20
    assert out["L"] < 1e-20


def test_global_rigid_motion_invariance():
    Di, Dj, wj = step_scene(1)
    Ti, Tj = poses(1)
    S = np.vstack([np.hstack([Rotation.from_rotvec([0.5, -0.3, 0.2]).as_matrix(), [[1.0], [-2.0], [0.5]]]),
                   [0, 0, 0, 1]])
    a = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj)
    b = E.edge_warp(CAM, Di, Dj, wj, Ti @ S, Tj @ S)
    assert a["n"] == b["n"] and a["n"] > 20
    assert abs(a["L"] - b["L"]) <= 1e-10 * a["L"]


def test_depth_and_translation_scaling():
    # scaling depths, translations and the Huber threshold by s leaves u' and
    # the (relative) edge set unchanged and scales every residual by s: L
    # scales by s^2
    Di, Dj, wj = step_scene(2)
    Ti, Tj = poses(2)
    s = 1.7
    a = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj)
    Ti2, Tj2 = Ti.copy(), Tj.copy()
    Ti2[:, 3] *= s
    Tj2[:, 3] *= s
    cfg = E.EdgeConfig(huber=0.05 * s, z_near=0.2 * s)
    b = E.edge_warp(CAM, s * Di, s * Dj, wj, Ti2, Tj2, cfg)
    assert a["n"] == b["n"]
    assert abs(b["L"] - s * s * a["L"]) <= 1e-9 * b["L"]


def test_literal_reading_agrees_without_motion_along_the_view():
    # a pure lateral translation keeps every depth: z_ref = Y_z = D_i(u)
    Di, Dj, wj = step_scene(3)
    Ti = np.hstack([np.eye(3), np.zeros((3, 1))])
    Tj = np.hstack([np.eye(3), [[0.013], [-0.007], [0.0]]])
    a = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj)
    b = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj, E.EdgeConfig(literal=True))
    assert a["n"] > 20 and abs(a["L"] - b["L"]) <= 1e-12 * a["L"]
    Tj[2, 3] = 0.05
    c = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj)
    d = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj, E.EdgeConfig(literal=True))
    assert abs(c["L"] - d["L"]) > 1e-3 * c["L"]


@pytest.mark.parametrize("seed,literal", [(4, False), (5, True)])
def test_twist_gradients_central_differences(seed, literal):
    Di, Dj, wj = step_scene(seed)
    Ti, Tj = poses(seed)
    cfg = E.EdgeConfig(literal=literal)
    out = E.edge_warp(CAM, Di, Dj, wj, Ti, Tj, cfg)
    # a flagged pixel lies within 1e-3 px of a cell boundary, far beyond the
    # differences' 1e-7 steps (a few 1e-6 px)
    assert out["flagged"] <= 3 and out["n"] > 20
    h = 1e-7
    for which in ("i", "j"):
        fd = np.zeros(6)
        for k in range(6):
            xi = np.zeros(6)
            xi[k] = h
            if which == "i":
                p = E.edge_warp(CAM, Di, Dj, wj, opose.apply_left(xi, Ti), Tj, cfg)["L"]
                m = E.edge_warp(CAM, Di, Dj, wj, opose.apply_left(-xi, Ti), Tj, cfg)["L"]
            else:
                p = E.edge_warp(CAM, Di, Dj, wj, Ti, opose.apply_left(xi, Tj), cfg)["L"]
                m = E.edge_warp(CAM, Di, Dj, wj, Ti, opose.apply_left(-xi, Tj), cfg)["L"]
            fd[k] = (p - m) / (2 * h)
        an = out["grad_" + which]
        np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
