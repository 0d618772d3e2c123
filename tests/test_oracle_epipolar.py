"""Pins of the epipolar verification oracle (Sec. IV-C, Eqs. (18), (19)):
exact geometry, an independent point-to-line distance, numpy's sort for the
median, and the recovery rule (no GPU)."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import epipolar as E

CAM = (300.0, 310.0, 161.3, 118.7, 320, 240)


def poses():
    T1 = np.hstack([Rotation.from_rotvec([0.05, -0.1, 0.02]).as_matrix(), [[0.1], [-0.2], [0.3]]])
    T2 = np.hstack([Rotation.from_rotvec([0.08, -0.05, 0.0]).as_matrix(), [[0.25], [-0.1], [0.28]]])
    return T1, T2


def project(T, X):
    fx, fy, cx, cy = CAM[:4]
    Y = X @ T[:, :3].T + T[:, 3]
    return np.stack([fx * Y[:, 0] / Y[:, 2] + cx, fy * Y[:, 1] / Y[:, 2] + cy], 1), Y[:, 2]


def scene(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform([-1.0, -0.8, 2.0], [1.0, 0.8, 4.0], (n, 3))


def test_static_correspondences_lie_on_their_lines():
    T1, T2 = poses()
    X = scene(200, 0)
    p1, _ = project(T1, X)
    p2, _ = project(T2, X)
    d = E.distances(E.fundamental(CAM, T1, T2), p1, p2)
    assert d.max() < 1e-9


def test_distance_is_the_point_to_line_distance():
    # the epipolar line of p1 passes through the projections into frame 2 of
    # two points on p1's viewing ray; d is the distance of p2 from that line
    T1, T2 = poses()
    rng = np.random.default_rng(1)
    X = scene(50, 1)
    p1, z1 = project(T1, X)
    p2 = project(T2, X)[0] + rng.normal(0, 3.0, (50, 2))
    d = E.distances(E.fundamental(CAM, T1, T2), p1, p2)
    fx, fy, cx, cy = CAM[:4]
    for k in range(50):
        ray_c = np.array([(p1[k, 0] - cx) / fx, (p1[k, 1] - cy) / fy, 1.0])
        pts = []
        for depth in (1.0, 5.0):
            Xc = depth * ray_c
            Xw = T1[:, :3].T @ (Xc - T1[:, 3])
            pts.append(project(T2, Xw[None])[0][0])
        a, b = pts
        u = (b - a) / np.linalg.norm(b - a)
        w = p2[k] - a
        ref = abs(u[0] * w[1] - u[1] * w[0])
        assert abs(d[k] - ref) <= 1e-8 * max(1.0, ref)


def test_sliding_along_the_epipolar_line_keeps_zero():
    T1, T2 = poses()
    X = scene(20, 2)
    p1, z1 = project(T1, X)
    # the same pixel in frame 1 at another depth: a different 3D point on the ray
    fx, fy, cx, cy = CAM[:4]
    ray = np.stack([(p1[:, 0] - cx) / fx, (p1[:, 1] - cy) / fy, np.ones(20)], 1)
    Xc = ray * (1.3 * z1)[:, None]
    Xw = (Xc - T1[:, 3]) @ T1[:, :3]
    p2, _ = project(T2, Xw)
    assert E.distances(E.fundamental(CAM, T1, T2), p1, p2).max() < 1e-9


def test_rectified_stereo_lines_are_rows():
    # textbook special case: same intrinsics, R = I, a baseline along x.
    # The epipolar line of (u1, v1) is the row v = v1, so d = |v2 - v1| for
    # any u1, u2, whatever fx != fy and the principal point
    T1 = np.hstack([np.eye(3), [[0.0], [0.0], [0.0]]])
    T2 = np.hstack([np.eye(3), [[-0.12], [0.0], [0.0]]])
    rng = np.random.default_rng(7)
    p1 = rng.uniform([0, 0], [320, 240], (40, 2))
    p2 = rng.uniform([0, 0], [320, 240], (40, 2))
    d = E.distances(E.fundamental(CAM, T1, T2), p1, p2)
    np.testing.assert_allclose(d, np.abs(p2[:, 1] - p1[:, 1]), rtol=1e-12, atol=1e-10)


def test_median_and_recovery_rule():
    T1, T2 = poses()
    rng = np.random.default_rng(3)
    n = 30
    gid = rng.integers(0, 25, 400)            # Gaussians 25..29 have no matches
    X = scene(400, 3)
    p1, _ = project(T1, X)
    p2 = project(T2, X)[0] + rng.normal(0, 1.0, (400, 2)) * (1 + (gid % 3 == 0))[:, None] * 1.5
    mp = rng.uniform(0, 1, n)
    labels = (rng.random(n) < 0.5).astype(np.uint8)
    out = E.verify(CAM, T1, T2, p1, p2, gid, n, mp, labels)
    d = E.distances(E.fundamental(CAM, T1, T2), p1, p2)
    for g in range(n):
        sel = np.sort(d[gid == g])
        if len(sel) == 0:
            assert np.isnan(out["dbar"][g]) and not out["consistent"][g]
            assert out["labels"][g] == labels[g] and out["mp"][g] == mp[g]
            continue
        assert out["dbar"][g] == sel[(len(sel) - 1) // 2]
        ok = sel[(len(sel) - 1) // 2] < 1.0
        assert out["consistent"][g] == ok
        if ok and labels[g] == 1:
            assert out["labels"][g] == 0 and out["mp"][g] == min(mp[g], 0.1)
        else:
            assert out["labels"][g] == labels[g] and out["mp"][g] == mp[g]
    assert out["restored"].sum() >= 1 and (out["consistent"] & (labels == 0)).sum() >= 1
