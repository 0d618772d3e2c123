"""FP64 oracle of the epipolar verification and static recovery (Sec. IV-C,
Eqs. (18), (19)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  F        = K^-T [t]x R K^-1 from the intrinsics and the relative pose
             (R, t) = T_21 = T_2W T_1W^-1 (frame 1 to frame 2)
  l2       = F p1 = (a, b, c),  d = |p2^T F p1| / sqrt(a^2 + b^2)      Eq. (18)
  dbar(G)  = lower median of d over the matches associated with G     Eq. (19)
  G is epipolar-consistent iff dbar(G) < eps (1 px, Sec. V-A(c)).

Readings:
- The matches and their Gaussian are inputs (the feature front end and its
  RANSAC refinement of F are outside the hot path); F comes from the
  estimated poses and the calibrated intrinsics only.
- The median of an even count is the lower middle element, as everywhere in
  this library.
- "Restored as static": a Gaussian labelled dynamic (label 1) whose dbar is
  below eps gets label 0 and M <- min(M, m_static), m_static = 0.1 (the
  background class prior mu(bg) of the MP update's defaults). Gaussians
  without matches are left alone. Densification is not part of the path.

Pins (tests/test_oracle_epipolar.py): exact correspondences of a static
scene give d = 0 and so do points slid along the epipolar line; d against
the point-to-line distance of the line through two projected points of the
back-projected ray; the median against numpy's sort; the recovery rule on a
hand-made case.
"""
from __future__ import annotations

import numpy as np


def fundamental(cam, pose_1, pose_2):
    """F (3x3) mapping homogeneous pixels of frame 1 to epipolar lines of frame 2."""
    fx, fy, cx, cy = cam[:4]
    K = np.array([[fx, 0.0, cx], [0.0, fy, cy], [0.0, 0.0, 1.0]])
    T1 = np.asarray(pose_1, np.float64).reshape(3, 4)
    T2 = np.asarray(pose_2, np.float64).reshape(3, 4)
    R = T2[:, :3] @ T1[:, :3].T
    t = T2[:, 3] - R @ T1[:, 3]
    tx = np.array([[0.0, -t[2], t[1]], [t[2], 0.0, -t[0]], [-t[1], t[0], 0.0]])
    Ki = np.linalg.inv(K)
    return Ki.T @ tx @ R @ Ki


def distances(F, p1, p2):
    """Eq. (18) for every match (p1, p2: m x 2 pixel coordinates)."""
    p1 = np.asarray(p1, np.float64).reshape(-1, 2)
    p2 = np.asarray(p2, np.float64).reshape(-1, 2)
    h1 = np.hstack([p1, np.ones((len(p1), 1))])
    h2 = np.hstack([p2, np.ones((len(p2), 1))])
    l2 = h1 @ F.T
    return np.abs(np.sum(h2 * l2, axis=1)) / np.sqrt(l2[:, 0] ** 2 + l2[:, 1] ** 2)


def verify(cam, pose_1, pose_2, p1, p2, gid, n, mp, labels, eps=1.0, m_static=0.1):
    """Returns dict(d (m), dbar (n, NaN without matches), count (n),
    consistent (n bool), mp, labels (after recovery), restored (n bool))."""
    F = fundamental(cam, pose_1, pose_2)
    d = distances(F, p1, p2)
    gid = np.asarray(gid, np.int64)
    dbar = np.full(n, np.nan)
    count = np.bincount(gid, minlength=n)[:n]
    order = np.lexsort((d, gid))
    gs, ds = gid[order], d[order]
    starts = np.searchsorted(gs, np.arange(n), side="left")
    for g in np.nonzero(count)[0]:
        c = count[g]
        dbar[g] = ds[starts[g] + (c - 1) // 2]
    consistent = np.nan_to_num(dbar, nan=np.inf) < eps
    labels = np.asarray(labels, np.uint8).copy()
    mp = np.asarray(mp, np.float64).copy()
    restored = consistent & (labels == 1)
    labels[restored] = 0
    mp[restored] = np.minimum(mp[restored], m_static)
    return dict(d=d, dbar=dbar, count=count, consistent=consistent, mp=mp, labels=labels, restored=restored)
