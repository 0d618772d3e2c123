"""FP64 oracle of the MP-based motion-consistency regulariser (Sec. IV-D,
Eqs. (23), (24)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  mu_hat_k = T_{t<-t-1} mu_k^{t-1}                          Eq. (23)
  L_MP     = sum_k Mbar_k |mu_k - mu_hat_k|^2, Mbar = 1 - M  Eq. (24)

Readings:
- The map's means are world coordinates (the poses are world-to-camera), a
  frame-consistent system, so the relative pose is the identity and mu_hat is
  the mean after the previous mapping update. A relative pose (3x4) may still
  be given, for a camera-centric use.
- M_k is the record's motion probability, held constant: the MP update sets
  it, the loss does not optimise it. The sum runs over every Gaussian of the
  map (not only the ones a view sees).
- The weight lambda_3 (500, Sec. V-A(c)) multiplies L_MP and its gradient
  d(lambda L_MP)/d mu_k = 2 lambda Mbar_k (mu_k - mu_hat_k).

Pins (tests/test_oracle_regular.py): hand-computed two-Gaussian values, the
dynamic (M = 1) and static (M = 0) limits, a relative pose that maps the
previous means onto the current ones giving zero, and central differences.
"""
from __future__ import annotations

import numpy as np


def mp_consistency(means, mp, prev_means, lam=1.0, rel_pose=None):
    """(lam * L_MP, d(lam L_MP)/d means (n x 3))."""
    mu = np.asarray(means, np.float64).reshape(-1, 3)
    prev = np.asarray(prev_means, np.float64).reshape(-1, 3)
    if rel_pose is not None:
        T = np.asarray(rel_pose, np.float64).reshape(3, 4)
        prev = prev @ T[:, :3].T + T[:, 3]
    mbar = 1.0 - np.asarray(mp, np.float64).ravel()
    d = mu - prev
    L = float(np.sum(mbar * np.sum(d * d, axis=1)))
    return lam * L, 2.0 * lam * mbar[:, None] * d
