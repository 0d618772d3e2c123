"""FP64 oracle of the uncertainty-aware semantic-on-demand trigger (Sec. IV-B,
Eqs. (13)-(16)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per frame t, after the MP update of that frame:

  U_bar^t   Eq. (13): the lower median of U_tilde over the observed
            Gaussians; the MP update's own output (oracle.mp.mp_update)
  e_bar^t   the mean reprojection residual over "verified correspondences".
            The hot path has no feature matches, so the residual is the
            per-pixel e(p) of the MP update and the verified set is the
            background region (label 0: the pixels no instance mask claims);
            0 when that region is empty
  R^t       Eq. (14): clip(e_bar / e_ref, 0, 1)
  S^t       Eq. (15): w_u U_bar + w_r R, with w_u, w_r >= 0, w_u + w_r = 1
  trigger   Eq. (16): segmentation runs when S > theta or when the frames
            since the last segmentation reach N_max

Timing (a reading; the paper does not say which frame a trigger serves): the
score of frame t decides whether frame t + 1 gets a fresh instance prior.
Delta t at frame t + 1 counts the frames since the last refresh, so with a
score that never exceeds theta the prior is refreshed every N_max frames.

Pins (tests/test_oracle_schedule.py): the fixed cadence when theta >= 1, the
one-signal cases w_u = 1 and w_r = 1, the clip of Eq. (14) at 0 and e_ref,
the region-0 mean against a direct pixel average of e(p), and the threshold
being strict.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ScheduleConfig:
    w_u: float = 0.5      # weight of U_bar, Eq. (15)
    w_r: float = 0.5      # weight of R, Eq. (15)
    theta: float = 0.35   # trigger threshold, Eq. (16)
    e_ref: float = 0.05   # reference residual (m), Eq. (14)
    n_max: int = 10       # maximum skip interval, Eq. (16)


def residual_mean(e: np.ndarray, inst: np.ndarray) -> float:
    """e_bar: the mean of the per-pixel residual over the background region."""
    e = np.asarray(e, np.float64).ravel()
    bg = np.asarray(inst).ravel() == 0
    return float(e[bg].mean()) if bg.any() else 0.0


def score(U_bar: float, e_bar: float, cfg: ScheduleConfig = None):
    """(R, S) of Eqs. (14), (15)."""
    cfg = ScheduleConfig() if cfg is None else cfg
    R = min(max(e_bar / cfg.e_ref, 0.0), 1.0)
    S = cfg.w_u * U_bar + cfg.w_r * R
    return R, S


def step(U_bar: float, e_bar: float, since: int, seg_refreshed: bool, cfg: ScheduleConfig = None):
    """One frame of the scheduler. since = frames since the last refresh as of
    the previous frame. Returns (since, R, S, refresh_next): since as of this
    frame (0 if this frame was refreshed) and the decision of Eq. (16) for the
    next frame."""
    cfg = ScheduleConfig() if cfg is None else cfg
    since = 0 if seg_refreshed else since + 1
    R, S = score(U_bar, e_bar, cfg)
    refresh_next = bool(S > cfg.theta or since + 1 >= cfg.n_max)
    return since, R, S, refresh_next


def run(U_bars, e_bars, cfg: ScheduleConfig = None):
    """Drive the scheduler over a sequence whose frame 0 is refreshed; frame
    t > 0 is refreshed iff frame t - 1 decided so. Returns the list of
    refreshed frames and the per-frame (R, S)."""
    cfg = ScheduleConfig() if cfg is None else cfg
    refreshed, rs = [], []
    since, nxt = 0, True
    for U, e in zip(U_bars, e_bars):
        cur = nxt
        if cur:
            refreshed.append(len(rs))
        since, R, S, nxt = step(U, e, since, cur, cfg)
        rs.append((R, S))
    return refreshed, rs
