"""FP64 oracle of the Levenberg-Marquardt pose refinement (Sec. V-A(c)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper states only that camera poses are refined with Levenberg-Marquardt.
The reading, step by step, for the MP-weighted L1 objective of Eqs. (20)-(22)
with w(u) held constant in the linearisation:

  linearise  at the pose T_try: the loss L, and the IRLS normal equations
             H = sum W J J^T, g = sum W r J (oracle.render_jac)
  accept     if L < L_best (always on the first iteration): T_best = T_try,
             keep (L, H, g), mu <- max(mu * down, mu_min);
             otherwise keep T_best and its (H, g), mu <- min(mu * up, mu_max)
  solve      (H + mu diag(H) + floor (tr H / 6) I) Delta = -g; Delta = 0
             when tr H <= 0 (nothing observed)
  step       T_try = exp(Delta^) T_best (left perturbation, oracle.pose)

Each iteration renders once; the pose returned is T_best. A rejected
linearisation costs one render and raises the damping.

Pins (tests/test_oracle_lm.py): on a linear least-squares model one undamped
step lands on numpy's lstsq solution; large damping gives the scaled
steepest-descent step; the accept/reject bookkeeping on scripted losses; a
pure-translation model converging in one accepted step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import pose as opose


@dataclass
class LMConfig:
    mu0: float = 1e-2      # initial damping
    mu_min: float = 1e-9
    mu_max: float = 1e9
    down: float = 0.1      # damping factor after an accepted step
    up: float = 10.0       # damping factor after a rejected step
    delta: float = 0.01    # IRLS floor on |r| (colour units and metres)
    floor: float = 1e-9    # ridge, relative to tr(H) / 6


def solve(H, g, mu, floor=1e-9):
    """The damped step Delta of one LM iteration."""
    H = np.asarray(H, np.float64)
    tr = float(np.trace(H))
    if not tr > 0.0:
        return np.zeros(6)
    A = H + mu * np.diag(np.diag(H)) + floor * (tr / 6.0) * np.eye(6)
    return np.linalg.solve(A, -np.asarray(g, np.float64))


def track(normal_fn, pose0, iters, cfg: LMConfig = None):
    """Run `iters` LM iterations from pose0 (3x4). normal_fn(pose) returns
    (L, H, g) at a pose. Returns (T_best, history) with history a list of
    dicts (L, accepted, mu after the decision, Delta)."""
    cfg = LMConfig() if cfg is None else cfg
    T_try = np.asarray(pose0, np.float64).reshape(3, 4).copy()
    T_best, L_best, H_best, g_best = T_try.copy(), np.inf, None, None
    mu = cfg.mu0
    hist = []
    for _ in range(iters):
        L, H, g = normal_fn(T_try)
        accepted = bool(L < L_best)
        if accepted:
            T_best, L_best, H_best, g_best = T_try.copy(), L, np.asarray(H), np.asarray(g)
            mu = max(mu * cfg.down, cfg.mu_min)
        else:
            mu = min(mu * cfg.up, cfg.mu_max)
        d = solve(H_best, g_best, mu, cfg.floor)
        T_try = opose.apply_left(d, T_best)
        hist.append(dict(L=L, accepted=accepted, mu=mu, delta=d))
    return T_best, hist
