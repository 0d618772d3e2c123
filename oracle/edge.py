"""FP64 oracle of the MP-guided edge-warp regulariser (Sec. IV-D, Eqs. (25),
(26)).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For an edge pixel u of frame i, with the aligned depth observation D_i(u):
  X   = D_i(u) K^-1 [u_x, u_y, 1]                    back-projection
  Y   = T_ji X,  T_ji = T_jW T_iW^-1                 frame j coordinates
  u'  = pi(K Y)                                      Eq. (25)
  r   = w^j(u') (D_j(u') - z_ref)                    D_j, w^j bilinear at u'
  L   = lambda_4 sum_u rho(r)                        Eq. (26), rho Huber

Readings (the paper leaves these open):
- Edge pixels E_i: depth discontinuities of the observation, relative to the
  depth (sensor noise grows with it). u is an edge if D_i(u) > 0 and some
  4-neighbour n with D_i(n) > 0 has |D_i(n) - D_i(u)| > edge_rel D_i(u)
  (edge_rel = 0.05).
- z_ref: the depth of the warped point in frame j, Y_z. Eq. (26) writes
  D_i(u), which equals Y_z only when the relative motion has no component
  along the viewing direction; literal=True uses D_i(u).
- Pixel centres are the integer coordinates (u = i). Bilinear sampling uses
  the four pixels around u'; a pixel counts only if all four lie in the image
  with D_j > 0 and Y_z > z_near (0.2 m).
- rho is the Huber kernel with threshold delta_h (0.05 m): r^2 / 2 for
  |r| <= delta_h, delta_h (|r| - delta_h / 2) beyond.
- w^j is the static-weight map of frame j (Eq. (20), channel 7 of a
  splat_forward image), held constant; lambda_4 = 300 (Sec. V-A(c)).
- Gradients are with respect to the left-perturbation twists of the two
  world-to-camera poses, T <- exp(xi^) T.

Decisions that a float can take differently are flagged: an edge test within
1e-5 relative of its threshold, u' within 1e-3 px of a cell boundary or the image
border, Y_z within 1e-5 of z_near, |r| within 1e-5 relative of delta_h.

Pins (tests/test_oracle_edge.py): the Huber kernel against scipy; identical
frames under one pose give zero; invariance under a global rigid motion of
both poses; L scales by s^2 when depths, translations and thresholds scale
by s; the literal reading equals the default under lateral motion and not
under forward motion; central differences of both twist gradients.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class EdgeConfig:
    edge_rel: float = 0.05
    huber: float = 0.05
    z_near: float = 0.2
    lam: float = 300.0
    literal: bool = False


def edge_mask(D, W, H, rel):
    """(edge bool [H*W], flag bool [H*W]) of the depth discontinuities:
    a valid 4-neighbour differs by more than rel D(u)."""
    D = np.asarray(D, np.float64).reshape(H, W)
    edge = np.zeros((H, W), bool)
    flag = np.zeros((H, W), bool)
    valid = D > 0
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        n = np.zeros_like(D)
        nv = np.zeros_like(valid)
        ys = slice(max(0, dy), H + min(0, dy))
        yd = slice(max(0, -dy), H + min(0, -dy))
        xs = slice(max(0, dx), W + min(0, dx))
        xd = slice(max(0, -dx), W + min(0, -dx))
        n[yd, xd] = D[ys, xs]
        nv[yd, xd] = valid[ys, xs]
        diff = np.abs(n - D)
        thr = rel * D
        ok = valid & nv
        edge |= ok & (diff > thr)
        flag |= ok & (np.abs(diff - thr) <= 1e-5 * thr)
    return edge.ravel(), flag.ravel()


def huber(r, d):
    a = np.abs(r)
    return np.where(a <= d, 0.5 * r * r, d * (a - 0.5 * d)), np.where(a <= d, r, d * np.sign(r))


def edge_warp(cam, Di, Dj, wj, pose_i, pose_j, cfg: EdgeConfig = None):
    """Returns dict(L, grad_i (6), grad_j (6), n (pixels counted), flagged).
    cam = (fx, fy, cx, cy, W, H); Di, Dj, wj: H*W arrays; poses 3x4 world->camera."""
    cfg = EdgeConfig() if cfg is None else cfg
    fx, fy, cx, cy, W, H = cam
    W, H = int(W), int(H)
    Di = np.asarray(Di, np.float64).ravel()
    Dj = np.asarray(Dj, np.float64).ravel()
    wj = np.asarray(wj, np.float64).ravel()
    Ti = np.asarray(pose_i, np.float64).reshape(3, 4)
    Tj = np.asarray(pose_j, np.float64).reshape(3, 4)
    Ri, ti, Rj, tj = Ti[:, :3], Ti[:, 3], Tj[:, :3], Tj[:, 3]
    R = Rj @ Ri.T
    t = tj - R @ ti
    edge, flag = edge_mask(Di, W, H, cfg.edge_rel)
    L = 0.0
    gi = np.zeros(6)
    gj = np.zeros(6)
    n = 0
    nflag = int(flag.sum())
    for p in np.nonzero(edge)[0]:
        y, x = divmod(int(p), W)
        d = Di[p]
        X = np.array([d * (x - cx) / fx, d * (y - cy) / fy, d])
        Y = R @ X + t
        if abs(Y[2] - cfg.z_near) <= 1e-5:
            nflag += 1
        if not Y[2] > cfg.z_near:
            continue
        u = fx * Y[0] / Y[2] + cx
        v = fy * Y[1] / Y[2] + cy
        x0, y0 = int(np.floor(u)), int(np.floor(v))
        fu, fv = u - x0, v - y0
        if min(fu, 1 - fu, fv, 1 - fv) <= 1e-3 or min(abs(u), abs(u - (W - 1)), abs(v), abs(v - (H - 1))) <= 1e-3:
            nflag += 1
        if x0 < 0 or y0 < 0 or x0 + 1 > W - 1 or y0 + 1 > H - 1:
            continue
        q = [y0 * W + x0, y0 * W + x0 + 1, (y0 + 1) * W + x0, (y0 + 1) * W + x0 + 1]
        if np.any(Dj[q] <= 0):
            continue
        wts = np.array([(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv])
        dU = np.array([-(1 - fv), 1 - fv, -fv, fv])       # d wts / d u
        dV = np.array([-(1 - fu), -fu, 1 - fu, fu])       # d wts / d v
        Ds, ws = wts @ Dj[q], wts @ wj[q]
        zref = d if cfg.literal else Y[2]
        r = ws * (Ds - zref)
        if abs(abs(r) - cfg.huber) <= 1e-5 * cfg.huber:
            nflag += 1
        rho, drho = huber(r, cfg.huber)
        L += float(rho)
        n += 1
        # dr/du', dr/dv', then d(u', v')/dY and dr/dY
        dr_du = (dU @ wj[q]) * (Ds - zref) + ws * (dU @ Dj[q])
        dr_dv = (dV @ wj[q]) * (Ds - zref) + ws * (dV @ Dj[q])
        duY = np.array([fx / Y[2], 0.0, -fx * Y[0] / Y[2] ** 2])
        dvY = np.array([0.0, fy / Y[2], -fy * Y[1] / Y[2] ** 2])
        drY = dr_du * duY + dr_dv * dvY
        if not cfg.literal:
            drY = drY - ws * np.array([0.0, 0.0, 1.0])
        gY = float(drho) * drY
        # pose j: Y <- exp(xi_j) Y, dY = rho_j + phi_j x Y;
        # pose i: Y = T_ji exp(-xi_i) X, dY = -R (rho_i + phi_i x X)
        gj[:3] += gY
        gj[3:] += np.cross(Y, gY)
        gR = R.T @ gY
        gi[:3] -= gR
        gi[3:] -= np.cross(X, gR)
    return dict(L=cfg.lam * L, grad_i=cfg.lam * gi, grad_j=cfg.lam * gj, n=n, flagged=nflag, edges=int(edge.sum()))
