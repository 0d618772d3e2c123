"""FP64 oracle of the per-Gaussian spatiotemporal motion-probability update.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. IV-A and Eq. (17) step by step, one view:

  per pixel p (the "features" of the hot path are the image pixels)
    e(p)        residual between observed and rendered RGB-D: the hot path has
                no feature matches, so the reprojection error of Eq. (3) is
                read as |D_obs - D_rend| + kappa_c * ||C_obs - C_rend||_1 (m);
                the depth term only where D_obs > 0
    region k    the instance label of p (0 = background, its own region)
    mu_e, sigma_e, e_ub   Eq. (4) over the region's pixels (population std);
                e_ub is floored at e_floor (a reading: without it a static
                instance normalises its own noise to MP_geo ~ 1); the
                background pixels normalise by the background region's e_ub
                (Eq. (4) is a statistic of a region; the background is the
                region no instance claims)
    MP_geo      Eq. (5); inside an instance whose sigma_e < sigma_min the
                instance mean replaces e(p) ("use the instance-mean error")
    MP_ins, Gamma_ins     Eq. (2) from the instance table (row 0 = background)
    Gamma_geo   exp(-sigma / sigma_g) (the sentence after Eq. (7)): for a
                pixel of instance k, sigma = sigma_e,k of its region; for a
                pixel no instance claims, sigma = the population std of e
                over the pixel's associated neighbourhood, read as the disk
                of Eq. (1) centred on the pixel: the pixels (i + di, j + dj)
                of the image with di^2 + dj^2 <= r_s^2, whatever their label
    K_p, M_p    Eqs. (6), (7)  (fusion_mode 1 forces K = 0, 2 forces K = 1)
  per Gaussian G
    N(G)        Eq. (1): the union over pyramid levels s = 0 .. S-1 of the
                level-s pixels within r_s of pi(G) / 2^s (S = cfg.scales;
                level s + 1 is the 2x2 box mean of level s for M_p and e and
                the 2x2 max for D_rend, odd last rows/columns dropped);
                w(p, G) = 2^-s exp(-|p - pi(G) / 2^s|^2 / (2 sigma_w^2))
                for a member of level s (S = 1: the single-scale disk)
    observed    z > z_near, N(G) non-empty, and not behind the rendered
                surface: z <= max_{N(G)} D_rend + vis_tol
    M_hat       Eq. (8)
    U           Eq. (10): binary entropy of M^{t-1} (natural log, eps) +
                lambda_u * Var{M_p} (population variance over N(G))
    U_tilde     min-max normalisation over the observed Gaussians (0 if all equal)
    C           exp(-sigma_e,G / sigma_c), sigma_e,G = population std of e over N(G)
    alpha       Eq. (11); alpha' = rho * alpha when the prior was not
                refreshed, Eq. (17)
    M^t         Eq. (9)
  per frame
    tau         Eq. (12) with the lower median of M^t over observed Gaussians
    labels      dynamic iff M^t > tau; unobserved Gaussians keep M and label
    U_bar       Eq. (13): lower median of U_tilde over observed Gaussians

An external per-pixel MP map (the learned proposal between semantic
invocations, not in the paper) may replace M_p in the association.

Pins: the K = 0 / K = 1 special cases, fixed and instant rates, the rho
scaling, M in [0, 1], tau >= 0.5, unobserved unchanged, the external map
reducing to the fused M_p and to a constant, and closed-form cases in
tests/test_oracle_mp.py.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np


@dataclass
class MPConfig:
    kappa_c: float = 0.05      # m per unit of L1 colour residual
    lam: float = 2.0           # lambda in e_ub = mu_e + lambda sigma_e, Eq. (4)
    sigma_min: float = 0.005   # "sigma_e is small" threshold (m)
    e_floor: float = 0.05      # floor on e_ub (m)
    sigma_g: float = 0.05      # Gamma_geo scale (m), Eq. (7)
    sigma_c: float = 0.05      # C scale (m), Eq. (11)
    lam_u: float = 1.0         # lambda_u, Eq. (10)
    eps: float = 1e-6          # epsilon, Eq. (10)
    alpha_min: float = 0.05
    alpha_max: float = 0.6
    rho: float = 0.5           # Eq. (17)
    r_s: float = 2.0           # association radius (px), Eq. (1)
    sigma_w: float = 1.0       # association kernel width (px)
    vis_tol: float = 0.1       # occlusion tolerance (m); <= 0 disables
    z_near: float = 0.2
    tau_floor: float = 0.5     # Eq. (12)
    fusion_mode: int = 0       # 0 fused, 1 K = 0 (MP_ins only), 2 K = 1 (MP_geo only)
    scales: int = 1            # pyramid levels S of the association, Eq. (1)

    def as_dict(self):
        return asdict(self)


def lower_median(x: np.ndarray) -> float:
    """Element at index floor((n-1)/2) of the ascending sort."""
    s = np.sort(np.asarray(x, dtype=np.float64))
    return float(s[(len(s) - 1) // 2])


def pyramid(x, W, H, S, pool):
    """Levels 0 .. S-1 of a per-pixel map: level 0 is x (H x W); level s + 1
    has floor(W_s / 2) x floor(H_s / 2) pixels, each the mean (pool = "mean")
    or the maximum (pool = "max") of the 2 x 2 level-s pixels it covers.
    Returns [(flat values, W_s, H_s)]."""
    a = np.asarray(x, np.float64).reshape(H, W)
    out = [(a.ravel(), W, H)]
    for _ in range(1, S):
        h, w = a.shape[0] // 2, a.shape[1] // 2
        q = a[:2 * h, :2 * w].reshape(h, 2, w, 2)
        a = q.mean(axis=(1, 3)) if pool == "mean" else q.max(axis=(1, 3))
        out.append((a.ravel(), w, h))
    return out


def neighbourhood_std(e, W, H, r_s):
    """Population std of e over each pixel's disk {(di, dj): di^2 + dj^2 <=
    r_s^2} clipped to the image (the associated neighbourhood of a pixel that
    no instance claims, sentence after Eq. (7)). Two passes: the mean over
    the disk, then the mean squared deviation from it."""
    e = np.asarray(e, np.float64).reshape(H, W)
    R = int(np.floor(r_s))
    offs = [(di, dj) for dj in range(-R, R + 1) for di in range(-R, R + 1) if di * di + dj * dj <= r_s * r_s]

    def shifted(a, di, dj):
        # out[j, i] = a[j + dj, i + di] where that pixel exists, else nan
        out = np.full((H, W), np.nan)
        ys, ye = max(0, -dj), min(H, H - dj)
        xs, xe = max(0, -di), min(W, W - di)
        if ys < ye and xs < xe:
            out[ys:ye, xs:xe] = a[ys + dj:ye + dj, xs + di:xe + di]
        return out

    cnt = np.zeros((H, W))
    tot = np.zeros((H, W))
    for di, dj in offs:
        sv = shifted(e, di, dj)
        ok = ~np.isnan(sv)
        cnt += ok
        tot += np.where(ok, sv, 0.0)
    mean = tot / cnt
    sq = np.zeros((H, W))
    for di, dj in offs:
        sv = shifted(e, di, dj)
        ok = ~np.isnan(sv)
        sq += np.where(ok, (sv - mean) ** 2, 0.0)
    return np.sqrt(sq / cnt).ravel()


def pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, table, cfg: MPConfig, shape):
    """Per-pixel fused MP observation on a W x H image (shape = (W, H)).
    Returns dict(e, e_used, M_p, K, sigma_geo (the dispersion in Gamma_geo),
    region stats (count, mean, std, e_ub) per label)."""
    W, H = int(shape[0]), int(shape[1])
    inst = np.asarray(inst).astype(np.int64).ravel()
    d_obs = np.asarray(d_obs, np.float64).ravel()
    d_rend = np.asarray(d_rend, np.float64).ravel()
    c_obs = np.asarray(c_obs, np.float64).reshape(-1, 3)
    c_rend = np.asarray(c_rend, np.float64).reshape(-1, 3)
    table = np.asarray(table, np.float64).reshape(-1, 2)
    nreg = table.shape[0]
    e = np.where(d_obs > 0, np.abs(d_obs - d_rend), 0.0) + cfg.kappa_c * np.abs(c_obs - c_rend).sum(1)
    cnt = np.zeros(nreg)
    mean = np.zeros(nreg)
    std = np.zeros(nreg)
    for k in range(nreg):
        sel = e[inst == k]
        cnt[k] = sel.size
        if sel.size:
            mean[k] = sel.mean()
            std[k] = np.sqrt(np.mean((sel - mean[k]) ** 2))
    e_ub = np.maximum(mean + cfg.lam * std, cfg.e_floor)
    small = (np.arange(nreg) >= 1) & (std < cfg.sigma_min)
    e_used = np.where(small[inst], mean[inst], e)
    mp_geo = np.clip(e_used / e_ub[inst], 0.0, 1.0)
    mp_ins = table[inst, 0]
    g_ins = table[inst, 1]
    sigma_geo = std[inst]
    bg = inst == 0
    if bg.any():
        sigma_geo = np.where(bg, neighbourhood_std(e, W, H, cfg.r_s), sigma_geo)
    g_geo = np.exp(-sigma_geo / cfg.sigma_g)
    K = g_geo / (g_ins + g_geo)
    if cfg.fusion_mode == 1:
        K = np.zeros_like(K)
    elif cfg.fusion_mode == 2:
        K = np.ones_like(K)
    M_p = (1.0 - K) * mp_ins + K * mp_geo
    return dict(e=e, e_used=e_used, mp_geo=mp_geo, mp_ins=mp_ins, K=K, M_p=M_p, count=cnt, mean=mean,
                std=std, e_ub=e_ub, sigma_geo=sigma_geo)


def mp_update(means, mp_prev, labels_prev, cam, pose, inst, d_obs, c_obs, d_rend, c_rend, table,
              cfg: MPConfig = None, seg_refreshed: bool = True, mp_map=None):
    """One MP update. cam = (fx, fy, cx, cy, W, H); pose 3x4 world->camera.

    mp_map: optional per-pixel MP (e.g. the learned network's proposal
    between semantic invocations); when given it stands in for the fused M_p
    of Eqs. (2)-(7) in the association of Eqs. (8) and (10). The residuals
    (sigma_e,G, C) and the region statistics still come from the frame.

    Returns dict with mp (n), labels (n, uint8), observed (n bool), m_hat,
    U, U_tilde, alpha (after Eq. (17)), tau, U_bar, median_M, the pixel dict,
    and decision-margin flags: label_flag (|M^t - tau| small), disk_flag (a
    pixel within FP32 coordinate rounding of the association radius),
    vis_flag (occlusion test within 1e-5).
    """
    cfg = MPConfig() if cfg is None else cfg
    fx, fy, cx, cy, W, H = cam
    W, H = int(W), int(H)
    px = pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, table, cfg, (W, H))
    M_p, e = px["M_p"], px["e"]
    if mp_map is not None:
        M_p = np.asarray(mp_map, np.float64).ravel()
    d_rend = np.asarray(d_rend, np.float64).ravel()
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    pose = np.asarray(pose, np.float64).reshape(3, 4)
    pc = means @ pose[:, :3].T + pose[:, 3]
    mp_prev = np.asarray(mp_prev, np.float64)
    out_mp = mp_prev.copy()
    labels = np.asarray(labels_prev).astype(np.uint8).copy()
    observed = np.zeros(n, bool)
    m_hat = np.zeros(n)
    var = np.zeros(n)
    sig_e = np.zeros(n)
    disk_flag = np.zeros(n, bool)
    vis_flag = np.zeros(n, bool)
    # Eq. (1) for all Gaussians at once: at each pyramid level the candidate
    # pixels are a square of integer offsets around the scaled projected mean;
    # N(G) keeps those inside the level within r_s, over all levels.
    S = int(cfg.scales)
    lv_m = pyramid(M_p, W, H, S, "mean")
    lv_e = pyramid(e, W, H, S, "mean")
    lv_d = pyramid(d_rend, W, H, S, "max")
    R = int(np.ceil(cfg.r_s)) + 1
    off = np.arange(-R, R + 2)
    oi, oj = np.meshgrid(off, off, indexing="xy")
    oi, oj = oi.ravel(), oj.ravel()
    for c0 in range(0, n, 20000):
        c1 = min(n, c0 + 20000)
        x, y, z = pc[c0:c1, 0], pc[c0:c1, 1], pc[c0:c1, 2]
        front = z > cfg.z_near
        with np.errstate(divide="ignore", invalid="ignore"):
            u = np.where(front, fx * x / z + cx, 0.0)
            v = np.where(front, fy * y / z + cy, 0.0)
        ok_uv = front & np.isfinite(u) & np.isfinite(v) & (np.abs(u) < 1e7) & (np.abs(v) < 1e7)
        u = np.where(ok_uv, u, -1e6)
        v = np.where(ok_uv, v, -1e6)
        # a pixel whose distance lies within the FP32 rounding of the projected
        # centre (a few ulps of |u|, |v|, scaled with the level) of the radius
        # is an undecided member
        ecoord0 = 2.0 ** -22 * np.maximum(np.maximum(np.abs(u), np.abs(v)), 1.0)[:, None]
        sel_l, w_l, m_l, e_l, d_l = [], [], [], [], []
        dflag = np.zeros(c1 - c0, bool)
        for s, ((Mv, Ws, Hs), (Ev, _, _), (Dv, _, _)) in enumerate(zip(lv_m, lv_e, lv_d)):
            us, vs = u / 2.0 ** s, v / 2.0 ** s
            ii = np.floor(us).astype(np.int64)[:, None] + oi[None, :]
            jj = np.floor(vs).astype(np.int64)[:, None] + oj[None, :]
            inside = (ii >= 0) & (ii < Ws) & (jj >= 0) & (jj < Hs) & ok_uv[:, None]
            d2 = (ii - us[:, None]) ** 2 + (jj - vs[:, None]) ** 2
            dmarg = 4.0 * cfg.r_s * ecoord0 / 2.0 ** s + 1e-5 * cfg.r_s ** 2
            dflag |= np.any(inside & (np.abs(d2 - cfg.r_s ** 2) <= dmarg), axis=1)
            sel = inside & (d2 <= cfg.r_s ** 2)
            pidx = np.where(sel, jj * Ws + ii, 0)
            sel_l.append(sel)
            w_l.append(np.where(sel, 2.0 ** -s * np.exp(-d2 / (2.0 * cfg.sigma_w ** 2)), 0.0))
            m_l.append(np.where(sel, Mv[pidx] if Mv.size else 0.0, 0.0))
            e_l.append(np.where(sel, Ev[pidx] if Ev.size else 0.0, 0.0))
            d_l.append(np.where(sel, Dv[pidx] if Dv.size else 0.0, -np.inf))
        disk_flag[c0:c1] = dflag
        sel = np.concatenate(sel_l, axis=1)
        w = np.concatenate(w_l, axis=1)
        mps = np.concatenate(m_l, axis=1)
        es = np.concatenate(e_l, axis=1)
        cnt = sel.sum(1)
        dmax = np.concatenate(d_l, axis=1).max(1)
        lim = dmax + cfg.vis_tol
        occl = (cfg.vis_tol > 0) & (dmax > 0) & (z > lim)
        vis_flag[c0:c1] = (cfg.vis_tol > 0) & (dmax > 0) & (np.abs(z - lim) <= 1e-5 * np.abs(lim))
        obs = (cnt > 0) & ~occl
        cntf = np.maximum(cnt, 1)
        with np.errstate(invalid="ignore", divide="ignore"):
            mh = (w * mps).sum(1) / w.sum(1)                      # Eq. (8)
        mm = mps.sum(1) / cntf
        vv = np.where(sel, (mps - mm[:, None]) ** 2, 0.0).sum(1) / cntf
        me = es.sum(1) / cntf
        se = np.sqrt(np.where(sel, (es - me[:, None]) ** 2, 0.0).sum(1) / cntf)
        observed[c0:c1] = obs
        m_hat[c0:c1] = np.where(obs, mh, 0.0)
        var[c0:c1] = np.where(obs, vv, 0.0)
        sig_e[c0:c1] = np.where(obs, se, 0.0)
    M0 = mp_prev
    ent = -M0 * np.log(M0 + cfg.eps) - (1.0 - M0) * np.log(1.0 - M0 + cfg.eps)
    U = ent + cfg.lam_u * var
    U_t = np.zeros(n)
    alpha = np.zeros(n)
    tau = cfg.tau_floor
    U_bar = 0.0
    med = float("nan")
    label_flag = np.zeros(n, bool)
    if observed.any():
        uo = U[observed]
        umin, umax = uo.min(), uo.max()
        if umax > umin:
            U_t[observed] = (uo - umin) / (umax - umin)
        C = np.exp(-sig_e / cfg.sigma_c)
        a = cfg.alpha_min + (cfg.alpha_max - cfg.alpha_min) * (1.0 - U_t) * C
        a = np.clip(a, cfg.alpha_min, cfg.alpha_max)
        if not seg_refreshed:
            a = cfg.rho * a
        alpha = np.where(observed, a, 0.0)
        out_mp = np.where(observed, (1.0 - alpha) * M0 + alpha * m_hat, M0)
        med = lower_median(out_mp[observed])
        tau = max(med, cfg.tau_floor)
        U_bar = lower_median(U_t[observed])
        labels = np.where(observed, (out_mp > tau).astype(np.uint8), labels).astype(np.uint8)
        label_flag = observed & (np.abs(out_mp - tau) <= 1e-5)
    return dict(mp=out_mp, labels=labels, observed=observed, m_hat=m_hat, var=var, sigma_e=sig_e, U=U,
                U_tilde=U_t, alpha=alpha, tau=tau, U_bar=U_bar, median_M=med, pixel=px,
                label_flag=label_flag, disk_flag=disk_flag, vis_flag=vis_flag)
