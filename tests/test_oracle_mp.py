"""Pins of the FP64 MP-update oracle: special cases that reduce each step of
Sec. IV-A to a closed form (no GPU)."""
import numpy as np

from oracle import mp as M
from paper_2602_21644_gb300 import synth

W, H = 24, 20
CAM = (30.0, 30.0, 12.0, 10.0, W, H)


def flat_obs(inst=None, e_depth=0.0, d_rend=2.0):
    """Maps where the residual is |D_obs - D_rend| = e_depth everywhere."""
    inst = np.zeros(W * H, np.uint8) if inst is None else inst
    d_obs = np.full(W * H, d_rend + e_depth)
    c = np.full((W * H, 3), 0.5)
    return inst, d_obs, c, np.full(W * H, d_rend), c.copy()


def points_on_grid(n, z=2.0, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(3, W - 4, n)
    v = rng.uniform(3, H - 4, n)
    return np.stack([(u - 12.0) * z / 30.0, (v - 10.0) * z / 30.0, np.full(n, z)], 1)


TABLE = np.array([[0.1, 0.05], [0.9, 0.8]])


def test_lower_median():
    assert M.lower_median([3, 1, 2]) == 2
    assert M.lower_median([4, 1, 3, 2]) == 2
    assert M.lower_median([5.0]) == 5.0


def test_fusion_special_cases():
    rng = np.random.default_rng(0)
    inst = (rng.random(W * H) < 0.3).astype(np.uint8)
    d_obs = rng.uniform(1, 3, W * H)
    d_rend = d_obs + rng.normal(0, 0.1, W * H)
    c_obs = rng.uniform(0, 1, (W * H, 3))
    c_rend = rng.uniform(0, 1, (W * H, 3))
    k0 = M.pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, TABLE, M.MPConfig(fusion_mode=1), (W, H))
    np.testing.assert_array_equal(k0["M_p"], TABLE[inst, 0])          # K = 0: MP_ins, Eq. (2)
    k1 = M.pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, TABLE, M.MPConfig(fusion_mode=2), (W, H))
    np.testing.assert_array_equal(k1["M_p"], k1["mp_geo"])             # K = 1: MP_geo
    fz = M.pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, TABLE, M.MPConfig(), (W, H))
    lo = np.minimum(fz["mp_ins"], fz["mp_geo"]) - 1e-15
    hi = np.maximum(fz["mp_ins"], fz["mp_geo"]) + 1e-15
    assert np.all((fz["M_p"] >= lo) & (fz["M_p"] <= hi))                # convex combination
    assert np.all((fz["K"] >= 0) & (fz["K"] <= 1))


def test_geometric_mp_closed_form():
    # Region statistics by hand: background residuals 0.01 / 0.03 alternating
    # (mean 0.02, std 0.01) -> e_ub = max(0.02 + 2 * 0.01, 0.05) = 0.05;
    # instance residual 0.3 everywhere (std 0 < sigma_min -> instance mean).
    inst = np.zeros(W * H, np.uint8)
    inst[: W * 4] = 1
    e = np.where(np.arange(W * H) % 2 == 0, 0.01, 0.03)
    e[inst == 1] = 0.3
    d_rend = np.full(W * H, 2.0)
    c = np.full((W * H, 3), 0.5)
    cfg = M.MPConfig()
    px = M.pixel_mp(inst, d_rend + e, c, d_rend, c, TABLE, cfg, (W, H))
    np.testing.assert_allclose(px["mean"], [0.02, 0.3], rtol=1e-12)
    np.testing.assert_allclose(px["std"], [0.01, 0.0], atol=1e-12)
    np.testing.assert_allclose(px["e_ub"], [0.05, 0.3], rtol=1e-12)
    bg = inst == 0
    np.testing.assert_allclose(px["mp_geo"][bg], e[bg] / 0.05, rtol=1e-12)
    np.testing.assert_allclose(px["mp_geo"][~bg], 1.0, rtol=1e-12)
    # Gamma_geo of a background pixel uses the dispersion over its own disk of
    # radius 2 (13 pixels): away from the instance and the image border, 7 of
    # them share the pixel's column parity (di in {0, +-2}) and 6 do not, so
    # sigma = |0.03 - 0.01| sqrt(p (1 - p)) with p = 7/13
    jj, ii = np.divmod(np.arange(W * H), W)
    interior = bg & (jj >= 6) & (jj <= H - 3) & (ii >= 2) & (ii <= W - 3)
    sig = 0.02 * np.sqrt(7 * 6) / 13
    np.testing.assert_allclose(px["sigma_geo"][interior], sig, rtol=1e-12)
    g_geo_bg = np.exp(-sig / 0.05)
    K_bg = g_geo_bg / (0.05 + g_geo_bg)
    np.testing.assert_allclose(px["K"][interior], K_bg, rtol=1e-12)
    np.testing.assert_allclose(px["M_p"][interior], (1 - K_bg) * 0.1 + K_bg * e[interior] / 0.05, rtol=1e-12)
    K_in = 1.0 / (0.8 + 1.0)
    np.testing.assert_allclose(px["M_p"][~bg], (1 - K_in) * 0.9 + K_in * 1.0, rtol=1e-12)


def test_background_gamma_uses_the_pixel_neighbourhood():
    # Sentence after Eq. (7): a pixel that no instance claims takes the
    # dispersion of e "within the associated neighborhood", here its disk of
    # radius r_s = 2 clipped to the image. One residual of 1 at pixel (0, 0)
    # and a 3x3 patch of 1 at columns 10-12, rows 8-10; everything else 0.
    e = np.zeros((H, W))
    e[0, 0] = 1.0
    e[8:11, 10:13] = 1.0
    inst = np.zeros(W * H, np.uint8)
    d_rend = np.full(W * H, 2.0)
    c = np.full((W * H, 3), 0.5)
    cfg = M.MPConfig()
    px = M.pixel_mp(inst, d_rend + e.ravel(), c, d_rend, c, TABLE, cfg, (W, H))
    sg = px["sigma_geo"].reshape(H, W)
    # (0, 0): the disk clipped to 6 pixels, one of them 1
    assert abs(sg[0, 0] - np.sqrt(5.0) / 6.0) < 1e-12
    # (1, 1): 11 pixels ((-1, 1) and (1, -1) fall outside), one of them 1
    assert abs(sg[1, 1] - np.sqrt(10.0) / 11.0) < 1e-12
    # (14, 9): two to the right of the patch; only (12, 9) of its 13 is 1
    assert abs(sg[9, 14] - np.sqrt(12.0) / 13.0) < 1e-12
    # (15, 9): three to the right; nothing of the patch in its disk
    assert sg[9, 15] == 0.0 and sg[4, 4] == 0.0
    # inside the patch centre all 9 patch pixels and 4 zeros ((0, +-2), (+-2, 0))
    assert abs(sg[9, 11] - np.sqrt(9 * 4) / 13.0) < 1e-12
    # Gamma_geo and K follow: exp(-sigma / sigma_g), K = G / (c_bg + G)
    g = np.exp(-px["sigma_geo"] / cfg.sigma_g)
    np.testing.assert_allclose(px["K"], g / (TABLE[0, 1] + g), rtol=1e-13)
    # the one-region reading would give every background pixel the same K
    assert np.ptp(px["K"]) > 0.1


def test_neighbourhood_std_against_brute_force():
    rng = np.random.default_rng(5)
    w, h = 9, 7
    e = rng.uniform(0, 1, (h, w))
    for r_s in (1.0, 2.0, 2.5):
        got = M.neighbourhood_std(e.ravel(), w, h, r_s).reshape(h, w)
        for y in range(h):
            for x in range(w):
                vals = [e[yy, xx] for yy in range(h) for xx in range(w)
                        if (xx - x) ** 2 + (yy - y) ** 2 <= r_s * r_s]
                assert abs(got[y, x] - np.std(vals)) < 1e-12


def test_instance_pixels_keep_the_region_dispersion():
    # an instance pixel's Gamma_geo is the region's: a single outlier inside
    # the instance changes every instance pixel's K alike
    inst = np.zeros(W * H, np.uint8)
    inst[W * 10:W * 14] = 1
    e = np.zeros(W * H)
    e[W * 12 + 5] = 0.5
    d_rend = np.full(W * H, 2.0)
    c = np.full((W * H, 3), 0.5)
    px = M.pixel_mp(inst, d_rend + e, c, d_rend, c, TABLE, M.MPConfig(), (W, H))
    sel = e[inst == 1]
    np.testing.assert_allclose(px["sigma_geo"][inst == 1], np.std(sel), rtol=1e-12)


def test_instant_update_equals_observation():
    # alpha_min = alpha_max = 1 -> M^t = M_hat (Instant MP, Sec. V-E Ablation I)
    # and with uniform M_p the observation is that value exactly.
    n = 40
    means = points_on_grid(n)
    inst, d_obs, c, d_rend, c2 = flat_obs()
    cfg = M.MPConfig(alpha_min=1.0, alpha_max=1.0, fusion_mode=1)
    r = M.mp_update(means, np.full(n, 0.7), np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c,
                    d_rend, c2, TABLE, cfg)
    assert r["observed"].all()
    np.testing.assert_allclose(r["mp"], 0.1, rtol=1e-12)
    assert r["tau"] == 0.5 and not r["labels"].any()


def test_fixed_rate_and_rho():
    n = 30
    means = points_on_grid(n, seed=1)
    inst, d_obs, c, d_rend, c2 = flat_obs()
    prev = np.linspace(0.05, 0.95, n)
    cfg = M.MPConfig(alpha_min=0.3, alpha_max=0.3, fusion_mode=1)
    r = M.mp_update(means, prev, np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c, d_rend, c2,
                    TABLE, cfg)
    np.testing.assert_allclose(r["mp"], 0.7 * prev + 0.3 * 0.1, rtol=1e-12)    # Eq. (9), fixed rate
    r2 = M.mp_update(means, prev, np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c, d_rend, c2,
                     TABLE, cfg, seg_refreshed=False)
    np.testing.assert_allclose(r2["mp"], (1 - 0.15) * prev + 0.15 * 0.1, rtol=1e-12)  # Eq. (17), rho = 0.5


def test_adaptive_rate_closed_form():
    # Two observed Gaussians with known uncertainty: Var{M_p} = 0 (uniform map)
    # so U is the entropy of M^{t-1}; min-max normalisation gives U~ = 0 for the
    # more certain and 1 for the less certain one. With sigma_e,G = 0, C = 1:
    # alpha = alpha_max for the first and alpha_min for the second (Eq. (11)).
    means = points_on_grid(2, seed=2)
    inst, d_obs, c, d_rend, c2 = flat_obs()
    prev = np.array([0.05, 0.45])
    cfg = M.MPConfig(fusion_mode=1)
    r = M.mp_update(means, prev, np.zeros(2, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c, d_rend, c2,
                    TABLE, cfg)
    ent = -prev * np.log(prev + 1e-6) - (1 - prev) * np.log(1 - prev + 1e-6)
    np.testing.assert_allclose(r["U"], ent, rtol=1e-12)
    np.testing.assert_allclose(r["U_tilde"], [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(r["alpha"], [0.6, 0.05], rtol=1e-12)
    np.testing.assert_allclose(r["mp"], (1 - r["alpha"]) * prev + r["alpha"] * 0.1, rtol=1e-12)
    assert r["U_bar"] == 0.0                                      # lower median of {0, 1}


def test_weighted_observation_and_variance():
    # One Gaussian projected exactly on a pixel centre p0 of a map where
    # M_p = 1 at p0 and 0 elsewhere (K = 0, table values): its disk of radius 2
    # holds 13 pixels; M_hat = 1 / sum_{13} exp(-d^2/2) and Var = (1/13)(12/13).
    n = 1
    z = 2.0
    means = np.array([[(15 - 12.0) * z / 30.0, (9 - 10.0) * z / 30.0, z]])
    inst = np.zeros(W * H, np.uint8)
    inst[9 * W + 15] = 1
    table = np.array([[0.0, 0.05], [1.0, 0.8]])
    d_rend = np.full(W * H, 2.0)
    c = np.full((W * H, 3), 0.5)
    cfg = M.MPConfig(fusion_mode=1, alpha_min=1.0, alpha_max=1.0)
    r = M.mp_update(means, np.array([0.5]), np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_rend, c,
                    d_rend, c, table, cfg)
    d2 = np.array([0, 1, 1, 1, 1, 2, 2, 2, 2, 4, 4, 4, 4], float)
    np.testing.assert_allclose(r["m_hat"], 1.0 / np.exp(-d2 / 2).sum(), rtol=1e-12)
    np.testing.assert_allclose(r["var"], (1 / 13) * (12 / 13), rtol=1e-12)


def test_unobserved_unchanged_and_bounds():
    rng = np.random.default_rng(4)
    n = 200
    means = np.concatenate([points_on_grid(150, seed=3), [[0, 0, -1.0]] * 10,        # behind the camera
                            [[50.0, 0, 2.0]] * 10,                                   # outside the image
                            points_on_grid(30, z=3.0, seed=5)])                       # occluded (behind 2 m)
    inst = (rng.random(W * H) < 0.3).astype(np.uint8)
    d_obs = rng.uniform(1.5, 2.5, W * H)
    d_rend = np.full(W * H, 2.0)
    c_obs = rng.uniform(0, 1, (W * H, 3))
    c_rend = rng.uniform(0, 1, (W * H, 3))
    prev = rng.uniform(0, 1, n)
    lab = (rng.random(n) < 0.5).astype(np.uint8)
    for refreshed in (True, False):
        r = M.mp_update(means, prev, lab, CAM, synth.identity_pose(), inst, d_obs, c_obs, d_rend, c_rend, TABLE,
                        M.MPConfig(), refreshed)
        obs = r["observed"]
        assert obs[:150].all() and not obs[150:].any()
        np.testing.assert_array_equal(r["mp"][~obs], prev[~obs])
        np.testing.assert_array_equal(r["labels"][~obs], lab[~obs])
        assert np.all((r["mp"] >= 0) & (r["mp"] <= 1))
        assert r["tau"] >= 0.5
        assert np.all((r["alpha"][obs] >= (0.5 if not refreshed else 1) * 0.05 - 1e-15))
        assert np.all(r["alpha"][obs] <= 0.6 + 1e-15)
        np.testing.assert_array_equal(r["labels"][obs], (r["mp"][obs] > r["tau"]).astype(np.uint8))


def test_external_map_reduces_to_fused_mp():
    # passing the frame's own fused M_p as the external map changes nothing
    rng = np.random.default_rng(12)
    n = 60
    means = points_on_grid(n, seed=3)
    inst = (rng.random(W * H) < 0.3).astype(np.uint8)
    d_rend = rng.uniform(1.9, 2.1, W * H)
    d_obs = d_rend + rng.normal(0, 0.05, W * H)
    c_obs, c_rend = rng.uniform(0, 1, (W * H, 3)), rng.uniform(0, 1, (W * H, 3))
    prev = rng.uniform(0.05, 0.95, n)
    args = (means, prev, np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c_obs, d_rend, c_rend, TABLE)
    a = M.mp_update(*args)
    b = M.mp_update(*args, mp_map=M.pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, TABLE, M.MPConfig(), (W, H))["M_p"])
    for k in ("mp", "m_hat", "var", "U", "alpha"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["labels"], b["labels"])


def test_external_map_closed_forms():
    # a constant map gives M_hat = c and Var = 0; a one-pixel map at the
    # projected centre gives the kernel-weight closed form of Eq. (8)
    n = 1
    z = 2.0
    means = np.array([[(15 - 12.0) * z / 30.0, (9 - 10.0) * z / 30.0, z]])
    inst, d_obs, c, d_rend, c2 = flat_obs()
    cfg = M.MPConfig(alpha_min=1.0, alpha_max=1.0)
    args = (means, np.array([0.5]), np.zeros(n, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c, d_rend, c2,
            TABLE, cfg)
    r = M.mp_update(*args, mp_map=np.full(W * H, 0.8))
    np.testing.assert_allclose(r["m_hat"], 0.8, rtol=1e-14)
    np.testing.assert_allclose(r["var"], 0.0, atol=1e-15)
    np.testing.assert_allclose(r["mp"], 0.8, rtol=1e-14)
    one = np.zeros(W * H)
    one[9 * W + 15] = 1.0
    r = M.mp_update(*args, mp_map=one)
    d2 = np.array([0, 1, 1, 1, 1, 2, 2, 2, 2, 4, 4, 4, 4], float)
    np.testing.assert_allclose(r["m_hat"], 1.0 / np.exp(-d2 / 2).sum(), rtol=1e-12)


def test_pyramid_levels_closed_form():
    # the 2x2 box mean of a linear ramp is the ramp at the block centre, the
    # 2x2 max its value at the block's far corner; odd sizes drop the last
    # row and column
    w, h = 7, 5
    jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    ramp = 0.3 * ii + 0.05 * jj + 1.0
    lv = M.pyramid(ramp.ravel(), w, h, 3, "mean")
    assert [(a.size, ws, hs) for a, ws, hs in lv] == [(35, 7, 5), (6, 3, 2), (1, 1, 1)]
    J, I = np.meshgrid(np.arange(2), np.arange(3), indexing="ij")
    np.testing.assert_allclose(lv[1][0], (0.3 * (2 * I + 0.5) + 0.05 * (2 * J + 0.5) + 1.0).ravel(), rtol=1e-14)
    np.testing.assert_allclose(lv[2][0], [0.3 * 1.5 + 0.05 * 1.5 + 1.0], rtol=1e-14)
    mx = M.pyramid(ramp.ravel(), w, h, 2, "max")
    np.testing.assert_allclose(mx[1][0], (0.3 * (2 * I + 1) + 0.05 * (2 * J + 1) + 1.0).ravel(), rtol=1e-14)


def _at_pixel(i, j, z):
    return np.array([[(i - 12.0) * z / 30.0, (j - 10.0) * z / 30.0, z]])


def test_multiscale_association_closed_form():
    # r_s = 0.5 keeps one pixel per level: (8, 8) at level 0, (4, 4) at
    # level 1, (2, 2) at level 2, each at distance 0; on the map
    # M(i, j) = i / 100 + j / 1000 they hold 0.088, the mean over i, j in
    # {8, 9} (0.0935) and over i, j in 8..11 (0.1045), weighted 1, 1/2, 1/4
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    mp_map = (ii / 100.0 + jj / 1000.0).ravel()
    inst, d_obs, c, d_rend, c2 = flat_obs()
    vals = np.array([0.088, 0.0935, 0.1045])
    wts = np.array([1.0, 0.5, 0.25])
    for S in (1, 2, 3):
        cfg = M.MPConfig(r_s=0.5, scales=S, alpha_min=1.0, alpha_max=1.0)
        r = M.mp_update(_at_pixel(8, 8, 2.0), np.array([0.5]), np.zeros(1, np.uint8), CAM, synth.identity_pose(),
                        inst, d_obs, c, d_rend, c2, TABLE, cfg, mp_map=mp_map)
        v, wt = vals[:S], wts[:S]
        assert r["observed"][0]
        np.testing.assert_allclose(r["m_hat"], (wt * v).sum() / wt.sum(), rtol=1e-13)
        np.testing.assert_allclose(r["var"], ((v - v.mean()) ** 2).mean(), rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(r["mp"], (wt * v).sum() / wt.sum(), rtol=1e-13)


def test_multiscale_reaches_past_the_image_edge():
    # projected at u = -3: the level-0 disk of radius 2 is empty; at level 1
    # (u = -1.5, v = 5) column 0 holds rows 4, 5, 6
    inst, d_obs, c, d_rend, c2 = flat_obs()
    means = _at_pixel(-3, 10, 2.0)
    for S, seen in ((1, False), (2, True), (3, True)):
        r = M.mp_update(means, np.array([0.5]), np.zeros(1, np.uint8), CAM, synth.identity_pose(), inst, d_obs, c,
                        d_rend, c2, TABLE, M.MPConfig(scales=S, alpha_min=1.0, alpha_max=1.0),
                        mp_map=np.full(W * H, 0.7))
        assert r["observed"][0] == seen
        if seen:
            np.testing.assert_allclose(r["mp"], 0.7, rtol=1e-14)
        else:
            assert r["mp"][0] == 0.5


def test_multiscale_occlusion_uses_the_max_pooled_depth():
    # rendered depth 1 except 3 at pixel (9, 9); a Gaussian at depth 2.5 on
    # pixel (8, 8), r_s = 0.5: alone, level 0 puts it behind the surface
    # (2.5 > 1 + 0.1); level 1's pixel (4, 4) covers (9, 9) and its max-pooled
    # depth 3 makes it visible (a box mean, 1.5, would not)
    inst, d_obs, c, d_rend, c2 = flat_obs(d_rend=1.0)
    d_rend = d_rend.copy()
    d_rend[9 * W + 9] = 3.0
    for S, seen in ((1, False), (2, True)):
        r = M.mp_update(_at_pixel(8, 8, 2.5), np.array([0.5]), np.zeros(1, np.uint8), CAM, synth.identity_pose(),
                        inst, d_obs, c, d_rend, c2, TABLE, M.MPConfig(r_s=0.5, scales=S))
        assert r["observed"][0] == seen


def test_multiscale_against_brute_force():
    # every pixel of every level visited one by one, the pyramid built by
    # explicit loops, odd image sizes
    w, h = 13, 11
    cam = (14.0, 14.0, 6.3, 5.1, w, h)
    rng = np.random.default_rng(21)
    n = 40
    z = rng.uniform(1.0, 3.0, n)
    u = rng.uniform(-4.0, w + 3.0, n)
    v = rng.uniform(-4.0, h + 3.0, n)
    means = np.stack([(u - 6.3) * z / 14.0, (v - 5.1) * z / 14.0, z], 1)
    inst = (rng.random(w * h) < 0.3).astype(np.uint8)
    d_rend = rng.uniform(1.0, 3.5, w * h)
    d_obs = d_rend + rng.normal(0, 0.1, w * h)
    c_obs, c_rend = rng.uniform(0, 1, (w * h, 3)), rng.uniform(0, 1, (w * h, 3))
    cfg = M.MPConfig(r_s=1.7, sigma_w=1.3, scales=3, vis_tol=0.3)
    r = M.mp_update(means, rng.uniform(0.05, 0.95, n), np.zeros(n, np.uint8), cam, synth.identity_pose(), inst,
                    d_obs, c_obs, d_rend, c_rend, TABLE, cfg)
    px = M.pixel_mp(inst, d_obs, c_obs, d_rend, c_rend, TABLE, cfg, (w, h))

    def down(grid, pool):
        hh, ww = len(grid) // 2, len(grid[0]) // 2
        out = [[0.0] * ww for _ in range(hh)]
        for J in range(hh):
            for I in range(ww):
                q = [grid[2 * J + a][2 * I + b] for a in (0, 1) for b in (0, 1)]
                out[J][I] = sum(q) / 4.0 if pool == "mean" else max(q)
        return out

    levels = []
    g = [[(px["M_p"][j * w + i], px["e"][j * w + i], d_rend[j * w + i]) for i in range(w)] for j in range(h)]
    gm, ge, gd = ([[t[k] for t in row] for row in g] for k in range(3))
    for s in range(3):
        levels.append((gm, ge, gd))
        gm, ge, gd = down(gm, "mean"), down(ge, "mean"), down(gd, "max")
    for k in range(n):
        mem = []
        for s, (lm, le, ld) in enumerate(levels):
            for j in range(len(lm)):
                for i in range(len(lm[0]) if lm else 0):
                    d2 = (i - u[k] / 2 ** s) ** 2 + (j - v[k] / 2 ** s) ** 2
                    if d2 <= cfg.r_s ** 2:
                        mem.append((2.0 ** -s * np.exp(-d2 / (2 * cfg.sigma_w ** 2)), lm[j][i], le[j][i], ld[j][i]))
        if r["disk_flag"][k] or r["vis_flag"][k]:
            continue
        seen = bool(mem) and not (max(t[3] for t in mem) > 0 and z[k] > max(t[3] for t in mem) + cfg.vis_tol)
        assert r["observed"][k] == seen
        if not seen:
            continue
        wt = np.array([t[0] for t in mem])
        mv = np.array([t[1] for t in mem])
        ev = np.array([t[2] for t in mem])
        np.testing.assert_allclose(r["m_hat"][k], (wt * mv).sum() / wt.sum(), rtol=1e-12)
        np.testing.assert_allclose(r["var"][k], mv.var(), rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(r["sigma_e"][k], ev.std(), rtol=1e-10, atol=1e-15)
    assert r["observed"].sum() > 15
