"""Pins of the FP64 splatting oracle against closed forms, invariants, brute
force, library routines and central finite differences (no GPU)."""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2602_21644_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gauss_row(mean, scale, quat=(1, 0, 0, 0), logit=0.0, mp=0.1, rgb=(0.5, 0.25, 0.75)):
    g = np.zeros(oracle.G_STRIDE)
    g[0:3] = mean
    g[3] = logit
    g[4:8] = quat
    g[8:11] = np.log(np.broadcast_to(np.asarray(scale, float), (3,)))
    g[11] = mp
    g[12:15] = rgb
    return g


def ident():
    return synth.identity_pose()


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def pixel_grid(W, H):
    jj, ii = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
    return ii.ravel(), jj.ravel()


def expected_single(W, H, u0, v0, cov2, o, rgb, z, mp):
    """Single Gaussian composited image from its 2D covariance (library inverse)."""
    Q = np.linalg.inv(cov2)
    ii, jj = pixel_grid(W, H)
    d = np.stack([u0 - ii, v0 - jj], 1)
    ag = o * np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, Q, d))
    alpha = np.where(ag >= 1 / 255, np.minimum(ag, 0.99), 0.0)
    out = np.zeros((W * H, oracle.PX_STRIDE))
    out[:, 0:3] = alpha[:, None] * np.asarray(rgb)[None]
    out[:, 3] = z * alpha
    out[:, 4] = alpha
    out[:, 5] = mp * alpha
    out[:, 6] = 1 - alpha
    return out, ag


def test_single_isotropic_on_axis_closed_form():
    # An isotropic 3D Gaussian of std s at depth z on the optical axis projects
    # to an isotropic 2D Gaussian of variance (f s / z)^2 (+ 0.3 dilation).
    W, H, f = 48, 40, 60.0
    cam = oracle.camera_vec(f, f, 23.3, 19.6, W, H)
    rng = np.random.default_rng(1)
    q = rng.normal(size=4)
    s, z, logit, mp = 0.05, 2.0, 1.2, 0.7
    G = gauss_row((0, 0, z), s, q / np.linalg.norm(q) * 3.0, logit, mp)[None]
    r = oracle.render(G, cam, ident())
    var = (f * s / z) ** 2 + 0.3
    exp, ag = expected_single(W, H, cam[2], cam[3], var * np.eye(2), sigmoid(logit), G[0, 12:15], z, mp)
    keep = np.abs(ag - 1 / 255) > 1e-9
    np.testing.assert_allclose(r["pix"][keep, :7], exp[keep, :7], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, 90.0, -55.0])
def test_anisotropic_rotated_about_axis(theta_deg):
    # Rotation by theta about the optical axis rotates the 2D covariance by the
    # same angle in the image plane (x right, y down): Sigma' = (f/z)^2 R2
    # diag(sx^2, sy^2) R2^T + 0.3 I. Pins the quaternion convention and the
    # conic's off-diagonal sign.
    W, H, f = 64, 48, 80.0
    cam = oracle.camera_vec(f, f, 31.7, 24.2, W, H)
    th = np.deg2rad(theta_deg)
    quat = (np.cos(th / 2), 0, 0, np.sin(th / 2))
    sx, sy, sz, z = 0.12, 0.04, 0.02, 2.5
    G = gauss_row((0, 0, z), (sx, sy, sz), quat, 2.0, 0.3)[None]
    r = oracle.render(G, cam, ident())
    R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    cov = (f / z) ** 2 * R2 @ np.diag([sx ** 2, sy ** 2]) @ R2.T + 0.3 * np.eye(2)
    exp, ag = expected_single(W, H, cam[2], cam[3], cov, sigmoid(2.0), G[0, 12:15], z, 0.3)
    keep = (np.abs(ag - 1 / 255) > 1e-9) & (np.abs(ag - 0.99) > 1e-9)
    np.testing.assert_allclose(r["pix"][keep, :7], exp[keep, :7], rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("x0,y0", [(0.4, -0.3), (-0.7, 0.5), (2.9, 0.1)])
def test_off_axis_covariance_is_local_affine_projection(x0, y0):
    # EWA: the 2D covariance is J Sigma_c J^T + 0.3 I with J the Jacobian of the
    # pinhole projection at the mean. J here comes from central differences of
    # the projection, not from a formula; beyond the 1.3x frustum guard the
    # Jacobian is taken at the guard (x/z clamped).
    W, H, f, z = 64, 48, 50.0, 2.0
    cam = oracle.camera_vec(f, f, 32.0, 24.0, W, H)
    rng = np.random.default_rng(3)
    q = rng.normal(size=4)
    G = gauss_row((x0, y0, z), (0.05, 0.1, 0.03), q, 1.0)[None]
    pj = oracle.project(G, cam, ident())[0]
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rq @ np.diag([0.05, 0.1, 0.03]) ** 2 @ Rq.T
    limx, limy = 1.3 * W / (2 * f), 1.3 * H / (2 * f)
    xc = np.clip(x0 / z, -limx, limx) * z
    yc = np.clip(y0 / z, -limy, limy) * z

    def proj(p):
        return np.array([f * p[0] / p[2], f * p[1] / p[2]])

    h = 1e-6
    J = np.stack([(proj(np.array([xc, yc, z]) + h * e) - proj(np.array([xc, yc, z]) - h * e)) / (2 * h)
                  for e in np.eye(3)], 1)
    cov = J @ Sig @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose([pj[oracle.PJ["SA"]], pj[oracle.PJ["SB"]], pj[oracle.PJ["SC"]]],
                               [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)
    np.testing.assert_allclose([pj[oracle.PJ["U"]], pj[oracle.PJ["V"]]], proj([x0, y0, z]) + [32, 24], rtol=1e-13)
    Q = np.linalg.inv(cov)
    np.testing.assert_allclose([pj[oracle.PJ["A"]], pj[oracle.PJ["B"]], pj[oracle.PJ["C"]]],
                               [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-7)


def test_pose_moves_the_camera():
    # A Gaussian at world (x, y, z) seen from a camera translated by -x (pose
    # t = (-x, 0, 0)) lands on the image centre: p_c = R mu + t.
    W, H, f = 40, 30, 40.0
    cam = oracle.camera_vec(f, f, 20.0, 15.0, W, H)
    G = gauss_row((0.3, -0.2, 2.0), 0.05, (1, 0, 0, 0), 1.0)[None]
    pose = ident()
    pose[:, 3] = [-0.3, 0.2, 0.5]
    pj = oracle.project(G, cam, pose)[0]
    assert pj[oracle.PJ["U"]] == pytest.approx(20.0, abs=1e-12)
    assert pj[oracle.PJ["V"]] == pytest.approx(15.0, abs=1e-12)
    assert pj[oracle.PJ["Z"]] == pytest.approx(2.5, abs=1e-12)
    # a 90 degree yaw of the camera maps world +x onto camera -z ... (R mu)
    R = Rotation.from_euler("y", 90, degrees=True).as_matrix()
    pose2 = np.zeros((3, 4))
    pose2[:, :3] = R
    G2 = gauss_row((-2.0, 0.0, 0.0), 0.05, (1, 0, 0, 0), 1.0)[None]
    pj2 = oracle.project(G2, cam, pose2)[0]
    np.testing.assert_allclose(pj2[[oracle.PJ["PX"], oracle.PJ["PY"], oracle.PJ["Z"]]], R @ [-2.0, 0, 0],
                               atol=1e-12)


def test_two_layers_front_to_back():
    # C = c1 a1 + c2 a2 (1 - a1) with the nearer Gaussian first, whatever the ids.
    W, H, f = 32, 24, 40.0
    cam = oracle.camera_vec(f, f, 16.0, 12.0, W, H)
    near = gauss_row((0, 0, 1.5), 0.05, logit=0.5, mp=0.9, rgb=(1.0, 0.0, 0.5))
    far = gauss_row((0, 0, 3.0), 0.1, logit=1.5, mp=0.1, rgb=(0.0, 1.0, 0.25))
    for G in (np.stack([near, far]), np.stack([far, near])):
        r = oracle.render(G, cam, ident())
        px = r["pix"][12 * W + 16]
        a1 = sigmoid(0.5)           # centre pixel: exp(0) = 1
        a2 = sigmoid(1.5)
        np.testing.assert_allclose(px[0:3], np.array([1.0, 0.0, 0.5]) * a1 + np.array([0.0, 1.0, 0.25]) * a2 * (1 - a1),
                                   rtol=1e-13)
        np.testing.assert_allclose(px[3], 1.5 * a1 + 3.0 * a2 * (1 - a1), rtol=1e-13)
        np.testing.assert_allclose(px[4], a1 + a2 * (1 - a1), rtol=1e-13)
        np.testing.assert_allclose(px[5], 0.9 * a1 + 0.1 * a2 * (1 - a1), rtol=1e-13)
        np.testing.assert_allclose(px[6], (1 - a1) * (1 - a2), rtol=1e-13)
        assert px[7] == 2


def test_transmittance_stop_before_threshold():
    # Four stacked layers of alpha 0.98 at the centre pixel: after two, T = 4e-4;
    # a third would take T to 8e-6 < 1e-4, so it and everything behind it are
    # dropped.
    W, H, f = 16, 16, 20.0
    cam = oracle.camera_vec(f, f, 8.0, 8.0, W, H)
    lg = np.log(0.98 / 0.02)
    G = np.stack([gauss_row((0, 0, 1.0 + k), 0.05, logit=lg, rgb=(0.25 * k, 0.5, 0.5)) for k in range(4)])
    r = oracle.render(G, cam, ident())
    px = r["pix"][8 * W + 8]
    assert px[7] == 2
    np.testing.assert_allclose(px[6], 0.02 * 0.02, rtol=1e-12)
    np.testing.assert_allclose(px[0], 0.0 * 0.98 + 0.25 * 0.98 * 0.02, rtol=1e-12)
    assert px[8] == 1


def test_alpha_clamp_and_skip():
    # o * G above 0.99 is clamped to 0.99; below 1/255 the Gaussian is skipped.
    W, H, f = 16, 16, 20.0
    cam = oracle.camera_vec(f, f, 8.0, 8.0, W, H)
    G = gauss_row((0, 0, 2.0), 0.05, logit=8.0)[None]
    r = oracle.render(G, cam, ident())
    assert r["pix"][8 * W + 8, 4] == pytest.approx(0.99, abs=1e-15)
    G2 = gauss_row((0, 0, 2.0), 0.05, logit=np.log((0.5 / 255) / (1 - 0.5 / 255)))[None]
    r2 = oracle.render(G2, cam, ident())
    assert np.all(r2["pix"][:, 4] == 0) and np.all(r2["pix"][:, 6] == 1)
    assert oracle.project(G2, cam, ident())[0, oracle.PJ["VIS"]] == 0


def test_invariants_tiny_scene():
    sc = synth.tiny_scene(0)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    r = oracle.render(G, cam, sc.poses[0])
    pix = r["pix"]
    O, T = pix[:, 4], pix[:, 6]
    np.testing.assert_allclose(O, 1 - T, atol=1e-12)          # weights sum to 1 - T_final
    assert np.all(pix[:, 5] <= O + 1e-15)                      # rendered MP <= opacity
    cov = O > 0
    col = pix[cov, 0:3] / O[cov, None]
    assert np.all(col >= -1e-12) and np.all(col <= 1 + 1e-12)  # colours stay in [0, 1]
    zs = oracle.project(G, cam, sc.poses[0])[:, oracle.PJ["Z"]]
    dep = pix[cov, 3] / O[cov]
    assert np.all(dep >= 1.0 - 1e-9) and np.all(dep <= 4.0 + 1e-9)
    assert np.all(T >= 1e-4)                                   # never below t_min
    # the cell-accelerated traversal tests a superset of the contributors
    r0 = oracle.render(G, cam, sc.poses[0], accel=False)
    np.testing.assert_array_equal(r["pix"], r0["pix"])


def test_transmittance_monotone_in_depth_order():
    # Composite pixel by pixel by hand from the projection table: the running
    # transmittance never increases, and the oracle's final T matches.
    sc = synth.tiny_scene(5, n=300, width=48, height=40, f=40.0)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    pj = oracle.project(G, cam, sc.poses[0])
    r = oracle.render(G, cam, sc.poses[0])
    vis = np.nonzero(pj[:, 0] > 0)[0]
    order = vis[np.lexsort((vis, pj[vis, oracle.PJ["ZKEY"]]))]
    for pix in [0, 77, 500, 1000, 1919]:
        i, j = pix % 48, pix // 48
        T, Ts = 1.0, [1.0]
        for g in order:
            dx, dy = pj[g, 1] - i, pj[g, 2] - j
            ag = pj[g, 7] * np.exp(-0.5 * (pj[g, 4] * dx * dx + pj[g, 6] * dy * dy) - pj[g, 5] * dx * dy)
            if ag < 1 / 255:
                continue
            a = min(ag, 0.99)
            if T * (1 - a) < 1e-4:
                break
            T *= 1 - a
            Ts.append(T)
        assert np.all(np.diff(Ts) <= 0)
        assert T == pytest.approx(r["pix"][pix, 6], rel=1e-12)


def test_render_pixel_matches_full_render():
    sc = synth.tiny_scene(0)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    r = oracle.render(G, cam, sc.poses[0])
    for pix in [0, 1234, 8000, 19199]:
        v, _ = oracle.render_pixel(G, cam, sc.poses[0], pix % 160, pix // 160)
        np.testing.assert_allclose(v, r["pix"][pix], rtol=1e-14, atol=1e-15)


def _quad(p, dx, dy):
    return p[4] * dx * dx + 2 * p[5] * dx * dy + p[6] * dy * dy


def test_binned_tiles_are_the_tiles_the_alpha_ellipse_reaches():
    # Brute force over pixels and over a fine sub-pixel grid of every
    # candidate tile: a tile is binned iff the ellipse q(d) <= 2 ln(255 o),
    # outside of which alpha < 1/255, reaches its pixel-centre rectangle; every
    # contributing pixel's tile is binned; the candidate range is the tile range
    # of the ellipse's bounding box.
    sc = synth.tiny_scene(2, n=400)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    pj = oracle.project(G, cam, sc.poses[0])
    tiles, ids, _ = oracle.binning(G, cam, sc.poses[0])
    binned = {}
    for t, g in zip(tiles.tolist(), ids.tolist()):
        binned.setdefault(g, set()).add(t)
    ii, jj = pixel_grid(160, 120)
    fine = np.arange(0, 15.001, 0.125)
    fx, fy = np.meshgrid(fine, fine, indexing="xy")
    checked = 0
    for g in np.nonzero(pj[:, 0] > 0)[0]:
        p = pj[g]
        cth = p[oracle.PJ["CTHR"]]
        np.testing.assert_allclose(cth, 2 * np.log(255 * p[7]), rtol=1e-12)
        ex, ey = p[oracle.PJ["EX"]], p[oracle.PJ["EY"]]
        assert (p[13], p[15]) == (max(0, np.floor((p[1] - ex) / 16)), min(10, np.floor((p[1] + ex) / 16) + 1))
        assert (p[14], p[16]) == (max(0, np.floor((p[2] - ey) / 16)), min(8, np.floor((p[2] + ey) / 16) + 1))
        q = _quad(p, p[1] - ii, p[2] - jj)
        hit = q <= cth
        # alpha >= 1/255 exactly where q <= cthr
        ag = p[7] * np.exp(-0.5 * q)
        assert np.array_equal(hit, ag >= 1 / 255) or (np.abs(ag - 1 / 255) < 1e-12).any()
        pix_tiles = set(((jj[hit] // 16) * 10 + ii[hit] // 16).astype(int).tolist())
        got = binned.get(g, set())
        assert pix_tiles <= got
        for t in got:
            tx, ty = t % 10, t // 10
            assert p[13] <= tx < p[15] and p[14] <= ty < p[16]
            if t in pix_tiles:
                continue
            # a binned tile without a contributing pixel: the ellipse still
            # reaches its (continuous) rectangle
            xs = np.minimum(16 * tx + fx, 159) - p[1]
            ys = np.minimum(16 * ty + fy, 119) - p[2]
            assert _quad(p, xs, ys).min() <= cth * (1 + 1e-3)
        for ty in range(int(p[14]), int(p[16])):
            for tx in range(int(p[13]), int(p[15])):
                if ty * 10 + tx in got:
                    continue
                xs = np.minimum(16 * tx + fx, 159) - p[1]
                ys = np.minimum(16 * ty + fy, 119) - p[2]
                assert _quad(p, xs, ys).min() > cth * (1 - 1e-9)
                checked += 1
    assert checked > 50      # the exact test drops tiles the bounding box holds


def test_binning_order_and_content():
    sc = synth.tiny_scene(0)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    pj = oracle.project(G, cam, sc.poses[0])
    tiles, ids, _ = oracle.binning(G, cam, sc.poses[0])
    # every pair lies in its Gaussian's candidate range, no pair twice
    assert len(set(zip(tiles.tolist(), ids.tolist()))) == len(tiles)
    tx, ty = tiles % 10, tiles // 10
    assert np.all((tx >= pj[ids, 13]) & (tx < pj[ids, 15]) & (ty >= pj[ids, 14]) & (ty < pj[ids, 16]))
    # order: (tile, FP32 depth key, id)
    order = np.lexsort((ids, pj[ids, oracle.PJ["ZKEY"]], tiles))
    np.testing.assert_array_equal(order, np.arange(len(ids)))


# ---------------------------------------------------------- adjoint vs FD

def fd_scene(seed):
    rng = np.random.default_rng(seed)
    n = 10
    W, H, f = 28, 22, 30.0
    rows = []
    for k in range(n):
        mean = (rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(1.5, 3.0))
        scale = np.exp(rng.normal(-2.3, 0.3, 3))
        q = rng.normal(size=4)
        rows.append(gauss_row(mean, scale, q, rng.normal(0.5, 1.0), rng.uniform(0, 1), rng.uniform(0, 1, 3)))
    G = np.stack(rows)
    cam = oracle.camera_vec(f, f, 13.7, 10.9, W, H)
    tg = np.zeros((W * H, 4))
    tg[:, 0:3] = rng.uniform(0, 1, (W * H, 3))
    tg[:, 3] = rng.uniform(1, 3, W * H)
    tg[rng.random(W * H) < 0.2, 3] = 0.0        # some invalid depth
    pose = np.zeros((3, 4))
    pose[:, :3] = Rotation.from_rotvec(rng.normal(0, 0.05, 3)).as_matrix()
    pose[:, 3] = rng.normal(0, 0.05, 3)
    return G, cam, pose, tg


@pytest.mark.parametrize("seed,wmode,wgrad", [(11, 0, 0), (12, 0, 1), (13, 1, 1)])
def test_adjoint_matches_central_differences(seed, wmode, wgrad):
    G, cam, pose, tg = fd_scene(seed)
    lc = oracle.loss_vec(weight_mode=wmode, weight_grad=wgrad)
    r = oracle.render(G, cam, pose, lc=lc, targets=tg, grads=True)
    assert not np.any(r["flags"]), "scene has decisions within the FP margin"
    assert r["pix"][:, 7].max() >= 3           # several layers per pixel somewhere

    # with weight_grad = 0 the weight w(u) is a constant of the adjoint
    wfix = None if wgrad else r["pix"][:, oracle.PX["W"]].copy()

    def loss(Gx, posex):
        return oracle.render(Gx, cam, posex, lc=lc, targets=tg, wfix=wfix)["loss"]

    fd = np.zeros_like(G)
    for g in range(G.shape[0]):
        for c in list(range(0, 11)) + [12, 13, 14]:
            h = 1e-6 * max(1.0, abs(G[g, c]))
            Gp, Gm = G.copy(), G.copy()
            Gp[g, c] += h
            Gm[g, c] -= h
            fd[g, c] = (loss(Gp, pose) - loss(Gm, pose)) / (2 * h)
    an = r["grad"]
    scale = np.abs(an).max()
    np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-6 * scale)
    # pose: left perturbation exp(h e_k) T
    pfd = np.zeros(6)
    h = 1e-6
    for k in range(6):
        vals = []
        for s in (h, -h):
            P = pose.copy()
            if k < 3:
                P[k, 3] += s
            else:
                Rr = Rotation.from_rotvec(s * np.eye(3)[k - 3]).as_matrix()
                P = Rr @ pose
            vals.append(loss(G, P))
        pfd[k] = (vals[0] - vals[1]) / (2 * h)
    np.testing.assert_allclose(r["pose_grad"], pfd, rtol=1e-5, atol=1e-6 * np.abs(pfd).max())


def test_paper_constants_fixture():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        c = json.load(f)
    lc = oracle.loss_vec()
    assert lc[0] == c["lambda_1"]["value"] and lc[1] == c["lambda_2"]["value"]


def test_depth_key_is_fp32_camera_depth():
    # The key is the FP32 evaluation of r20 mx + r21 my + r22 mz + tz (no FMA),
    # written here with numpy float32 scalars; it equals the FP64 depth to
    # FP32 precision.
    sc = synth.tiny_scene(3, n=200)
    G = oracle.params_from_records(sc.records)
    pose = synth.look_at_pose([0.3, -0.2, -0.5], [0.1, 0.0, 2.0])
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    pj = oracle.project(G, cam, pose)
    f = np.float32
    r = pose.astype(np.float32)
    m = sc.records[:, 0:3]
    key = ((r[2, 0] * m[:, 0] + r[2, 1] * m[:, 1]) + r[2, 2] * m[:, 2]) + r[2, 3]
    assert key.dtype == np.float32
    np.testing.assert_array_equal(pj[:, oracle.PJ["ZKEY"]].astype(np.float32), key)
    vis = pj[:, 0] > 0
    np.testing.assert_allclose(pj[vis, oracle.PJ["ZKEY"]], pj[vis, oracle.PJ["Z"]], rtol=3e-7)
    del f


def test_upstream_adjoint_matches_central_differences():
    # A caller's own function of the rendered channels, F = sum_u up(u) .
    # (C_r, C_g, C_b, D, O, R_MP)(u) with a fixed random upstream: the
    # oracle's adjoint with that upstream against central differences of F.
    G, cam, pose, _ = fd_scene(14)
    W, H = int(cam[4]), int(cam[5])
    up = np.random.default_rng(3).normal(size=(W * H, 6))
    r = oracle.render(G, cam, pose, upstream=up, grads=True)
    assert not np.any(r["flags"] & oracle.PIXEL_DECISION_FLAGS)
    assert r["loss"] is None

    def F(Gx, posex):
        pix = oracle.render(Gx, cam, posex)["pix"]
        return float((pix[:, 0:6] * up).sum())

    fd = np.zeros_like(G)
    for g in range(G.shape[0]):
        for c in list(range(0, 11)) + [12, 13, 14]:
            h = 1e-6 * max(1.0, abs(G[g, c]))
            Gp, Gm = G.copy(), G.copy()
            Gp[g, c] += h
            Gm[g, c] -= h
            fd[g, c] = (F(Gp, pose) - F(Gm, pose)) / (2 * h)
    an = r["grad"]
    np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-6 * np.abs(an).max())
    pfd = np.zeros(6)
    h = 1e-6
    for k in range(6):
        vals = []
        for s in (h, -h):
            P = pose.copy()
            if k < 3:
                P[k, 3] += s
            else:
                P = Rotation.from_rotvec(s * np.eye(3)[k - 3]).as_matrix() @ pose
            vals.append(F(G, P))
        pfd[k] = (vals[0] - vals[1]) / (2 * h)
    np.testing.assert_allclose(r["pose_grad"], pfd, rtol=1e-5, atol=1e-6 * np.abs(pfd).max())


def test_upstream_of_the_l1_loss_reproduces_the_loss_adjoint():
    # The loss adjoint forms its upstream from Eqs. (20)-(22): lambda_1 w
    # sgn(r_C) per colour channel, lambda_2 w sgn(r_D) where D_gt > 0, and
    # nothing on O and R_MP while w is held constant. Passing that upstream
    # must give the same gradients by the other route.
    G, cam, pose, tg = fd_scene(11)
    r = oracle.render(G, cam, pose, targets=tg, grads=True)
    pix = r["pix"]
    w = pix[:, oracle.PX["W"]]
    lc = oracle.loss_vec()
    up = np.zeros((pix.shape[0], 6))
    up[:, 0:3] = lc[0] * w[:, None] * np.sign(pix[:, 0:3] - tg[:, 0:3])
    up[:, 3] = np.where(tg[:, 3] > 0, lc[1] * w * np.sign(pix[:, 3] - tg[:, 3]), 0.0)
    r2 = oracle.render(G, cam, pose, upstream=up, grads=True)
    np.testing.assert_allclose(r2["grad"], r["grad"], rtol=1e-12, atol=1e-14 * np.abs(r["grad"]).max())
    np.testing.assert_allclose(r2["pose_grad"], r["pose_grad"], rtol=1e-12, atol=1e-14)


def test_gradient_magnitude_bounds_the_gradient_and_is_exact_for_one_signed_sum():
    # grad_mag = sum over pixels and 2D words of |term| |d param / d word|:
    # (1) it bounds |grad| (triangle inequality); (2) for the colour, whose
    # chain is the identity, an all-positive upstream on the colour channels
    # makes every term positive, so grad_mag equals grad exactly; (3) it
    # scales with |upstream|.
    G, cam, pose, _ = fd_scene(15)
    W, H = int(cam[4]), int(cam[5])
    up = np.random.default_rng(7).normal(size=(W * H, 6))
    r = oracle.render(G, cam, pose, upstream=up, grads=True, grad_mag=True)
    assert np.all(r["grad_mag"] >= np.abs(r["grad"]) * (1 - 1e-12))
    r3 = oracle.render(G, cam, pose, upstream=-3.0 * up, grads=True, grad_mag=True)
    np.testing.assert_allclose(r3["grad_mag"], 3.0 * r["grad_mag"], rtol=1e-12, atol=0)
    pos = np.zeros((W * H, 6))
    pos[:, 0:3] = np.abs(up[:, 0:3]) + 0.1
    rp = oracle.render(G, cam, pose, upstream=pos, grads=True, grad_mag=True)
    cols = [12, 13, 14]                      # colour slots
    np.testing.assert_allclose(rp["grad_mag"][:, cols], rp["grad"][:, cols], rtol=1e-12, atol=0)
    assert np.all(rp["grad"][:, cols] >= 0)
