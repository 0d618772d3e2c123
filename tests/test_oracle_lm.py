"""Pins of the Levenberg-Marquardt pose oracle (Sec. V-A(c)): the forward-mode
Jacobian against central finite differences of the render, the normal
equations' gradient against the independent reverse-mode adjoint, and the LM
iteration against closed forms (no GPU)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle import lm as olm
from oracle import pose as opose
from test_oracle_splat import fd_scene


def perturbed(pose, k, s):
    """exp(s e_k^) pose for twist component k (rho first)."""
    xi = np.zeros(6)
    xi[k] = s
    return opose.apply_left(xi, pose)


@pytest.mark.parametrize("seed", [11, 14])
def test_jacobian_matches_central_differences(seed):
    G, cam, pose, tg = fd_scene(seed)
    r = oracle.render_jac(G, cam, pose, tg)
    assert not np.any(r["flags"])
    ref = oracle.render(G, cam, pose)["pix"]
    np.testing.assert_allclose(r["pix"][:, :6], ref[:, :6], rtol=0, atol=1e-14)
    h = 1e-6
    chans = [0, 1, 2, 3]                        # r, g, b, depth
    for k in range(6):
        pp = oracle.render(G, cam, perturbed(pose, k, h))["pix"]
        pm = oracle.render(G, cam, perturbed(pose, k, -h))["pix"]
        same = (pp[:, 7] == ref[:, 7]) & (pm[:, 7] == ref[:, 7]) & (pp[:, 8] == ref[:, 8]) & (pm[:, 8] == ref[:, 8])
        assert same.mean() > 0.95
        fd = (pp[:, chans] - pm[:, chans]) / (2 * h)
        an = r["J"][:, :, k]
        scale = np.abs(an).max()
        assert scale > 0
        np.testing.assert_allclose(an[same], fd[same], rtol=1e-5, atol=1e-6 * scale)


@pytest.mark.parametrize("seed", [11, 13])
def test_gradient_equals_reverse_mode_adjoint(seed):
    # with a vanishing IRLS floor W r = c sgn(r), so g is the gradient of the
    # stop-gradient L1 loss, which the reverse-mode adjoint computes by a
    # different route
    G, cam, pose, tg = fd_scene(seed)
    lc = oracle.loss_vec(weight_mode=0, weight_grad=0)
    r = oracle.render_jac(G, cam, pose, tg, lc=lc, delta=1e-300)
    a = oracle.render(G, cam, pose, lc=lc, targets=tg, grads=True)
    assert not np.any(a["flags"] & oracle.FLAGS["SIGN"])
    np.testing.assert_allclose(r["g"], a["pose_grad"], rtol=1e-9, atol=1e-12 * np.abs(a["pose_grad"]).max())
    assert abs(r["L"] - a["loss"]) <= 1e-12 * abs(a["loss"])


def test_normal_matrix_psd_and_floor_scaling():
    G, cam, pose, tg = fd_scene(12)
    r1 = oracle.render_jac(G, cam, pose, tg, delta=1e3)
    r2 = oracle.render_jac(G, cam, pose, tg, delta=1e4)
    # every |r| is below both floors: W = c / delta, so delta H is the same
    np.testing.assert_allclose(1e3 * r1["H"], 1e4 * r2["H"], rtol=1e-12)
    np.testing.assert_allclose(1e3 * r1["g"], 1e4 * r2["g"], rtol=1e-12, atol=1e-15)
    r = oracle.render_jac(G, cam, pose, tg)
    assert np.allclose(r["H"], r["H"].T)
    assert np.linalg.eigvalsh(r["H"]).min() >= -1e-12 * np.abs(r["H"]).max()


def test_undamped_step_solves_linear_least_squares():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(40, 6))
    b = rng.normal(size=40)
    x0 = rng.normal(size=6)
    H = A.T @ A
    g = A.T @ (A @ x0 - b)
    d = olm.solve(H, g, 0.0, 0.0)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x0 + d, x_ls, rtol=1e-10, atol=1e-12)


def test_large_damping_is_scaled_steepest_descent():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(30, 6))
    H = A.T @ A
    g = rng.normal(size=6)
    mu = 1e8
    d = olm.solve(H, g, mu, 0.0)
    np.testing.assert_allclose(d, -g / (mu * np.diag(H)), rtol=1e-6)
    assert d @ g < 0


def test_nothing_observed_gives_no_step():
    assert np.all(olm.solve(np.zeros((6, 6)), np.ones(6), 1.0) == 0.0)


def test_translation_model_converges_in_one_step():
    # residual r = t - t_star on the translation only (a pure-translation
    # pose, rho steps with phi = 0 add rho to t): H = I on the rho block,
    # zero on phi; the ridge keeps the system definite
    t_star = np.array([0.3, -0.2, 0.5])

    def normal(T):
        r = T[:, 3] - t_star
        H = np.zeros((6, 6))
        H[:3, :3] = np.eye(3)
        g = np.zeros(6)
        g[:3] = r
        return float(r @ r), H, g

    cfg = olm.LMConfig(mu0=1e-6, mu_min=0.0, floor=1e-12)
    T0 = np.hstack([np.eye(3), np.zeros((3, 1))])
    T, hist = olm.track(normal, T0, 3, cfg)
    # the second linearisation point is one step from T0: at t_star up to the
    # damping mu * |r| and the ridge
    assert hist[0]["accepted"] and hist[1]["accepted"]
    assert hist[1]["L"] < 1e-12
    np.testing.assert_allclose(T[:, 3], t_star, rtol=0, atol=1e-6)
    np.testing.assert_allclose(T[:, :3], np.eye(3), atol=1e-15)


def test_reject_keeps_best_and_raises_damping():
    # scripted losses: 5, 7 (reject), 4 (accept), 4 (equal: reject)
    losses = iter([5.0, 7.0, 4.0, 4.0])
    H = np.eye(6)
    g = np.full(6, 1e-3)

    def normal(T):
        return next(losses), H, g

    cfg = olm.LMConfig(mu0=1.0)
    T0 = np.hstack([Rotation.from_rotvec([0.1, 0.0, 0.0]).as_matrix(), np.ones((3, 1))])
    T, hist = olm.track(normal, T0, 4, cfg)
    assert [h["accepted"] for h in hist] == [True, False, True, False]
    np.testing.assert_allclose([h["mu"] for h in hist], [0.1, 1.0, 0.1, 1.0])
    # the best pose is the third linearisation point: T0 stepped by the
    # second iteration's solve (damping 1 after the reject)
    T1 = opose.apply_left(olm.solve(H, g, 0.1), T0)
    T2 = opose.apply_left(olm.solve(H, g, 1.0), T0)
    np.testing.assert_allclose(hist[1]["delta"], olm.solve(H, g, 1.0))
    np.testing.assert_allclose(T, T2)
    assert not np.allclose(T1, T2)


def test_render_lm_reduces_the_loss():
    G, cam, pose, tg = fd_scene(11)
    # targets rendered at the pose; start from a perturbed pose
    ref = oracle.render(G, cam, pose)["pix"]
    tg2 = tg.copy()
    tg2[:, 0:4] = ref[:, 0:4]
    tg2[ref[:, 4] < 0.5, 3] = 0.0
    start = opose.apply_left(np.array([0.01, -0.01, 0.02, 0.01, -0.01, 0.005]), pose)

    def normal(T):
        r = oracle.render_jac(G, cam, T, tg2)
        return r["L"], r["H"], r["g"]

    T, hist = olm.track(normal, start, 8)
    Ls = [h["L"] for h in hist if h["accepted"]]
    assert all(b < a for a, b in zip(Ls, Ls[1:]))
    assert Ls[-1] < 0.3 * Ls[0]
