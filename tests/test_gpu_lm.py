"""GPU Levenberg-Marquardt pose refinement (C ABI) against the FP64 oracle
(oracle.render_jac, oracle/lm.py; Sec. V-A(c)):
- the per-pixel forward-mode pose Jacobian and the IRLS normal equations
  (L, H, g) on the tiny scene and on the full-size tracking frame;
- the FP64 LM decision and damped step against oracle.lm on given normal
  equations, including scripted accept/reject sequences;
- the tracking loop: convergence towards the ground-truth pose, graph replay
  identical to direct launches, determinism."""
import numpy as np
import pytest

import oracle
from oracle import lm as olm
from oracle import pose as opose
from paper_2602_21644_gb300 import synth

from gpu_common import mask_flagged_targets, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# FP32 forward-mode tangents against FP64: the Jacobian per channel
# normwise, and the normal equations (sums of W J J^T over the image)
JAC_NORM = 2e-4
H_REL = 1e-3
G_REL = 1e-3
L_REL = 1e-5


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    oracle.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def gpu_normal(dags, sc, delta=0.01, jac=True):
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    normal, J = ctx.normal_equations(gauss, cam, poses[0].contiguous(), targets[0].contiguous(), delta=delta, jac=jac)
    torch.cuda.synchronize()
    ctx.check()
    out = normal.cpu().numpy(), None if J is None else J.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


def compare_normal(sc, normal, J, delta=0.01, label=""):
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    ref = oracle.render_jac(G, cam, sc.poses[0], sc.targets[0], delta=delta)
    ok = (ref["flags"] & oracle.PIXEL_DECISION_FLAGS) == 0
    rep = []
    if J is not None:
        for ch in range(4):
            a, b = J[ok, ch, :], ref["J"][ok, ch, :]
            nrm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            rep.append(f"J ch{ch} {nrm:.2e}")
            assert nrm <= JAC_NORM, f"{label} Jacobian channel {ch}: normwise {nrm:.3e}"
    Hg, gg = oracle.unpack_normal(normal)
    eL = abs(normal[0] - ref["L"]) / abs(ref["L"])
    eH = np.linalg.norm(Hg - ref["H"]) / np.linalg.norm(ref["H"])
    eg = np.linalg.norm(gg - ref["g"]) / np.linalg.norm(ref["g"])
    rep.append(f"L {eL:.2e} H {eH:.2e} g {eg:.2e} flagged {int((~ok).sum())}")
    print(f"\n{label}: " + ", ".join(rep))
    assert eL <= L_REL and eH <= H_REL and eg <= G_REL, rep


def test_normal_equations_tiny(dags):
    sc, _ = mask_flagged_targets(synth.tiny_scene(0))
    normal, J = gpu_normal(dags, sc)
    compare_normal(sc, normal, J, label="tiny")


@pytest.mark.parametrize("delta", [1e-3, 0.05])
def test_normal_equations_ragged_and_delta(dags, delta):
    # 100x70: a ragged last tile row and column; other IRLS floors
    sc, _ = mask_flagged_targets(synth.tiny_scene(3, n=1500, width=100, height=70, f=80.0))
    normal, J = gpu_normal(dags, sc, delta=delta)
    compare_normal(sc, normal, J, delta=delta, label=f"ragged delta {delta}")


@pytest.mark.parametrize("wmode", [0, 1])
def test_normal_equations_weight_modes_and_invalid_targets(dags, wmode):
    # the unnormalised static weight (O - R_MP), 25% invalid depth, 10%
    # pixels without a valid colour (r < 0: out of both terms)
    sc = synth.tiny_scene(4, n=1800, width=120, height=88, f=100.0)
    rng = np.random.default_rng(4)
    tg = sc.targets.copy()
    tg[0, rng.random(tg.shape[1]) < 0.25, 3] = 0.0
    tg[0, rng.random(tg.shape[1]) < 0.10, 0] = -1.0
    sc = synth.Scene(sc.records, sc.camera, sc.poses, tg)
    lc = oracle.loss_vec(weight_mode=wmode)
    sc, _ = mask_flagged_targets(sc, lc=lc)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    normal, J = ctx.normal_equations(gauss, cam, poses[0].contiguous(), targets[0].contiguous(), jac=True,
                                     lcfg=dags.default_loss_cfg(weight_mode=wmode))
    torch.cuda.synchronize()
    ctx.check()
    ctx.close()
    G = oracle.params_from_records(sc.records)
    ref = oracle.render_jac(G, oracle.camera_vec(*sc.camera.as_tuple()), sc.poses[0], sc.targets[0], lc=lc)
    Hg, gg = oracle.unpack_normal(normal.cpu().numpy())
    assert abs(normal[0].item() - ref["L"]) <= L_REL * abs(ref["L"])
    assert np.linalg.norm(Hg - ref["H"]) <= H_REL * np.linalg.norm(ref["H"])
    assert np.linalg.norm(gg - ref["g"]) <= G_REL * np.linalg.norm(ref["g"])
    ok = (ref["flags"] & oracle.PIXEL_DECISION_FLAGS) == 0
    Jg = J.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Jg[ok] - ref["J"][ok]) <= JAC_NORM * np.linalg.norm(ref["J"][ok])


def test_normal_equations_full_size_tracking_frame(dags):
    sc, masked = mask_flagged_targets(synth.tracking_scene(300_000, frame=10))
    assert masked < 0.01 * sc.targets.shape[1]
    normal, _ = gpu_normal(dags, sc, jac=False)
    compare_normal(sc, normal, None, label="tracking frame")


def test_gradient_matches_the_adjoint(dags):
    # with a vanishing IRLS floor g is the loss gradient the reverse-mode
    # adjoint (splat_backward) returns
    sc, _ = mask_flagged_targets(synth.tiny_scene(2))
    normal, _ = gpu_normal(dags, sc, delta=1e-30, jac=False)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    image, last, _ = ctx.forward(gauss, cam, poses, targets)
    _, gp = ctx.backward(gauss, cam, poses, targets, image, last, dags.GRAD_POSE)
    torch.cuda.synchronize()
    gp = gp.cpu().numpy()[0]
    _, g = oracle.unpack_normal(normal)
    assert np.linalg.norm(g - gp) / np.linalg.norm(gp) <= 1e-3
    ctx.close()


def spd(rng, scale):
    A = rng.normal(size=(20, 6)) * scale
    return A.T @ A


def pack(L, H, g):
    out = [L]
    for k in range(6):
        for m in range(k, 6):
            out.append(H[k, m])
    return np.array(out + list(g))


def test_lm_step_matches_oracle(dags):
    rng = np.random.default_rng(0)
    pose0 = opose.apply_left(rng.normal(0, 0.1, 6), np.hstack([np.eye(3), np.zeros((3, 1))]))
    ctx = dags.Context(16, 16, 16, 1)
    cfg = dags.default_lm_cfg()
    ocfg = olm.LMConfig()
    state = torch.empty(dags.LM_STATE, dtype=torch.float64, device="cuda")
    ptry = torch.empty(12, dtype=torch.float64, device="cuda")
    pbest = torch.empty(12, dtype=torch.float64, device="cuda")
    pose_d = torch.from_numpy(pose0.ravel().copy()).cuda()
    ctx.lm_init(pose_d, state, ptry, cfg)
    # scripted losses: accept, reject, accept, equal (reject), NaN (reject)
    losses = [5.0, 7.0, 4.0, 4.0, float("nan")]
    Hs = [spd(rng, s) for s in (1.0, 2.0, 0.5, 1.5, 1.0)]
    gs = [rng.normal(0, 0.1, 6) for _ in losses]
    it = iter(range(len(losses)))
    tries = []

    def normal_fn(T):
        k = next(it)
        tries.append(T.copy())
        return losses[k], Hs[k], gs[k]

    T_ref, hist = olm.track(normal_fn, pose0, len(losses), ocfg)
    for k in range(len(losses)):
        nrm = torch.from_numpy(pack(losses[k], Hs[k], gs[k])).cuda()
        # the oracle linearised at tries[k]; the GPU's pose_try must be the same point
        np.testing.assert_allclose(ptry.cpu().numpy().reshape(3, 4), tries[k], rtol=0, atol=1e-13)
        ctx.lm_step(nrm, state, ptry, pbest, cfg)
        st = state.cpu().numpy()
        assert bool(st[44]) == hist[k]["accepted"]
        assert st[13] == hist[k]["mu"]
    torch.cuda.synchronize()
    np.testing.assert_allclose(pbest.cpu().numpy().reshape(3, 4), T_ref, rtol=0, atol=1e-13)
    st = state.cpu().numpy()
    assert st[41] == 2 and st[42] == 5
    ctx.close()


def test_lm_step_without_observations_keeps_the_pose(dags):
    ctx = dags.Context(16, 16, 16, 1)
    pose = torch.from_numpy(np.hstack([np.eye(3), np.ones((3, 1))]).ravel().copy()).cuda()
    state = torch.empty(dags.LM_STATE, dtype=torch.float64, device="cuda")
    ptry = torch.empty(12, dtype=torch.float64, device="cuda")
    pbest = torch.empty(12, dtype=torch.float64, device="cuda")
    ctx.lm_init(pose, state, ptry)
    ctx.lm_step(torch.zeros(dags.LM_NORMAL, dtype=torch.float64, device="cuda"), state, ptry, pbest)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ptry.cpu().numpy(), pose.cpu().numpy())
    np.testing.assert_array_equal(pbest.cpu().numpy(), pose.cpu().numpy())
    ctx.close()


def pose_error(T, T_gt):
    """(camera-centre distance in m, rotation angle in rad) of world-to-camera poses."""
    T = np.asarray(T).reshape(3, 4)
    T_gt = np.asarray(T_gt).reshape(3, 4)
    c = -T[:, :3].T @ T[:, 3]
    c_gt = -T_gt[:, :3].T @ T_gt[:, 3]
    Rr = T[:, :3] @ T_gt[:, :3].T
    ang = np.arccos(np.clip((np.trace(Rr) - 1.0) / 2.0, -1.0, 1.0))
    return float(np.linalg.norm(c - c_gt)), float(ang)


def self_consistent_frame(n=300_000):
    """The tracking frame with targets the oracle renders from the map itself
    at the ground-truth pose (depth only where the rendered opacity exceeds
    0.5): the loss is then minimal at the ground truth. Against the ray-cast
    targets it is not: the sparse map under-covers the surfaces, and the
    unnormalised compositing moves the minimum by centimetres."""
    sc = synth.tracking_scene(n, frame=10)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    pix = oracle.render(G, cam, sc.extra["gt_pose"])["pix"]
    tg = np.zeros_like(sc.targets)
    tg[0, :, 0:4] = pix[:, 0:4]
    tg[0, pix[:, 4] <= 0.5, 3] = 0.0
    return synth.Scene(sc.records, sc.camera, sc.poses, tg.astype(np.float32), sc.dynamic, sc.extra)


def test_track_lm_converges_and_replays_identically(dags):
    sc = self_consistent_frame()
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    e0 = pose_error(sc.poses[0], sc.extra["gt_pose"])
    results = []
    for use_graph in (False, True, True):
        pose = poses[0].clone().contiguous()
        state = ctx.track_lm(gauss, cam, pose, targets[0].contiguous(), 15, use_graph=use_graph)
        torch.cuda.synchronize()
        ctx.check()
        results.append((pose.cpu().numpy(), state.cpu().numpy()))
    p, st = results[0]
    e1 = pose_error(p, sc.extra["gt_pose"])
    # the first-order tracker on the same frame, for the record
    pa = poses.clone()
    adam = torch.zeros((1, 13), dtype=torch.float64, device="cuda")
    P = cam.width * cam.height
    image = torch.empty((1, 8, cam.height, cam.width), dtype=torch.float32, device="cuda")
    last = torch.empty((1, P), dtype=torch.int32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    gp = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    ctx.track(gauss, cam, pa, targets, 100, adam, image, last, loss, gp)
    torch.cuda.synchronize()
    ea = pose_error(pa[0].cpu().numpy(), sc.extra["gt_pose"])
    print(f"\nstart {e0[0] * 1e3:.3f} mm {np.degrees(e0[1]):.4f} deg; LM 15 it {e1[0] * 1e3:.3f} mm "
          f"{np.degrees(e1[1]):.4f} deg (accepted {int(st[41])}); Adam 100 it {ea[0] * 1e3:.3f} mm "
          f"{np.degrees(ea[1]):.4f} deg")
    assert st[42] == 15 and st[41] >= 3
    assert e1[0] < 0.05 * e0[0] and e1[1] < 0.05 * e0[1]
    for q, st2 in results[1:]:
        np.testing.assert_array_equal(q, p)
        np.testing.assert_array_equal(st2, st)
    ctx.close()


def test_capacity_overflow_rejects_the_point(dags):
    # a pair-capacity overflow renders nothing: the loss is NaN, the LM step
    # rejects the point (the pose stays) and the status reports the capacity
    sc = synth.tiny_scene(0)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1, max_pairs=2000)
    normal, _ = ctx.normal_equations(gauss, cam, poses[0].contiguous(), targets[0].contiguous())
    torch.cuda.synchronize()
    assert np.isnan(normal[0].item())
    assert ctx.sync_status()[0] == -3
    pose = poses[0].clone().contiguous()
    state = ctx.track_lm(gauss, cam, pose, targets[0].contiguous(), 3, use_graph=False)
    torch.cuda.synchronize()
    assert ctx.sync_status()[0] == -3
    st = state.cpu().numpy()
    assert st[41] == 0 and st[42] == 3                     # nothing accepted
    np.testing.assert_array_equal(pose.cpu().numpy(), sc.poses[0])
    ctx.close()


def test_empty_map_and_argument_errors(dags):
    sc = synth.tiny_scene(1)
    cam = dags.Camera(*sc.camera.as_tuple())
    _, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(100, cam.width, cam.height, 1)
    empty = torch.zeros((0, 16), dtype=torch.float32, device="cuda")
    normal, _ = ctx.normal_equations(empty, cam, poses[0].contiguous(), targets[0].contiguous())
    torch.cuda.synchronize()
    ctx.check()
    assert np.all(normal.cpu().numpy() == 0.0)
    pose = poses[0].clone().contiguous()
    ctx.track_lm(empty, cam, pose, targets[0].contiguous(), 2, use_graph=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pose.cpu().numpy(), sc.poses[0])    # tr H = 0: no step
    g = torch.from_numpy(sc.records[:100]).cuda()
    for kw in (dict(delta=0.0), dict(delta=float("inf"))):
        with pytest.raises(dags.DagsError):
            ctx.normal_equations(g, cam, poses[0].contiguous(), targets[0].contiguous(), **kw)
    for kw in (dict(down=0.0), dict(up=0.5), dict(mu_max=1e-12, mu_min=1.0), dict(delta=-1.0)):
        with pytest.raises(dags.DagsError):
            ctx.track_lm(g, cam, pose, targets[0].contiguous(), 1, cfg=dags.default_lm_cfg(**kw))
    ctx.close()
