"""The full loop at scale (1M Gaussians, 1200x680 RGB-D, three moving
ellipsoids, spline camera): full-image parity of one frame's forward and
adjoint against the FP64 oracle; the LM normal equations, lambda_3 L_MP and
the edge warp at the same scale; and the loop itself through the C ABI for a
dozen frames. Per frame: tracking (LM), the MP update, semantic refreshes
every 10 frames with the learned proposal in between, the trigger's score.
Every 5th frame: mapping over a window of up to 8 keyframes, the MP-weighted
loss and its Gaussian gradient with lambda_3 L_MP."""
import time

import numpy as np
import pytest

import oracle
from paper_2602_21644_gb300 import synth

from gpu_common import GRAD_NORM, LOSS_REL, POSE_REL, compare_grads, mask_flagged_targets, oracle_views
from test_gpu_splat import assert_image_parity, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    oracle.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


@pytest.fixture(scope="module")
def sequence():
    return synth.full_loop_sequence(frames=range(0, 12))


def test_full_scale_frame_parity(dags, sequence):
    rec, cam, seq, _ = sequence
    # frame 10's target from frame 9's pose (the tracking starting point)
    sc = synth.Scene(rec, cam, seq[9]["gt_pose"][None], seq[10]["target"][None].astype(np.float32))
    sc, masked = mask_flagged_targets(sc)
    assert masked < 0.01 * sc.targets.shape[1]
    res = run(dags, sc, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, ocam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "full loop 1200x680", report)
    assert abs(res["loss"] - outs[0]["loss"]) <= LOSS_REL * abs(outs[0]["loss"])
    pg = np.linalg.norm(res["gp"][0] - outs[0]["pose_grad"]) / np.linalg.norm(outs[0]["pose_grad"])
    g = compare_grads(res["gg"], outs[0]["grad"], report, mag=outs[0]["grad_mag"])
    report.append(f"pose grad rel {pg:.3e}")
    print("\n" + "\n".join(report))
    # the twist gradient is one sum over every pixel-Gaussian term, accumulated
    # in FP32 (atomics per Gaussian, then the per-Gaussian chain): rounding
    # grows like the square root of the terms, so the 300k x 640x480 bound
    # scales by sqrt(P N / (P0 N0))
    scale = np.sqrt((cam.width * cam.height * rec.shape[0]) / (640 * 480 * 300_000))
    assert pg <= POSE_REL * scale
    for k, v in g.items():
        assert v <= GRAD_NORM, f"gradient group {k}: {v:.3e}"
    res["ctx"].close()


def pose_error(T, T_gt):
    T = np.asarray(T).reshape(3, 4)
    T_gt = np.asarray(T_gt).reshape(3, 4)
    return float(np.linalg.norm(T[:, :3].T @ T[:, 3] - T_gt[:, :3].T @ T_gt[:, 3]))


def rendered_targets(dags, ctx, rec, cam, ex, frame_ids, poses, fps=30.0, seed=0, moving=True):
    """The loop's RGB-D frames rendered from the ground-truth map: the room's
    records with each moving object's Gaussians translated by its velocity
    times the frame's time (moving=False: left in place), seen from the
    frame's ground-truth pose; depth where the rendered opacity exceeds 0.5,
    with 1% multiplicative noise."""
    vel = np.zeros((rec.shape[0], 3), np.float32)
    for k, ob in enumerate(ex["objects"]):
        if moving:
            vel[ex["object_id"] == k] = ob.velocity
    vel_d = torch.from_numpy(vel).cuda()
    base = torch.from_numpy(rec).cuda()
    W, H = cam.width, cam.height
    gen = torch.Generator(device="cuda").manual_seed(seed)
    out = []
    for f, T in zip(frame_ids, poses):
        g = base.clone()
        g[:, 0:3] += vel_d * (f / fps)
        image, _, _ = ctx.forward(g, cam, torch.from_numpy(np.ascontiguousarray(T[None])).cuda())
        img = image[0].reshape(dags.IMG_CHANNELS, W * H)
        tg = torch.zeros((W * H, 4), dtype=torch.float32, device="cuda")
        tg[:, 0:3] = img[0:3].t()
        noise = 1.0 + 0.01 * torch.randn(W * H, generator=gen, device="cuda")
        tg[:, 3] = torch.where(img[4] > 0.5, img[3] * noise, torch.zeros_like(img[3]))
        out.append(tg)
    return out


def test_full_loop_runs_at_scale(dags, sequence):
    rec, scam, seq, ex = sequence
    cam = dags.Camera(*scam.as_tuple())
    n, P, W, H = rec.shape[0], cam.width * cam.height, cam.width, cam.height
    dev = "cuda"
    tctx = dags.Context(n, W, H, 1)
    mctx = dags.Context(n, W, H, 8)
    # the frames: renders of the ground-truth map (moving objects at their
    # frame's positions) from the ground-truth poses, so that the objective's
    # minimum for the static scene is the true pose
    targets = rendered_targets(dags, tctx, rec, cam, ex, [fr["frame"] for fr in seq], [fr["gt_pose"] for fr in seq])
    gauss = torch.from_numpy(rec.copy()).to(dev)
    gauss[:, 11] = 0.2                                   # uninformed initial MP
    prev = gauss.clone()                                 # the snapshot of Eq. (23)
    table = torch.tensor([[0.1, 0.05]] + [[0.9, 0.8]] * ex["n_instances"], dtype=torch.float32, device=dev)
    labels = torch.zeros(n, dtype=torch.uint8, device=dev)
    blob, _ = synth.mpnet_init(0)
    net = torch.from_numpy(blob).to(dev)
    state = torch.zeros(2, dtype=torch.int32, device=dev)
    score = torch.zeros(3, dtype=torch.float64, device=dev)
    image = torch.empty((1, dags.IMG_CHANNELS, H, W), dtype=torch.float32, device=dev)
    last = torch.empty((1, H, W), dtype=torch.int32, device=dev)
    pose = torch.from_numpy(seq[0]["gt_pose"].copy()).to(dev)
    prev_pose = None
    adam = mctx.gauss_adam_state(gauss)
    # fine-tuning rates: the map starts at the ground truth the frames render
    acfg = dags.default_gauss_adam_cfg(lr_mean=1e-4, lr_opacity=5e-3, lr_quat=1e-4, lr_scale=5e-4, lr_colour=2.5e-4)
    adam_step = 0
    keyframes, errors, times, accepted, map_losses = [], [], [], [], []
    refresh_inst = None
    for k, fr in enumerate(seq):
        t0 = time.perf_counter()
        tg = targets[k]
        if k > 0:
            # constant-velocity start: the last frame's motion applied again
            cur = pose.cpu().numpy()
            if prev_pose is not None:
                Rd = cur[:, :3] @ prev_pose[:, :3].T
                init = np.hstack([Rd @ cur[:, :3], (Rd @ cur[:, 3] + cur[:, 3] - Rd @ prev_pose[:, 3])[:, None]])
                pose.copy_(torch.from_numpy(init))
            prev_pose = cur
            st = tctx.track_lm(gauss, cam, pose, tg, 15)
            accepted.append(int(st[41].item()))
        tctx.forward(gauss, cam, pose[None], tg[None], image=image, last=last)
        refreshed = k % 10 == 0
        if refreshed:
            refresh_inst = torch.from_numpy(fr["instance"]).to(dev)
        mp_map = None
        if not refreshed:
            feats = tctx.mpnet_features(image[0].reshape(dags.IMG_CHANNELS, P), tg, refresh_inst, table, cam)
            mp_map = tctx.mpnet_infer(net, feats[None]).reshape(-1)
        stats = tctx.mp_update(gauss, cam, pose[None], tg, image[0].reshape(dags.IMG_CHANNELS, P), refresh_inst,
                               table, labels, seg_refreshed=refreshed, mp_map=mp_map)
        tctx.semantic_trigger(stats, state, refreshed, score=score)
        if k % 5 == 0:
            # mapping (Eq. (27)): the window's MP-weighted loss and lambda_3
            # L_MP, three Adam steps on the Gaussian parameters
            keyframes = (keyframes + [(pose.clone(), tg)])[-8:]
            poses = torch.stack([p for p, _ in keyframes])
            tgs = torch.stack([t for _, t in keyframes])
            window = []
            for _ in range(3):
                img, lst, loss = mctx.forward(gauss, cam, poses, tgs)
                gg, gp = mctx.backward(gauss, cam, poses, tgs, img, lst, dags.GRAD_GAUSS | dags.GRAD_POSE)
                lmp = mctx.mp_consistency(gauss, prev, 500.0, grad=gg)
                adam_step += 1
                mctx.gauss_adam_step(gauss, adam, gg, adam_step, acfg)
                torch.cuda.synchronize()
                assert np.isfinite(loss.item()) and np.isfinite(lmp.item())
                assert torch.isfinite(gg).all() and torch.isfinite(gp).all()
                window.append(loss.item() + lmp.item())
            map_losses.append(window)
            prev.copy_(gauss)
        torch.cuda.synchronize()
        tctx.check()
        mctx.check()
        times.append(time.perf_counter() - t0)
        if k == 10:
            mp10 = gauss[:, 11].cpu().numpy()           # right after the second refresh
        errors.append(pose_error(pose.cpu().numpy(), fr["gt_pose"]))
    mp = gauss[:, 11].cpu().numpy()
    moved = np.abs(gauss[:, 0:3].cpu().numpy() - rec[:, 0:3]).max()
    dyn = ex["dynamic"]
    seen = mp10 != np.float32(0.2)
    print(f"\npose errors (mm): {' '.join(f'{1e3 * e:.2f}' for e in errors)}; LM accepted: {accepted}")
    print(f"frame wall times (ms): {' '.join(f'{1e3 * t:.0f}' for t in times)}")
    print(f"mapping windows (loss + lambda_3 L_MP over 3 Adam steps): {map_losses}; largest mean shift {moved:.2e} m")
    print(f"mean MP after the frame-10 refresh: dynamic {mp10[dyn & seen].mean():.3f}, "
          f"static {mp10[~dyn & seen].mean():.3f}; last trigger score {score[2].item():.3f}")
    assert np.all((mp >= 0) & (mp <= 1))
    # the network is a seeded draw (untrained): the separation is the
    # refreshed priors' work
    assert mp10[dyn & seen].mean() > mp10[~dyn & seen].mean() + 0.05
    # the map moves under the mapping steps and stays near the map the frames
    # render (the loss falling over many mapping iterations is
    # test_gpu_gauss_adam's)
    assert 1e-5 < moved < 0.05
    assert all(np.all(np.isfinite(w)) for w in map_losses)
    # every frame's LM accepted steps and tracking keeps the true pose to
    # within one frame's motion (the camera moves about 19 mm per frame).
    # The moving objects bias the photometric optimum: the map keeps them
    # where the first frame saw them, the MP weights down-weight them only as
    # far as the refreshed priors have raised their M, and the fine-tuning
    # mapping does not carry them along; measured errors 2.6-13.7 mm, falling
    # after the frame-5 refresh. Without moving objects the loop converges to
    # the true pose (test_tracking_converges_on_a_static_scene)
    assert min(accepted) >= 2
    assert max(errors) < 0.019, errors
    tctx.close()
    mctx.close()


def test_tracking_converges_on_a_static_scene(dags, sequence):
    # The same frames with the objects left in place: the static scene's
    # photometric and depth optimum is the true pose, and LM tracking from
    # the constant-velocity start reaches it frame after frame to within the
    # 1% depth noise's effect (sub-millimetre), with no drift
    rec, scam, seq, ex = sequence
    cam = dags.Camera(*scam.as_tuple())
    n, W, H = rec.shape[0], cam.width, cam.height
    tctx = dags.Context(n, W, H, 1)
    frames = seq[:8]
    targets = rendered_targets(dags, tctx, rec, cam, ex, [fr["frame"] for fr in frames],
                               [fr["gt_pose"] for fr in frames], moving=False)
    gauss = torch.from_numpy(rec.copy()).cuda()
    gauss[:, 11] = 0.2
    pose = torch.from_numpy(frames[0]["gt_pose"].copy()).cuda()
    prev_pose, errors, start = None, [], []
    for k in range(1, len(frames)):
        cur = pose.cpu().numpy()
        if prev_pose is None:
            init = cur
        else:
            Rd = cur[:, :3] @ prev_pose[:, :3].T
            init = np.hstack([Rd @ cur[:, :3], (Rd @ cur[:, 3] + cur[:, 3] - Rd @ prev_pose[:, 3])[:, None]])
        start.append(pose_error(init, frames[k]["gt_pose"]))
        pose.copy_(torch.from_numpy(init))
        prev_pose = cur
        tctx.track_lm(gauss, cam, pose, targets[k], 15)
        torch.cuda.synchronize()
        tctx.check()
        errors.append(pose_error(pose.cpu().numpy(), frames[k]["gt_pose"]))
    print(f"\nstart errors (mm): {' '.join(f'{1e3 * e:.2f}' for e in start)}")
    print(f"tracked errors (mm): {' '.join(f'{1e3 * e:.3f}' for e in errors)}")
    assert max(errors) < 1e-3, errors
    assert errors[-1] < 0.05 * start[0], (start, errors)
    tctx.close()


def test_full_scale_normal_equations_and_regularisers(dags, sequence):
    # the next rows at the loop's scale: LM normal equations of frame 10 from
    # frame 9's pose, lambda_3 L_MP over 1M Gaussians, the edge warp 9 -> 10
    from oracle import edge as oedge
    from oracle import regular as oreg
    rec, scam, seq, _ = sequence
    sc = synth.Scene(rec, scam, seq[9]["gt_pose"][None], seq[10]["target"][None].astype(np.float32))
    sc, _ = mask_flagged_targets(sc)
    cam = dags.Camera(*scam.as_tuple())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = dags.Context(rec.shape[0], cam.width, cam.height, 1)
    normal, _ = ctx.normal_equations(t(rec), cam, t(sc.poses[0]), t(sc.targets[0]))
    rng = np.random.default_rng(5)
    prev = rec.copy()
    prev[:, 0:3] += rng.normal(0, 0.005, (rec.shape[0], 3)).astype(np.float32)
    grad = torch.zeros((rec.shape[0], 16), dtype=torch.float32, device="cuda")
    lmp = ctx.mp_consistency(t(rec), t(prev), 500.0, grad=grad)
    Di, Dj = seq[9]["target"][:, 3].copy(), seq[10]["target"][:, 3].copy()
    yy, xx = np.mgrid[0:cam.height, 0:cam.width]
    wj = (0.6 + 0.3 * np.cos(0.02 * xx) * np.sin(0.03 * yy)).astype(np.float32).ravel()
    eo = ctx.edge_warp(cam, t(Di), t(Dj), t(wj), t(seq[9]["gt_pose"].ravel()), t(seq[10]["gt_pose"].ravel()), 300.0)
    torch.cuda.synchronize()
    ctx.check()
    ctx.close()
    G = oracle.params_from_records(rec)
    ref = oracle.render_jac(G, oracle.camera_vec(*scam.as_tuple()), sc.poses[0], sc.targets[0])
    Hg, gg = oracle.unpack_normal(normal.cpu().numpy())
    eL = abs(normal[0].item() - ref["L"]) / abs(ref["L"])
    eH = np.linalg.norm(Hg - ref["H"]) / np.linalg.norm(ref["H"])
    eg = np.linalg.norm(gg - ref["g"]) / np.linalg.norm(ref["g"])
    L_ref, g_ref = oreg.mp_consistency(rec[:, 0:3], rec[:, 11], prev[:, 0:3], 500.0)
    e_ref = oedge.edge_warp(scam.as_tuple(), Di, Dj, wj, seq[9]["gt_pose"], seq[10]["gt_pose"])
    eo = eo.cpu().numpy()
    print(f"\nnormal equations: L {eL:.2e} H {eH:.2e} g {eg:.2e}; L_MP {abs(lmp.item() - L_ref) / L_ref:.2e}; "
          f"edge: {e_ref['n']} pixels, L {abs(eo[0] - e_ref['L']) / e_ref['L']:.2e}")
    # the normal equations' sums run over 4x the pixels and 3x the Gaussians
    # of the 300k frame: the bound on g scales as for the twist gradient
    scale = np.sqrt((cam.width * cam.height * rec.shape[0]) / (640 * 480 * 300_000))
    assert eL <= 1e-5 and eH <= 1e-3 * scale and eg <= 1e-3 * scale
    assert abs(lmp.item() - L_ref) <= 1e-5 * L_ref
    gm = grad.cpu().numpy()[:, 0:3].astype(np.float64)
    assert np.linalg.norm(gm - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    assert abs(eo[0] - e_ref["L"]) <= 2e-4 * e_ref["L"]
    assert np.linalg.norm(eo[1:7] - e_ref["grad_i"]) <= 2e-3 * np.linalg.norm(e_ref["grad_i"])
    assert np.linalg.norm(eo[7:13] - e_ref["grad_j"]) <= 2e-3 * np.linalg.norm(e_ref["grad_j"])
