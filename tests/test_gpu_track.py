"""GPU tracking loop (splat_track): graph replay, direct launches and the
oracle's own forward/backward/pose-step loop agree."""
import numpy as np
import pytest

import oracle
from oracle import pose as opose
from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def setup(dags, sc):
    cam = dags.Camera(*sc.camera.as_tuple())
    dev = "cuda"
    t = dict(gauss=torch.from_numpy(sc.records).to(dev),
             pose=torch.from_numpy(np.ascontiguousarray(sc.poses)).to(dev),
             targets=torch.from_numpy(np.ascontiguousarray(sc.targets)).to(dev),
             state=torch.zeros((1, 13), dtype=torch.float64, device=dev),
             image=torch.empty((1, 8, cam.height, cam.width), device=dev),
             last=torch.empty((1, cam.height, cam.width), dtype=torch.int32, device=dev),
             loss=torch.empty(1, dtype=torch.float64, device=dev),
             gp=torch.empty((1, 6), dtype=torch.float64, device=dev))
    return cam, t


def test_graph_and_direct_tracking_agree_with_oracle_loop(dags):
    sc = synth.tiny_scene(0)
    # start from a perturbed pose: the tracking loop pulls it back
    sc.poses[0] = opose.apply_left(np.array([0.02, -0.01, 0.015, 0.01, -0.02, 0.005]), sc.poses[0])
    lr = [2e-3, 2e-3, 2e-3, 1e-3, 1e-3, 1e-3]
    iters = 6
    cam, t = setup(dags, sc)
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    pcfg = dags.default_pose_cfg(lr=lr)
    results = {}
    for use_graph in (False, True, True):   # the second graph run replays the cached graph
        t["pose"].copy_(torch.from_numpy(np.ascontiguousarray(sc.poses)))
        t["state"].zero_()
        ctx.track(t["gauss"], cam, t["pose"], t["targets"], iters, t["state"], t["image"], t["last"], t["loss"],
                  t["gp"], pcfg=pcfg, use_graph=use_graph)
        torch.cuda.synchronize()
        ctx.check()
        results.setdefault(use_graph, []).append(t["pose"].cpu().numpy()[0].copy())
    # float atomics in the adjoint make repeated runs differ at rounding level;
    # after a step the runs sit at slightly different poses, where a pixel
    # decision near its threshold may flip, so runs agree to the oracle bound
    np.testing.assert_allclose(results[True][0], results[True][1], rtol=0, atol=1e-6)
    np.testing.assert_allclose(results[True][0], results[False][0], rtol=0, atol=1e-6)
    # the oracle's loop: FP64 render + adjoint + pose step, same number of iterations
    G = oracle.params_from_records(sc.records)
    ocam = oracle.camera_vec(*sc.camera.as_tuple())
    pose = sc.poses[0].copy()
    st = np.zeros(13)
    for _ in range(iters):
        r = oracle.render(G, ocam, pose, targets=sc.targets[0], grads=True)
        pose, st = opose.pose_step(pose, r["pose_grad"], st, lr)
    # each Adam step moves a component by ~lr; gradients agree to ~1e-6
    np.testing.assert_allclose(results[False][0], pose, rtol=0, atol=1e-6)


def test_tracking_converges_to_the_pose_that_rendered_the_target(dags):
    # Self-consistent target: the map rendered at a known pose, so the loss is
    # minimal there; tracking from a perturbed pose must move towards it.
    sc = synth.tracking_scene(60_000, frame=0, width=320, height=240)
    cam, t = setup(dags, sc)
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    gt = sc.extra["gt_pose"]
    t["pose"].copy_(torch.from_numpy(gt[None]))
    image, last, _ = ctx.forward(t["gauss"], cam, t["pose"])
    tg = torch.zeros_like(t["targets"])
    img = image[0].reshape(8, -1)
    tg[0, :, 0:3] = img[0:3].T
    tg[0, :, 3] = torch.where(img[4] > 0.5, img[3], torch.zeros_like(img[3]))
    start = opose.apply_left(np.array([0.01, -0.008, 0.006, 0.004, -0.006, 0.003]), gt)
    t["pose"].copy_(torch.from_numpy(start[None]))
    t["state"].zero_()
    pcfg = dags.default_pose_cfg(lr=[5e-4] * 3 + [2.5e-4] * 3)
    ctx.track(t["gauss"], cam, t["pose"], tg, 150, t["state"], t["image"], t["last"], t["loss"], t["gp"], pcfg=pcfg)
    torch.cuda.synchronize()
    ctx.check()

    def err(p):
        return np.linalg.norm(p[:, 3] - gt[:, 3]) + np.linalg.norm(p[:, :3] - gt[:, :3])

    e0, e1 = err(start), err(t["pose"].cpu().numpy()[0])
    assert e1 < 0.25 * e0, (e0, e1)


@pytest.mark.parametrize("size", ["tiny", "full"])
def test_tracking_iteration_equals_forward_and_backward(dags, size):
    # One tracking iteration with a zero learning rate (the pose stays put)
    # bins into the fixed-capacity buckets and runs the adjoint over the
    # entries the forward recorded per warp; splat_forward + splat_backward
    # bin into packed buckets and run the adjoint over the box-tested entries.
    # Image and last are bit-identical, the loss too (the same FP64 tile sums
    # in the same order); the pose gradient differs by the order of the FP32
    # atomics only.
    if size == "tiny":
        sc = synth.tiny_scene(2)
    else:
        sc = synth.tracking_scene(300_000, frame=10, width=640, height=480)
    cam, t = setup(dags, sc)
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    pcfg = dags.default_pose_cfg(lr=[0.0] * 6)
    ctx.track(t["gauss"], cam, t["pose"], t["targets"], 1, t["state"], t["image"], t["last"], t["loss"], t["gp"],
              pcfg=pcfg, use_graph=False)
    torch.cuda.synchronize()
    ctx.check()
    np.testing.assert_array_equal(t["pose"].cpu().numpy(), sc.poses)
    image, last, loss = ctx.forward(t["gauss"], cam, t["pose"], t["targets"])
    _, gp = ctx.backward(t["gauss"], cam, t["pose"], t["targets"], image, last, dags.GRAD_POSE)
    torch.cuda.synchronize()
    ctx.check()
    assert torch.equal(image, t["image"])
    assert torch.equal(last, t["last"])
    assert loss.item() == t["loss"].item()
    a, b = t["gp"].cpu().numpy(), gp.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), (a, b)
    ctx.close()


@pytest.mark.parametrize("lr", [4e-3, 5e-2])
def test_culled_iterations_render_what_an_unculled_forward_renders(dags, lr):
    # splat_track culls the map once at the frame's starting pose for every
    # pose within 0.01 rad and 0.01 m of it, and falls back to every Gaussian
    # beyond. Adam's first step moves each twist component by lr: 4e-3 keeps
    # the second iteration's pose inside the bounds (|rho|, |phi| ~ 7e-3),
    # 5e-2 takes it outside. Either way the second iteration's forward must
    # render what splat_forward (no culling) renders at that pose; a
    # Gaussian the culling missed would change whole pixels.
    sc = synth.tracking_scene(60_000, frame=12, width=320, height=240)
    cam, t = setup(dags, sc)
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    pcfg = dags.default_pose_cfg(lr=[lr] * 6)
    start = t["pose"].clone()
    ctx.track(t["gauss"], cam, t["pose"], t["targets"], 1, t["state"], t["image"], t["last"], t["loss"], t["gp"],
              pcfg=pcfg, use_graph=False)
    torch.cuda.synchronize()
    ctx.check()
    pose1 = t["pose"].clone()
    rel = pose1.cpu().numpy()[0][:, :3] @ start.cpu().numpy()[0][:, :3].T
    angle = np.arccos(np.clip((np.trace(rel) - 1) / 2, -1, 1))
    assert (angle < 0.01) == (lr < 0.01), angle
    image_ref, last_ref, loss_ref = ctx.forward(t["gauss"], cam, pose1, t["targets"])
    torch.cuda.synchronize()
    t["pose"].copy_(start)
    t["state"].zero_()
    ctx.track(t["gauss"], cam, t["pose"], t["targets"], 2, t["state"], t["image"], t["last"], t["loss"], t["gp"],
              pcfg=pcfg, use_graph=False)
    torch.cuda.synchronize()
    ctx.check()
    # the two runs' first steps agree to the rounding of the FP32 atomics in
    # the pose gradient (Adam's first step is lr g / (|g| + eps)), far below
    # a pixel's worth of motion
    np.testing.assert_allclose(t["image"].cpu().numpy(), image_ref.cpu().numpy(), rtol=1e-5, atol=1e-6)
    assert (t["last"] != last_ref).float().mean().item() < 1e-4
    ctx.close()


def test_recull_iterations_render_what_an_unculled_forward_renders(dags):
    # Adam's steps move each twist component by about lr = 5e-3: one step
    # stays within the culling bounds (0.01 rad, 0.01 m), two leave them, so
    # the third iteration re-culls at its pose and the fourth renders from
    # the re-culled candidates. Its image must be what splat_forward (no
    # culling) renders at that pose.
    sc = synth.tracking_scene(60_000, frame=12, width=320, height=240)
    cam, t = setup(dags, sc)
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    pcfg = dags.default_pose_cfg(lr=[5e-3] * 6)
    start = t["pose"].clone()

    def rel(a, b):
        a, b = a.cpu().numpy()[0], b.cpu().numpy()[0]
        R = a[:, :3] @ b[:, :3].T
        return np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)), np.linalg.norm(a[:, 3] - R @ b[:, 3])

    poses = []
    for iters in (1, 2, 3):
        t["pose"].copy_(start)
        t["state"].zero_()
        ctx.track(t["gauss"], cam, t["pose"], t["targets"], iters, t["state"], t["image"], t["last"], t["loss"],
                  t["gp"], pcfg=pcfg, use_graph=False)
        torch.cuda.synchronize()
        poses.append(t["pose"].clone())
    a1, d1 = rel(poses[0], start)
    a2, d2 = rel(poses[1], start)
    assert a1 < 0.01 and d1 < 0.01, (a1, d1)          # the second iteration uses the frame's list
    assert a2 > 0.01 or d2 > 0.01, (a2, d2)           # the third re-culls at its pose
    a3, d3 = rel(poses[2], poses[1])
    assert a3 < 0.01 and d3 < 0.01, (a3, d3)          # the fourth uses the re-culled list
    image_ref, last_ref, _ = ctx.forward(t["gauss"], cam, poses[2], t["targets"])
    torch.cuda.synchronize()
    t["pose"].copy_(start)
    t["state"].zero_()
    ctx.track(t["gauss"], cam, t["pose"], t["targets"], 4, t["state"], t["image"], t["last"], t["loss"], t["gp"],
              pcfg=pcfg, use_graph=False)
    torch.cuda.synchronize()
    ctx.check()
    np.testing.assert_allclose(t["image"].cpu().numpy(), image_ref.cpu().numpy(), rtol=1e-5, atol=1e-6)
    assert (t["last"] != last_ref).float().mean().item() < 1e-4
    ctx.close()
