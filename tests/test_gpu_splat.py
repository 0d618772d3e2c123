"""GPU parity of the splatting path (C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import pose as opose
from paper_2602_21644_gb300 import synth

from gpu_common import (GRAD_NORM, IMG_NORM, LOSS_REL, POSE_REL, T_NORM, compare_grads, compare_image,
                        image_rows, mask_flagged_targets, oracle_views, to_dev)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    import oracle as o
    o.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def run(dags, sc, flags=None, ctx=None, lcfg=None):
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    V = poses.shape[0]
    own = ctx is None
    if own:
        ctx = dags.Context(gauss.shape[0], cam.width, cam.height, V)
    image, last, loss = ctx.forward(gauss, cam, poses, targets, lcfg=lcfg)
    gg = gp = None
    if flags:
        gg, gp = ctx.backward(gauss, cam, poses, targets, image, last, flags, lcfg=lcfg)
    torch.cuda.synchronize()
    ctx.check()
    out = dict(image=image, last=last, loss=loss.item(), ctx=ctx, cam=cam,
               gg=None if gg is None else gg.cpu().numpy().astype(np.float64),
               gp=None if gp is None else gp.cpu().numpy())
    return out


def assert_image_parity(res, outs, label, report):
    for v, ref in enumerate(outs):
        worst, nflag = compare_image(image_rows(res["image"][v]), ref["pix"], ref["flags"], report, f"{label} v{v}")
        for c, (mx, nrm, bad) in worst.items():
            assert bad == 0, f"{label} view {v} channel {c}: {bad} pixels beyond tolerance (max {mx:.3e})"
            assert nrm <= (T_NORM if c == 6 else IMG_NORM), f"{label} view {v} channel {c}: normwise {nrm:.3e}"


def assert_bins_match(res, sc, dags, views_outs=None):
    """Tile lists bit-exact, except Gaussians whose rect sits within the FP
    margin of a tile boundary: those may differ by a boundary tile only."""
    cam = res["cam"]
    start, ids = res["ctx"].copy_bins(sc.poses.shape[0], cam)
    tx = (cam.width + 15) // 16
    T = tx * ((cam.height + 15) // 16)
    G = oracle.params_from_records(sc.records)
    ocam = oracle.camera_vec(*sc.camera.as_tuple())
    total_checked = 0
    for v in range(sc.poses.shape[0]):
        pj = oracle.project(G, ocam, sc.poses[v])
        flagged = (pj[:, oracle.PJ["FLAG"]].astype(np.int64) & (oracle.FLAGS["RECT"] | oracle.FLAGS["RADIUS"])) != 0
        tiles, oids, _ = oracle.binning(G, ocam, sc.poses[v])
        for t in range(T):
            g = ids[start[v * T + t]:start[v * T + t + 1]].astype(np.int64)
            o = oids[tiles == t]
            gk = g[~flagged[g]]
            ok = o[~flagged[o]]
            assert np.array_equal(gk, ok), f"view {v} tile {t}: order/content differs"
            total_checked += len(gk)
        # flagged Gaussians: GPU and oracle rects differ by at most one tile per side
    assert total_checked > 0


def test_forward_backward_tiny(dags):
    sc, _ = mask_flagged_targets(synth.tiny_scene(0))
    res = run(dags, sc, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, cam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "tiny", report)
    assert abs(res["loss"] - outs[0]["loss"]) <= LOSS_REL * abs(outs[0]["loss"])
    g = compare_grads(res["gg"], outs[0]["grad"], report, mag=outs[0]["grad_mag"])
    pg = np.linalg.norm(res["gp"][0] - outs[0]["pose_grad"]) / np.linalg.norm(outs[0]["pose_grad"])
    report.append(f"pose grad rel {pg:.3e}")
    print("\n".join(report))
    for k, v in g.items():
        assert v <= GRAD_NORM, f"gradient group {k}: {v:.3e}"
    assert pg <= POSE_REL
    assert_bins_match(res, sc, dags)


def test_binning_bit_exact_tiny(dags):
    sc = synth.tiny_scene(1)
    res = run(dags, sc)
    assert_bins_match(res, sc, dags)


@pytest.mark.parametrize("wmode,wgrad", [(0, 1), (1, 0), (1, 1)])
def test_loss_weight_modes(dags, wmode, wgrad):
    sc, _ = mask_flagged_targets(synth.tiny_scene(2, n=800, width=96, height=72, f=80.0),
                                 oracle.loss_vec(weight_mode=wmode, weight_grad=wgrad))
    lc = dags.default_loss_cfg(weight_mode=wmode, weight_grad=wgrad)
    res = run(dags, sc, flags=dags.GRAD_GAUSS | dags.GRAD_POSE, lcfg=lc)
    G, cam, outs = oracle_views(sc, lc=oracle.loss_vec(weight_mode=wmode, weight_grad=wgrad))
    report = []
    assert_image_parity(res, outs, "wmode", report)
    g = compare_grads(res["gg"], outs[0]["grad"], report, mag=outs[0]["grad_mag"])
    print("\n".join(report))
    for k, v in g.items():
        assert v <= GRAD_NORM, k
    pg = np.linalg.norm(res["gp"][0] - outs[0]["pose_grad"]) / np.linalg.norm(outs[0]["pose_grad"])
    assert pg <= POSE_REL


def test_ragged_image_and_pose(dags):
    # image size not a multiple of the tile, non-identity pose, partly outside
    sc = synth.tiny_scene(4, n=1500, width=150, height=101, f=110.0)
    sc.poses[0] = synth.look_at_pose([0.4, -0.3, -0.6], [0.1, 0.1, 2.5])
    sc, _ = mask_flagged_targets(sc)
    res = run(dags, sc, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, cam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "ragged", report)
    g = compare_grads(res["gg"], outs[0]["grad"], report, mag=outs[0]["grad_mag"])
    print("\n".join(report))
    for k, v in g.items():
        assert v <= GRAD_NORM, k
    assert_bins_match(res, sc, dags)


def test_multiview_equals_single_views(dags):
    sc = synth.tiny_scene(5, n=1200, width=112, height=96, f=100.0)
    poses = [synth.identity_pose(), synth.look_at_pose([0.2, 0.0, -0.3], [0.0, 0.0, 2.5]),
             synth.look_at_pose([-0.3, 0.2, 0.0], [0.1, -0.1, 2.0])]
    tg = np.repeat(sc.targets, 3, axis=0)
    scm, _ = mask_flagged_targets(synth.Scene(sc.records, sc.camera, np.stack(poses), tg))
    res = run(dags, scm, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, cam, outs = oracle_views(scm)
    report = []
    assert_image_parity(res, outs, "mv", report)
    gsum = sum(o["grad"] for o in outs)
    g = compare_grads(res["gg"], gsum, report, mag=sum(o["grad_mag"] for o in outs))
    for k, v in g.items():
        assert v <= GRAD_NORM, k
    for v in range(3):
        pg = np.linalg.norm(res["gp"][v] - outs[v]["pose_grad"]) / np.linalg.norm(outs[v]["pose_grad"])
        assert pg <= POSE_REL, (v, pg)
    assert abs(res["loss"] - sum(o["loss"] for o in outs)) <= LOSS_REL * sum(o["loss"] for o in outs)
    assert_bins_match(res, scm, dags)


def test_empty_and_culled(dags):
    sc = synth.tiny_scene(0, n=50)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(64, cam.width, cam.height, 1)
    # n = 0: background everywhere, zero loss
    image, last, loss = ctx.forward(gauss[:0], cam, poses, targets)
    gg, gp = ctx.backward(gauss[:0], cam, poses, targets, image, last, dags.GRAD_POSE | dags.GRAD_GAUSS)
    torch.cuda.synchronize()
    ctx.check()
    assert loss.item() == 0.0
    im = image[0].cpu().numpy()
    assert np.all(im[[0, 1, 2, 3, 4, 5, 7]] == 0) and np.all(im[6] == 1)
    assert np.all(gp.cpu().numpy() == 0)
    # every Gaussian behind the camera
    back = sc.records.copy()
    back[:, 2] = -back[:, 2]
    sc2 = synth.Scene(back, sc.camera, sc.poses, sc.targets)
    res = run(dags, sc2, flags=dags.GRAD_GAUSS | dags.GRAD_POSE, ctx=ctx)
    assert res["loss"] == 0.0 and np.all(res["gg"] == 0) and np.all(res["gp"] == 0)
    # NaN records are culled, not propagated
    bad = sc.records.copy()
    bad[::3, 0] = np.nan
    bad[1::3, 4:8] = 0.0
    res = run(dags, synth.Scene(bad, sc.camera, sc.poses, sc.targets), ctx=ctx)
    assert np.isfinite(res["image"].cpu().numpy()).all()


def test_oversized_tile_lists_use_the_merge_path(dags):
    # 20,000 small Gaussians over one 16x16 tile: its list exceeds both the
    # in-shared-memory sort (4096) and one merge chunk (16384).
    rng = np.random.default_rng(9)
    n = 20000
    means = np.stack([rng.uniform(-0.02, 0.02, n), rng.uniform(-0.02, 0.02, n), rng.uniform(1.0, 5.0, n)], 1)
    q = rng.normal(size=(n, 4))
    rec = synth.pack_records(means, rng.normal(-2, 0.5, n), q, np.full((n, 3), -4.5), rng.uniform(0, 1, n),
                             rng.uniform(0, 1, (n, 3)))
    camera = synth.Camera(40.0, 40.0, 16.0, 16.0, 32, 32)
    tg = np.zeros((1, 32 * 32, 4), np.float32)
    tg[0, :, :3] = rng.uniform(0, 1, (1024, 3))
    tg[0, :, 3] = rng.uniform(1, 5, 1024)
    sc = synth.Scene(rec, camera, synth.identity_pose()[None], tg)
    res = run(dags, sc, flags=dags.GRAD_POSE)
    start, ids = res["ctx"].copy_bins(1, res["cam"])
    assert np.diff(start).max() > 16384
    assert_bins_match(res, sc, dags)
    G, cam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "big", report)


def test_capacity_overflow_reports_required_pairs(dags):
    sc = synth.tiny_scene(0)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1, max_pairs=2000)
    ctx.forward(gauss, cam, poses, targets)
    code, req = ctx.sync_status()
    assert code == -3
    G = oracle.params_from_records(sc.records)
    tiles, _, _ = oracle.binning(G, oracle.camera_vec(*sc.camera.as_tuple()), sc.poses[0])
    assert abs(req - len(tiles)) <= 16  # equal up to FP-margin-flagged rect tiles
    # the status was cleared; a context big enough works
    ctx2 = dags.Context(gauss.shape[0], cam.width, cam.height, 1, max_pairs=req)
    ctx2.forward(gauss, cam, poses, targets)
    assert ctx2.sync_status()[0] == 0


def test_argument_errors(dags):
    sc = synth.tiny_scene(0, n=10)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss, poses, targets = to_dev(sc, torch)
    ctx = dags.Context(10, cam.width, cam.height, 1)
    image, last, loss = ctx.forward(gauss, cam, poses, targets)
    with pytest.raises(dags.DagsError) as e:
        ctx.backward(gauss, cam, poses, targets, image.clone(), last, dags.GRAD_POSE)
    assert e.value.code == -6
    big = dags.Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width + 1, cam.height)
    with pytest.raises(dags.DagsError) as e:
        ctx.forward(gauss, big, poses, targets)
    assert e.value.code == -1
    with pytest.raises(dags.DagsError):
        ctx.forward(torch.cat([gauss, gauss]), cam, poses, targets)


def test_pose_step_matches_oracle(dags):
    rng = np.random.default_rng(3)
    V = 3
    poses = np.stack([synth.look_at_pose(rng.normal(0, 0.3, 3), [0, 0, 2.0]) for _ in range(V)])
    state = np.zeros((V, 13))
    ctx = dags.Context(16, 16, 16, V)
    dp = torch.from_numpy(poses.copy()).cuda()
    ds = torch.zeros((V, 13), dtype=torch.float64, device="cuda")
    lr = [1e-3, 2e-3, 3e-3, 1e-2, 2e-2, 5e-2]
    cfg = dags.default_pose_cfg(lr=lr)
    for it in range(5):
        g = rng.normal(0, 100, (V, 6))
        ctx.pose_step(dp, torch.from_numpy(g).cuda(), ds, cfg)
        for v in range(V):
            poses[v], state[v] = opose.pose_step(poses[v], g[v], state[v], lr)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dp.cpu().numpy(), poses, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ds.cpu().numpy(), state, rtol=1e-14, atol=1e-12)


def test_full_size_tracking_frame(dags):
    # 300k Gaussians, 640x480: the whole image and the pose gradient against
    # the oracle (which takes about a second here).
    sc, masked = mask_flagged_targets(synth.tracking_scene(300_000, frame=10))
    assert masked < 0.01 * sc.targets.shape[1]
    res = run(dags, sc, flags=dags.GRAD_POSE)
    G, cam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "track", report)
    pg = np.linalg.norm(res["gp"][0] - outs[0]["pose_grad"]) / np.linalg.norm(outs[0]["pose_grad"])
    report.append(f"pose grad rel {pg:.3e}")
    print("\n".join(report))
    assert pg <= POSE_REL
    assert abs(res["loss"] - outs[0]["loss"]) <= LOSS_REL * abs(outs[0]["loss"])
    assert_bins_match(res, sc, dags)


def test_full_size_mapping_window(dags):
    # 200k Gaussians, 8 keyframes of 640x480, full parameter gradients.
    sc, masked = mask_flagged_targets(synth.mapping_scene(200_000, views=8))
    assert masked < 0.01 * sc.targets.shape[1] * 8
    res = run(dags, sc, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, cam, outs = oracle_views(sc)
    report = []
    assert_image_parity(res, outs, "map", report)
    g = compare_grads(res["gg"], sum(o["grad"] for o in outs), report, mag=sum(o["grad_mag"] for o in outs))
    print("\n".join(report))
    for k, v in g.items():
        assert v <= GRAD_NORM, k


def test_invalid_colour_pixels_leave_the_loss(dags):
    # r < 0 removes a pixel from the loss and the gradient on both sides
    sc = synth.tiny_scene(7, n=600, width=64, height=48, f=60.0)
    tg = sc.targets.copy()
    tg[0, ::3, 0] = -1.0
    sc2 = synth.Scene(sc.records, sc.camera, sc.poses, tg)
    sc2, _ = mask_flagged_targets(sc2)
    res = run(dags, sc2, flags=dags.GRAD_GAUSS | dags.GRAD_POSE)
    G, cam, outs = oracle_views(sc2)
    assert abs(res["loss"] - outs[0]["loss"]) <= LOSS_REL * abs(outs[0]["loss"])
    g = compare_grads(res["gg"], outs[0]["grad"], mag=outs[0]["grad_mag"])
    for k, v in g.items():
        assert v <= GRAD_NORM, k


def test_forward_is_deterministic(dags):
    # the forward has no order-dependent reduction: depth keys with id
    # tie-breaks, per-pixel compositing, fixed-order FP64 loss
    from paper_2602_21644_gb300 import synth
    sc = synth.tracking_scene(60_000, frame=7, width=320, height=240)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss = torch.from_numpy(sc.records).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    targets = torch.from_numpy(sc.targets).cuda()
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    i1, l1, s1 = [t.clone() for t in ctx.forward(gauss, cam, poses, targets)]
    i2, l2, s2 = ctx.forward(gauss, cam, poses, targets)
    torch.cuda.synchronize()
    ctx.check()
    assert torch.equal(i1, i2) and torch.equal(l1, l2) and torch.equal(s1, s2)
    ctx.close()
