"""GPU MP update (mp_update, C ABI) against the FP64 oracle (oracle/mp.py).

Inputs are synthetic and identical on both sides: observed RGB-D = the
ray-cast frame with moved objects; 'rendered' RGB-D = the ray-cast of the
map's static geometry at the same pose (the analytic stand-in for a render,
so that no oracle input comes from the CUDA path); instance labels with 5%
flips."""
import dataclasses

import numpy as np
import pytest

from oracle import mp as omp
from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

M_ABS = 1e-5           # per-Gaussian M^t and the medians (FP32 vs FP64)


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def mp_scene(n, frame, width, height, seed=0):
    sc = synth.tracking_scene(n, frame=frame, width=width, height=height, seed=seed)
    pose = sc.extra["gt_pose"]
    static, _ = synth.raycast(sc.camera, pose, sc.extra["objects"], 0.0)     # map geometry (frame 0)
    obs = sc.targets[0].copy()
    rng = np.random.default_rng(seed + 3)
    mp0 = rng.uniform(0.05, 0.95, n).astype(np.float32)
    rec = sc.records.copy()
    rec[:, 11] = mp0
    labels0 = (rng.random(n) < 0.3).astype(np.uint8)
    table = np.array([[0.1, 0.05]] + [[0.9, 0.8]] * sc.extra["n_instances"], np.float32)
    return dict(rec=rec, cam=sc.camera, pose=pose, obs=obs, rend=static, inst=sc.extra["instance"], table=table,
                labels0=labels0)


def run_both(dags, d, cfg_kw=None, seg_refreshed=True, mp_map=None):
    cfg_kw = cfg_kw or {}
    cam = dags.Camera(*d["cam"].as_tuple())
    P = cam.width * cam.height
    dev = "cuda"
    gauss = torch.from_numpy(d["rec"].copy()).to(dev)
    image = torch.zeros((8, P), dtype=torch.float32)
    image[0:3] = torch.from_numpy(d["rend"][:, 0:3].T.copy())
    image[3] = torch.from_numpy(d["rend"][:, 3].copy())
    image = image.to(dev)
    tg = torch.from_numpy(d["obs"].copy()).to(dev)
    inst = torch.from_numpy(d["inst"].copy()).to(dev)
    table = torch.from_numpy(d["table"].copy()).to(dev)
    labels = torch.from_numpy(d["labels0"].copy()).to(dev)
    pose = torch.from_numpy(np.ascontiguousarray(d["pose"])).to(dev)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    mp_pixel = torch.full((P,), -1.0, dtype=torch.float32, device=dev)
    gmap = None if mp_map is None else torch.from_numpy(np.asarray(mp_map, np.float32)).to(dev)
    stats = ctx.mp_update(gauss, cam, pose, tg, image, inst, table, labels, dags.default_mp_cfg(**cfg_kw),
                          seg_refreshed, mp_map=gmap, mp_pixel=mp_pixel)
    torch.cuda.synchronize()
    gpu = dict(mp=gauss[:, 11].cpu().numpy().astype(np.float64), labels=labels.cpu().numpy(),
               stats=stats.cpu().numpy(), mp_pixel=mp_pixel.cpu().numpy().astype(np.float64))
    cfg = dataclasses.replace(omp.MPConfig(), **cfg_kw)
    ref = omp.mp_update(d["rec"][:, 0:3], d["rec"][:, 11], d["labels0"], d["cam"].as_tuple(), d["pose"], d["inst"],
                        d["obs"][:, 3], d["obs"][:, 0:3], d["rend"][:, 3], d["rend"][:, 0:3], d["table"], cfg,
                        seg_refreshed, mp_map=None if mp_map is None else np.asarray(mp_map, np.float32))
    return gpu, ref


def check(gpu, ref, nreg):
    flag = ref["disk_flag"] | ref["vis_flag"]
    ok = ~flag
    assert ok.mean() > 0.99
    np.testing.assert_allclose(gpu["mp"][ok], ref["mp"][ok], rtol=0, atol=M_ABS)
    st = gpu["stats"]
    assert st[5] == ref["observed"].sum() or abs(st[5] - ref["observed"].sum()) <= flag.sum()
    assert abs(st[0] - ref["tau"]) <= M_ABS
    assert abs(st[1] - ref["U_bar"]) <= M_ABS
    lab_ok = ok & ~ref["label_flag"] & (np.abs(gpu["mp"] - st[0]) > M_ABS)
    np.testing.assert_array_equal(gpu["labels"][lab_ok], ref["labels"][lab_ok])
    px = ref["pixel"]
    for k in range(nreg):
        r = st[6 + 4 * k: 10 + 4 * k]
        assert r[0] == px["count"][k]
        np.testing.assert_allclose(r[1:4], [px["mean"][k], px["std"][k], px["e_ub"][k]], rtol=1e-5, atol=1e-7)
    assert np.all((gpu["mp"] >= 0) & (gpu["mp"] <= 1))
    assert st[0] >= 0.5
    # the fused per-pixel M_p map (FP32 vs FP64)
    np.testing.assert_allclose(gpu["mp_pixel"], ref["pixel"]["M_p"], rtol=0, atol=M_ABS)


@pytest.mark.parametrize("frame", [40, 59])
def test_mp_update_matches_oracle(dags, frame):
    d = mp_scene(60_000, frame, 320, 240)
    gpu, ref = run_both(dags, d)
    check(gpu, ref, d["table"].shape[0])


@pytest.mark.parametrize("kw,refreshed", [({"fusion_mode": 1}, True), ({"fusion_mode": 2}, True),
                                          ({"alpha_min": 0.3, "alpha_max": 0.3}, False), ({}, False),
                                          ({"vis_tol": 0.0}, True)])
def test_mp_update_variants(dags, kw, refreshed):
    d = mp_scene(40_000, 12, 256, 192, seed=1)
    gpu, ref = run_both(dags, d, kw, refreshed)
    check(gpu, ref, d["table"].shape[0])


def test_mp_update_full_size(dags):
    d = mp_scene(300_000, 20, 640, 480, seed=2)
    gpu, ref = run_both(dags, d)
    check(gpu, ref, d["table"].shape[0])
    # the observed Gaussians of the moving objects end with a higher MP than
    # the room's (their map position no longer matches the frame)
    dyn = synth.tracking_scene(300_000, frame=20, width=640, height=480, seed=2).dynamic
    obs = ref["observed"]
    assert (dyn & obs).sum() > 100 and (~dyn & obs).sum() > 100
    assert gpu["mp"][dyn & obs].mean() > gpu["mp"][~dyn & obs].mean() + 0.05


def test_mp_update_nothing_observed(dags):
    d = mp_scene(2_000, 5, 160, 120)
    d["pose"] = d["pose"].copy()
    d["pose"][:, 3] += np.array([0.0, 0.0, -100.0])    # everything behind the camera
    gpu, ref = run_both(dags, d)
    assert not ref["observed"].any()
    np.testing.assert_array_equal(gpu["mp"], d["rec"][:, 11].astype(np.float64))
    np.testing.assert_array_equal(gpu["labels"], d["labels0"])
    assert gpu["stats"][0] == 0.5 and gpu["stats"][5] == 0


def test_mp_update_external_map(dags):
    # a smooth external per-pixel MP map (the learned proposal's role) in
    # place of the fused M_p
    d = mp_scene(60_000, 33, 320, 240, seed=4)
    cam = d["cam"]
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    mp_map = (0.5 + 0.45 * np.sin(ii / 17.0) * np.cos(jj / 23.0)).astype(np.float32).ravel()
    gpu, ref = run_both(dags, d, mp_map=mp_map)
    check(gpu, ref, d["table"].shape[0])
    plain, _ = run_both(dags, d)
    assert np.abs(gpu["mp"] - plain["mp"]).max() > 0.01       # the map is used


def test_mpnet_features_match_oracle(dags):
    from oracle import mpnet as N
    rng = np.random.default_rng(5)
    W, H = 333, 77
    P = W * H
    image = rng.uniform(0, 1, (8, P)).astype(np.float32)
    image[3] = rng.uniform(0.5, 5, P)
    tg = rng.uniform(0, 1, (P, 4)).astype(np.float32)
    tg[:, 3] = rng.uniform(0.5, 5, P)
    tg[rng.random(P) < 0.2, 3] = 0.0
    nreg = 7
    inst = rng.integers(0, nreg, P).astype(np.uint8)
    table = rng.uniform(0, 1, (nreg, 2)).astype(np.float32)
    ctx = dags.Context(16, W, H, 1)
    cam = dags.Camera(300.0, 300.0, W / 2, H / 2, W, H)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f = ctx.mpnet_features(t(image), t(tg), t(inst), t(table), cam)
    torch.cuda.synchronize()
    ctx.check()
    ref = N.features(image[5], image[0:3].T, image[3], image[4], tg[:, 0:3], tg[:, 3], inst, table)
    np.testing.assert_array_equal(f.float().cpu().numpy().reshape(P, 8), ref)


@pytest.mark.parametrize("scales,size,frame", [(2, (320, 240), 40), (3, (320, 240), 40), (3, (251, 187), 25)])
def test_mp_update_multiscale(dags, scales, size, frame):
    # Eq. (1)'s union over pyramid levels: the pyramid is built from the
    # frame's M_p, e and rendered depth on the device; odd sizes drop the last
    # row and column of a level
    d = mp_scene(60_000, frame, *size, seed=5)
    gpu, ref = run_both(dags, d, {"scales": scales})
    check(gpu, ref, d["table"].shape[0])
    plain, _ = run_both(dags, d)
    assert np.abs(gpu["mp"] - plain["mp"]).max() > 1e-3        # the coarser levels are used


def test_mp_update_multiscale_external_map_full_size(dags):
    d = mp_scene(300_000, 20, 640, 480, seed=6)
    cam = d["cam"]
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    mp_map = (0.5 + 0.45 * np.sin(ii / 17.0) * np.cos(jj / 23.0)).astype(np.float32).ravel()
    gpu, ref = run_both(dags, d, {"scales": 3}, mp_map=mp_map)
    check(gpu, ref, d["table"].shape[0])


@pytest.mark.parametrize("scales", [0, 4])
def test_mp_update_rejects_bad_scales(dags, scales):
    d = mp_scene(2_000, 5, 160, 120)
    with pytest.raises(dags.DagsError) as e:
        run_both(dags, d, {"scales": scales})
    assert e.value.code == -1                                   # DAGS_E_INVAL


@pytest.mark.parametrize("w,h", [(7, 5), (5, 3), (3, 2)])
def test_mp_update_multiscale_tiny_images(dags, w, h):
    # images whose coarser levels have one pixel or none (5 x 3 -> 2 x 1 ->
    # 1 x 0; 3 x 2 -> 1 x 1 -> 0 x 0): Gaussians projected in and around them
    rng = np.random.default_rng(w * 10 + h)
    n = 400
    cam = synth.Camera(4.0, 4.0, w / 2.0, h / 2.0, w, h)
    z = rng.uniform(1.0, 3.0, n)
    u = rng.uniform(-4.0, w + 3.0, n)
    v = rng.uniform(-4.0, h + 3.0, n)
    rec = np.zeros((n, 16), np.float32)
    rec[:, 0] = (u - cam.cx) * z / cam.fx
    rec[:, 1] = (v - cam.cy) * z / cam.fy
    rec[:, 2] = z
    rec[:, 11] = rng.uniform(0.05, 0.95, n)
    P = w * h
    rend = np.concatenate([rng.uniform(0, 1, (P, 3)), rng.uniform(1.0, 3.5, (P, 1))], 1).astype(np.float32)
    obs = rend.copy()
    obs[:, 3] += rng.normal(0, 0.2, P).astype(np.float32)
    obs[:, 0:3] = rng.uniform(0, 1, (P, 3))
    d = dict(rec=rec, cam=cam, pose=synth.identity_pose(), obs=obs, rend=rend,
             inst=(rng.random(P) < 0.3).astype(np.uint8), table=np.array([[0.1, 0.05], [0.9, 0.8]], np.float32),
             labels0=(rng.random(n) < 0.3).astype(np.uint8))
    gpu, ref = run_both(dags, d, {"scales": 3, "vis_tol": 0.3})
    assert ref["observed"].sum() > 20
    check(gpu, ref, 2)
