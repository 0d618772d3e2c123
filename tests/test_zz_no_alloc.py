"""The allocation-free forward (splat_forward_static) against splat_forward.

splat_forward_static exists for callers that must not allocate device memory
once they run, such as a real-time pipeline that forbids allocation after
start-up or a plugin whose host owns all device memory. It keeps its
workspace in one fixed device array inside the library. This file checks,
through the C ABI, that two calls in a row on different inputs each give
what splat_forward gives on the same inputs (so the array's leftovers from
the first call do not leak into the second), that its status output reports
the pair count, and that sizes beyond its stated limits are refused.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_21644_gb300 import synth

from gpu_common import IMG_ATOL, IMG_RTOL, LOSS_REL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def static_forward(dags, sc, status=True):
    lib = dags.load()
    cam = dags.Camera(*sc.camera.as_tuple())
    g = torch.from_numpy(np.ascontiguousarray(sc.records)).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(sc.poses[0])).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(sc.targets)).cuda()
    image = torch.full((1, 8, cam.height, cam.width), float("nan"), device="cuda")
    last = torch.full((1, cam.height, cam.width), -7, dtype=torch.int32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.full((2,), -99, dtype=torch.int64, device="cuda") if status else None
    c = cam.c()
    rc, lc = dags.default_raster_cfg(), dags.default_loss_cfg()
    code = lib.splat_forward_static(ptr(g), g.shape[0], ctypes.byref(c), ptr(pose), ptr(tg), ctypes.byref(rc),
                                    ctypes.byref(lc), ptr(image), ptr(last), ptr(loss), ptr(st),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, image, last, loss, st


def ctx_forward(dags, sc):
    cam = dags.Camera(*sc.camera.as_tuple())
    g = torch.from_numpy(np.ascontiguousarray(sc.records)).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(sc.targets)).cuda()
    ctx = dags.Context(g.shape[0], cam.width, cam.height, 1)
    image, last, loss = ctx.forward(g, cam, poses, tg)
    code, req = ctx.sync_status()
    assert code == 0
    return image, last, loss, req


def test_two_calls_in_a_row_match_splat_forward(dags):
    scenes = [synth.tiny_scene(0),
              synth.tiny_scene(3, n=3000, width=200, height=150, f=140.0)]
    scenes[1].poses[0] = synth.look_at_pose([0.2, -0.1, -0.3], [0.0, 0.1, 2.5])
    for sc in scenes:
        code, image, last, loss, st = static_forward(dags, sc)
        assert code == 0
        ref_image, ref_last, ref_loss, req = ctx_forward(dags, sc)
        a = image.double().cpu().numpy()
        b = ref_image.double().cpu().numpy()
        np.testing.assert_allclose(a, b, rtol=IMG_RTOL, atol=IMG_ATOL)
        np.testing.assert_array_equal(last.cpu().numpy(), ref_last.cpu().numpy())
        assert abs(loss.item() - ref_loss.item()) <= LOSS_REL * abs(ref_loss.item())
        assert st.cpu().tolist() == [0, req]


def test_sizes_beyond_the_limit_are_refused(dags):
    sc = synth.tiny_scene(0)
    big = synth.Scene(np.concatenate([sc.records] * 9), sc.camera, sc.poses, sc.targets)   # 18,000 > 16,384
    assert static_forward(dags, big)[0] == -1
    wide = synth.tiny_scene(0, n=100, width=320, height=120)
    assert static_forward(dags, wide)[0] == -1


def test_pairs_beyond_the_limit_report_capacity_then_the_next_call_is_whole(dags):
    # 1,200 large, nearly opaque Gaussians in front of a 256 x 256 camera each
    # reach most of its 256 tiles: far more than the array's 131,072 (tile,
    # Gaussian) pairs, while n, width and height stay within the limits. The
    # status reports DAGS_E_CAPACITY and the pair count splat_forward needs;
    # a normal call afterwards still matches splat_forward.
    sc = synth.tiny_scene(6, n=1200, width=256, height=256, f=200.0)
    rec = sc.records.copy()
    rec[:, 8:11] = np.log(0.6)        # log-scales: 0.6 m at 1-4 m
    rec[:, 3] = 3.0                   # opacity logit
    big = synth.Scene(rec, sc.camera, sc.poses, sc.targets)
    code, image, last, loss, st = static_forward(dags, big)
    assert code == 0
    cam = dags.Camera(*big.camera.as_tuple())
    g = torch.from_numpy(np.ascontiguousarray(big.records)).cuda()
    ctx = dags.Context(g.shape[0], cam.width, cam.height, 1, max_pairs=4_000_000)
    ctx.forward(g, cam, torch.from_numpy(np.ascontiguousarray(big.poses)).cuda(),
                torch.from_numpy(np.ascontiguousarray(big.targets)).cuda())
    rc, req = ctx.sync_status()
    assert rc == 0 and req > 131_072
    assert st.cpu().tolist() == [-3, req]          # DAGS_E_CAPACITY
    ctx.close()
    sc = synth.tiny_scene(0)
    code, image, last, loss, st = static_forward(dags, sc)
    assert code == 0
    ref_image, ref_last, ref_loss, req = ctx_forward(dags, sc)
    np.testing.assert_allclose(image.double().cpu().numpy(), ref_image.double().cpu().numpy(), rtol=IMG_RTOL,
                               atol=IMG_ATOL)
    np.testing.assert_array_equal(last.cpu().numpy(), ref_last.cpu().numpy())
    assert st.cpu().tolist() == [0, req]
