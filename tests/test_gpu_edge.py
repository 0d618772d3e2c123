"""GPU edge-warp regulariser (splat_edge_warp, C ABI) against the FP64 oracle
(oracle/edge.py, Sec. IV-D, Eqs. (25), (26)): a two-plane step scene at
several sizes (ragged included) in both readings of the compared depth, and
two consecutive ray-cast tracking frames."""
import numpy as np
import pytest

from oracle import edge as oedge
from oracle import pose as opose
from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L_REL = 2e-4       # FP32 warp and bilinear sampling against FP64
G_REL = 2e-3       # the gradients, normwise per pose


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def step_frames(W, H, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    s = W / 48.0
    Di = np.where(xx < s * (20 + 0.3 * yy / s), 1.5 + 0.004 * xx / s, 2.4 - 0.003 * yy / s)
    Dj = np.where(xx < s * (20.6 + 0.3 * yy / s), 1.51 + 0.004 * xx / s, 2.38 - 0.003 * yy / s)
    Di[rng.random((H, W)) < 0.03] = 0.0
    Dj[rng.random((H, W)) < 0.01] = 0.0
    wj = 0.5 + 0.4 * np.sin(0.2 * xx / s) * np.cos(0.15 * yy / s)
    f = 40.0 * s
    cam = (f, f, W / 2.0 - 0.7, H / 2.0 - 0.4, W, H)
    Ti = opose.apply_left(rng.normal(0, 0.02, 6), np.hstack([np.eye(3), np.zeros((3, 1))]))
    Tj = opose.apply_left(rng.normal(0, 0.02, 6), Ti)
    return cam, Di.ravel().astype(np.float32), Dj.ravel().astype(np.float32), wj.ravel().astype(np.float32), Ti, Tj


def run(dags, cam, Di, Dj, wj, Ti, Tj, literal=False):
    W, H = int(cam[4]), int(cam[5])
    c = dags.Camera(*cam)
    ctx = dags.Context(16, W, H, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = ctx.edge_warp(c, t(Di), t(Dj), t(wj), t(Ti.ravel()), t(Tj.ravel()), 300.0,
                        cfg=dags.default_edge_cfg(literal=int(literal)))
    torch.cuda.synchronize()
    ctx.check()
    res = out.cpu().numpy()
    out2 = ctx.edge_warp(c, t(Di), t(Dj), t(wj), t(Ti.ravel()), t(Tj.ravel()), 300.0,
                         cfg=dags.default_edge_cfg(literal=int(literal)))
    assert np.array_equal(out2.cpu().numpy(), res)       # deterministic
    ctx.close()
    ref = oedge.edge_warp(cam, Di, Dj, wj, Ti, Tj, oedge.EdgeConfig(literal=literal))
    return res, ref


def compare(res, ref, label):
    eL = abs(res[0] - ref["L"]) / ref["L"]
    ei = np.linalg.norm(res[1:7] - ref["grad_i"]) / np.linalg.norm(ref["grad_i"])
    ej = np.linalg.norm(res[7:13] - ref["grad_j"]) / np.linalg.norm(ref["grad_j"])
    print(f"\n{label}: edges {ref['edges']} counted {ref['n']} flagged {ref['flagged']}: L {eL:.2e} "
          f"grad_i {ei:.2e} grad_j {ej:.2e}")
    assert ref["n"] > 50
    assert eL <= L_REL and ei <= G_REL and ej <= G_REL


@pytest.mark.parametrize("W,H,literal", [(48, 36, False), (160, 120, False), (161, 97, True), (640, 480, False)])
def test_step_scene(dags, W, H, literal):
    cam, Di, Dj, wj, Ti, Tj = step_frames(W, H, W + H)
    res, ref = run(dags, cam, Di, Dj, wj, Ti, Tj, literal)
    compare(res, ref, f"step {W}x{H} literal={literal}")


def test_consecutive_tracking_frames(dags):
    # frames 11 (i) and 12 (j) of the synthetic sequence at 320x240: ray-cast
    # depth with 1% noise, the ground-truth poses, a smooth weight map
    rec, cam, seq, _ = synth.tracking_sequence(20_000, frames=[11, 12], width=320, height=240)
    Di = seq[0]["target"][:, 3].copy()
    Dj = seq[1]["target"][:, 3].copy()
    yy, xx = np.mgrid[0:240, 0:320]
    wj = (0.6 + 0.3 * np.cos(0.05 * xx) * np.sin(0.04 * yy)).astype(np.float32).ravel()
    res, ref = run(dags, cam.as_tuple(), Di, Dj, wj, seq[0]["gt_pose"], seq[1]["gt_pose"])
    compare(res, ref, "tracking frames 11 -> 12")


def test_no_edges_gives_zero(dags):
    cam, Di, Dj, wj, Ti, Tj = step_frames(48, 36, 5)
    flat = np.full_like(Di, 2.0)
    res, ref = run(dags, cam, flat, flat, wj, Ti, Tj)
    assert ref["n"] == 0 and np.all(res == 0.0)
