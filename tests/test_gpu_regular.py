"""GPU MP motion-consistency regulariser (splat_mp_consistency, C ABI) against
the FP64 oracle (oracle/regular.py, Sec. IV-D, Eqs. (23), (24))."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import regular as oreg
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


def records(n, seed):
    rng = np.random.default_rng(seed)
    rec, _, _ = synth.room_scene(n, seed)
    rec = rec.copy()
    rec[:, 11] = rng.uniform(0, 1, n).astype(np.float32)
    prev = rec.copy()
    prev[:, 0:3] += rng.normal(0, 0.01, (n, 3)).astype(np.float32)
    return rec, prev


@pytest.mark.parametrize("n,rel", [(100_003, False), (300_000, False), (4_097, True)])
def test_matches_oracle(dags, n, rel):
    rec, prev = records(n, n)
    T = None
    if rel:
        T = np.hstack([Rotation.from_rotvec([0.01, -0.02, 0.005]).as_matrix(), [[0.02], [-0.01], [0.03]]])
    ctx = dags.Context(n, 16, 16, 1)
    g = torch.from_numpy(rec).cuda()
    p = torch.from_numpy(prev).cuda()
    grad = torch.full_like(g, 0.25)              # the gradient is added to what is there
    rel_d = None if T is None else torch.from_numpy(T.ravel().copy()).cuda()
    loss = ctx.mp_consistency(g, p, 500.0, rel_pose=rel_d, grad=grad)
    torch.cuda.synchronize()
    ctx.check()
    L, gm = oreg.mp_consistency(rec[:, 0:3], rec[:, 11], prev[:, 0:3], 500.0, rel_pose=T)
    assert abs(loss.item() - L) <= 1e-6 * L
    out = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(gm).max()
    np.testing.assert_allclose(out[:, 0:3] - 0.25, gm, rtol=1e-5, atol=(1e-5 if rel else 1e-6) * scale)
    assert np.all(out[:, 3:] == 0.25)
    # deterministic loss
    loss2 = ctx.mp_consistency(g, p, 500.0, rel_pose=rel_d)
    assert loss2.item() == loss.item()
    ctx.close()


def test_empty_and_loss_only(dags):
    ctx = dags.Context(1000, 16, 16, 1)
    g = torch.zeros((0, 16), dtype=torch.float32, device="cuda")
    assert ctx.mp_consistency(g, g.clone(), 500.0).item() == 0.0
    rec, prev = records(1000, 3)
    g = torch.from_numpy(rec).cuda()
    p = torch.from_numpy(prev).cuda()
    assert ctx.mp_consistency(g, p, 0.0).item() == 0.0
    # more Gaussians than the context holds
    big = torch.zeros((1001, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(dags.DagsError):
        ctx.mp_consistency(big, big.clone(), 500.0)
    ctx.close()


def test_autograd(dags):
    from paper_2602_21644_gb300 import autograd
    rec, prev = records(5000, 4)
    ctx = dags.Context(5000, 16, 16, 1)
    g = torch.from_numpy(rec).cuda().requires_grad_(True)
    p = torch.from_numpy(prev).cuda()
    loss = autograd.mp_consistency(ctx, g, p, 500.0)
    (2.0 * loss).sum().backward()
    L, gm = oreg.mp_consistency(rec[:, 0:3], rec[:, 11], prev[:, 0:3], 500.0)
    assert abs(loss.item() - L) <= 1e-6 * L
    np.testing.assert_allclose(g.grad.cpu().numpy()[:, 0:3], 2.0 * gm, rtol=1e-5, atol=1e-6 * np.abs(gm).max())
    assert not g.grad[:, 3:].any()
    ctx.close()
