"""The torch.autograd wrapper: gradients through SplatLoss equal the adjoint
kernels' outputs and, for the pose twist, the FP64 oracle's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def test_autograd_matches_adjoint_and_oracle(dags):
    import oracle
    from paper_2602_21644_gb300 import autograd, synth
    sc = synth.tiny_scene(1)
    cam = dags.Camera(*sc.camera.as_tuple())
    dev = "cuda"
    gauss = torch.from_numpy(sc.records).to(dev).requires_grad_(True)
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).to(dev)
    targets = torch.from_numpy(sc.targets).to(dev)
    xi = torch.zeros((1, 6), dtype=torch.float64, device=dev, requires_grad=True)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    loss = autograd.splat_loss(ctx, cam, gauss, poses, targets, xi)
    (2.0 * loss).sum().backward()
    torch.cuda.synchronize()
    ctx.check()
    image, last, loss2 = ctx.forward(gauss.detach(), cam, poses, targets)
    gg, gp = ctx.backward(gauss.detach(), cam, poses, targets, image, last, dags.GRAD_GAUSS | dags.GRAD_POSE)
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(loss2.item(), rel=1e-12)
    a, b = gauss.grad.cpu().numpy(), 2.0 * gg.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)      # atomics order only
    # the per-Gaussian 2D gradients are FP32 atomics: their order, and so the
    # rounding, differs between two backward launches (norm-wise, as for the
    # Gaussian gradients)
    xa, xb = xi.grad.cpu().numpy(), 2.0 * gp.cpu().numpy()
    assert np.linalg.norm(xa - xb) <= 1e-5 * np.linalg.norm(xb)
    G = oracle.params_from_records(sc.records)
    ref = oracle.render(G, oracle.camera_vec(*sc.camera.as_tuple()), sc.poses[0], targets=sc.targets[0], grads=True)
    rel = np.linalg.norm(xi.grad[0].cpu().numpy() / 2.0 - ref["pose_grad"]) / np.linalg.norm(ref["pose_grad"])
    assert rel < 1e-4
    ctx.close()


def test_autograd_without_pose_gradient(dags):
    from paper_2602_21644_gb300 import autograd, synth
    sc = synth.tiny_scene(2)
    cam = dags.Camera(*sc.camera.as_tuple())
    gauss = torch.from_numpy(sc.records).cuda().requires_grad_(True)
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    targets = torch.from_numpy(sc.targets).cuda()
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    loss = autograd.splat_loss(ctx, cam, gauss, poses, targets)
    loss.sum().backward()
    torch.cuda.synchronize()
    ctx.check()
    assert gauss.grad is not None and torch.isfinite(gauss.grad).all()
    assert gauss.grad.abs().sum().item() > 0
    ctx.close()


def test_render_autograd_with_a_user_loss_matches_the_oracle(dags):
    # A caller's own loss on the rendered channels: sum of a*C + b*D^2/2 +
    # c*O + d*R_MP with fixed random per-pixel weights. torch.autograd passes
    # dF/d(channels) to the library's adjoint; the FP64 oracle takes the same
    # upstream (its adjoint with a given upstream is pinned by central
    # differences).
    import oracle
    from paper_2602_21644_gb300 import autograd, synth
    from gpu_common import GRAD_MASK_FLAGS, compare_grads
    sc = synth.tiny_scene(3)
    cam = dags.Camera(*sc.camera.as_tuple())
    dev = "cuda"
    G = oracle.params_from_records(sc.records)
    ocam = oracle.camera_vec(*sc.camera.as_tuple())
    ref0 = oracle.render(G, ocam, sc.poses[0])
    P = cam.width * cam.height
    rng = np.random.default_rng(9)
    wts = rng.normal(size=(P, 6))
    wts[(ref0["flags"] & GRAD_MASK_FLAGS) != 0] = 0.0     # pixels whose decisions FP32 may take otherwise
    gauss = torch.from_numpy(sc.records).to(dev).requires_grad_(True)
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).to(dev)
    xi = torch.zeros((1, 6), dtype=torch.float64, device=dev, requires_grad=True)
    ctx = dags.Context(gauss.shape[0], cam.width, cam.height, 1)
    C, D, O, R = autograd.splat_render(ctx, cam, gauss, poses, xi)
    w = torch.from_numpy(wts.T.reshape(6, cam.height, cam.width)).to(dev).float()
    F = (w[0:3] * C[0]).sum() + 0.5 * (w[3] * D[0] * D[0]).sum() + (w[4] * O[0]).sum() + (w[5] * R[0]).sum()
    F.backward()
    torch.cuda.synchronize()
    ctx.check()
    # the same F's upstream for the oracle: dF/dD = w3 D
    up = wts.copy()
    up[:, 3] = wts[:, 3] * ref0["pix"][:, 3]
    ref = oracle.render(G, ocam, sc.poses[0], upstream=up, grads=True, grad_mag=True)
    report = []
    g = compare_grads(gauss.grad.cpu().numpy().astype(np.float64), ref["grad"], report, mag=ref["grad_mag"])
    print("\n".join(report))
    for k, v in g.items():
        assert v <= 1e-4, k
    pg = np.linalg.norm(xi.grad[0].cpu().numpy() - ref["pose_grad"]) / np.linalg.norm(ref["pose_grad"])
    assert pg <= 1e-4, pg
    # the rendered channels are the forward's (pixels whose decisions FP32
    # may take otherwise are compared within their validity envelope)
    from gpu_common import compare_image
    img = np.zeros((P, 8))
    img[:, 0:3] = C[0].permute(1, 2, 0).reshape(P, 3).detach().cpu().numpy()
    img[:, 3] = D[0].reshape(P).detach().cpu().numpy()
    img[:, 4] = O[0].reshape(P).detach().cpu().numpy()
    img[:, 5] = R[0].reshape(P).detach().cpu().numpy()
    ref_pix = ref0["pix"].copy()
    img[:, 6] = ref_pix[:, 6]           # transmittance and weight: not outputs of SplatRender
    img[:, 7] = ref_pix[:, 9]
    worst, _ = compare_image(img, ref_pix, ref0["flags"])
    for c in range(6):
        assert worst[c][2] == 0, (c, worst[c])
    ctx.close()
