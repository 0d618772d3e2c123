"""The mapping optimiser step (gauss_adam_step) against the FP64 oracle's
Adam, and a mapping loop that lowers the mapping loss."""
import numpy as np
import pytest

from oracle import gauss_adam as GA
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


def test_adam_steps_match_the_oracle(dags):
    sc = synth.tiny_scene(0, n=3000)
    rng = np.random.default_rng(4)
    n = sc.records.shape[0]
    gauss = torch.from_numpy(sc.records.copy()).cuda()
    ctx = dags.Context(n, 16, 16, 1)
    state = ctx.gauss_adam_state(gauss)
    cfg = dags.default_gauss_adam_cfg()
    lr = {"mean": cfg.lr_mean, "opacity": cfg.lr_opacity, "quat": cfg.lr_quat, "scale": cfg.lr_scale,
          "colour": cfg.lr_colour}
    torch.cuda.synchronize()
    master = state[0].cpu().numpy()
    p = GA.params_of(sc.records, master)
    m = np.zeros((n, 15))
    v = np.zeros((n, 15))
    for t in range(1, 4):
        g = rng.normal(0, 1, (n, 16)).astype(np.float32)
        g[:, 11] = 0.0
        g[:, 15] = 0.0
        g[rng.random(n) < 0.2] = 0.0                  # Gaussians outside every view
        ctx.gauss_adam_step(gauss, state, torch.from_numpy(g).cuda(), t, cfg)
        p, m, v = GA.adam_step(p, m, v, g[:, 0:15].astype(np.float64), t, lr)
    torch.cuda.synchronize()
    ctx.check()
    rec = gauss.cpu().numpy()
    # FP32 Adam against FP64: each step moves a parameter by at most ~lr;
    # the difference is FP32 rounding of the moments and of the parameter
    for name, cols in GA.GROUPS.items():
        if name == "colour":
            got = state[0].cpu().numpy()[:, 0:3].astype(np.float64)
        else:
            got = rec[:, cols].astype(np.float64)
        ref = p[:, cols]
        tol = 1e-4 * lr[name] + 4e-7 * np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol, (name, np.abs(got - ref).max(), tol)
    np.testing.assert_array_equal(rec[:, 11], sc.records[:, 11])         # MP untouched
    # the record's colour is exactly the BF16 of the master
    ref_rec = GA.records_after(sc.records, GA.params_of(sc.records, state[0].cpu().numpy()))
    np.testing.assert_array_equal(rec.view(np.uint32)[:, 12:14], ref_rec.view(np.uint32)[:, 12:14])
    ctx.close()


def test_mapping_iterations_lower_the_mapping_loss(dags):
    # 40k Gaussians of the room with perturbed means, opacities and colours,
    # fitted to 4 keyframes rendered from the unperturbed map: Adam on the
    # splat_backward gradient lowers the summed loss of Eqs. (21), (22).
    sc = synth.mapping_scene(40_000, views=4, width=320, height=240)
    cam = dags.Camera(*sc.camera.as_tuple())
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 4)
    gt = torch.from_numpy(sc.records).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    image, _, _ = ctx.forward(gt, cam, poses)
    V, P = poses.shape[0], cam.width * cam.height
    img = image.reshape(V, 8, P)
    tg = torch.zeros((V, P, 4), dtype=torch.float32, device="cuda")
    tg[:, :, 0:3] = img[:, 0:3].transpose(1, 2)
    tg[:, :, 3] = torch.where(img[:, 4] > 0.5, img[:, 3], torch.zeros_like(img[:, 3]))
    rng = np.random.default_rng(1)
    rec = sc.records.copy()
    rec[:, 0:3] += rng.normal(0, 0.01, (rec.shape[0], 3)).astype(np.float32)
    rec[:, 3] += rng.normal(0, 0.5, rec.shape[0]).astype(np.float32)
    gauss = torch.from_numpy(rec).cuda()
    state = ctx.gauss_adam_state(gauss)
    losses = []
    for t in range(1, 61):
        image, last, loss = ctx.forward(gauss, cam, poses, tg)
        gg, _ = ctx.backward(gauss, cam, poses, tg, image, last, dags.GRAD_GAUSS)
        ctx.gauss_adam_step(gauss, state, gg, t)
        losses.append(loss.item())
    torch.cuda.synchronize()
    ctx.check()
    print(f"\nmapping loss: {losses[0]:.1f} -> {losses[-1]:.1f}")
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0]
    ctx.close()
