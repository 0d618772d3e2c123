"""Learned MP network on the tensor cores (mpnet_infer, C ABI) against the
FP64 oracle (oracle/mpnet.py) with the same BF16 rounding points."""
import numpy as np
import pytest

from oracle import mpnet as N
from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

Y_ABS = 1e-2          # final MP, absolute (task statement)
ULP_FRAC = 0.999      # activations within one BF16 ulp on at least this fraction


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def bf16_bits(x):
    return synth.f32_to_bf16_bits(np.asarray(x, np.float32))


def weight_blob(p):
    w = N.pack_weights(p)
    blob = np.zeros(22016, np.uint8)
    blob[0:1024] = bf16_bits(w["W1"]).view(np.uint8).ravel()
    blob[1024:19456] = bf16_bits(w["W2"]).view(np.uint8).ravel()
    blob[19456:21504] = bf16_bits(w["W3"]).view(np.uint8).ravel()
    blob[21504:21568] = bf16_bits(w["w4"]).view(np.uint8).ravel()
    for off, key in ((21568, "b1"), (21696, "b2"), (21824, "b3")):
        blob[off:off + 128] = np.asarray(w[key], np.float32).view(np.uint8)
    blob[21952:21956] = np.asarray(w["b4"], np.float32).view(np.uint8)
    return blob


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = N.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = np.asarray(rng.normal(0, 0.2, 32), np.float32).astype(np.float64)
    p["b4"] = np.array([np.float32(rng.normal(0, 0.3))], np.float64)
    return p


def to_bf16_tensor(x):
    bits = bf16_bits(x)
    return torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).cuda()


def ulp_close(a, b):
    """Fraction of BF16 values equal or one ulp apart."""
    ai = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    bi = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    return np.mean(np.abs(ai - bi) <= (1 << 16))


@pytest.mark.parametrize("B,H,W", [(1, 6, 128), (2, 9, 300), (1, 3, 700), (1, 2, 1), (1, 1, 5), (3, 4, 17),
                                   (1, 70, 129)])
def test_forward_matches_oracle(dags, B, H, W):
    rng = np.random.default_rng(B * 100 + H)
    p = random_params(7)
    x = N.bf16_round(rng.uniform(0, 1, (B, H, W, 8)))
    ctx = dags.Context(16, 16, 16, 1)
    wt = torch.from_numpy(weight_blob(p)).cuda()
    feats = to_bf16_tensor(x)
    acts = torch.empty((B, H, W, 96), dtype=torch.bfloat16, device="cuda")
    y = ctx.mpnet_infer(wt, feats, acts=acts)
    torch.cuda.synchronize()
    ctx.check()
    f = N.forward(x, p)
    a = acts.float().cpu().numpy()
    for name, sl in (("a1", slice(0, 32)), ("a2", slice(32, 64)), ("a3", slice(64, 96))):
        frac = ulp_close(a[..., sl], f[name])
        assert frac >= ULP_FRAC, f"{name}: only {frac:.5f} within one BF16 ulp"
    err = np.abs(y.cpu().numpy() - f["y"])
    assert err.max() <= Y_ABS, err.max()
    assert np.mean(err <= 1e-3) >= 0.99


def test_forward_full_frame_batch(dags):
    # 16 frames of 640x480 per launch (the inference batch); sampled rows
    # against the oracle
    B, H, W = 16, 480, 640
    rng = np.random.default_rng(11)
    p = random_params(3)
    xs = rng.uniform(0, 1, (B, H, W, 8)).astype(np.float32)
    feats = to_bf16_tensor(xs)
    ctx = dags.Context(16, 16, 16, 1)
    y = ctx.mpnet_infer(torch.from_numpy(weight_blob(p)).cuda(), feats)
    torch.cuda.synchronize()
    ctx.check()
    yc = y.cpu().numpy()
    xb = N.bf16_round(xs)
    for b, r in ((0, 0), (5, 240), (15, 479)):
        lo, hi = max(0, r - 1), min(H, r + 2)
        f = N.forward(xb[b:b + 1, lo:hi], p)
        ref = f["y"][0, r - lo]
        assert np.abs(yc[b, r] - ref).max() <= Y_ABS


# ------------------------------------------------------------------ training

GRAD_REL = 1e-2       # per parameter group, relative L2 (BF16 backward operands)
LAYOUT = (("W1", 0, (32, 16)), ("W2", 512, (32, 288)), ("W3", 9728, (32, 32)), ("w4", 10752, (32,)),
          ("b1", 10784, (32,)), ("b2", 10816, (32,)), ("b3", 10848, (32,)), ("b4", 10880, (1,)))


def to_vec(d):
    """Oracle-layout dict (W1 [32, 8], W2 [32, 32, 3, 3], ...) -> parameter vector."""
    w = N.pack_weights(d)
    v = np.zeros(10881)
    for key, off, shape in LAYOUT:
        v[off:off + int(np.prod(shape))] = np.asarray(w[key], np.float64).ravel()
    return v


def from_vec(v):
    d = {}
    for key, off, shape in LAYOUT:
        d[key] = np.asarray(v[off:off + int(np.prod(shape))], np.float64).reshape(shape)
    d["W1"] = d["W1"][:, :8].copy()
    d["W2"] = np.transpose(d["W2"].reshape(32, 3, 3, 32), (0, 3, 1, 2)).copy()
    return d


def train_setup(p, x, target):
    wt = torch.from_numpy(weight_blob(p)).cuda()
    master = torch.from_numpy(to_vec(p).astype(np.float32)).cuda()
    m = torch.zeros(10881, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    feats = to_bf16_tensor(x)
    tg = torch.from_numpy(np.asarray(target, np.float32)).cuda()
    return wt, master, m, v, feats, tg


def group_errors(g_gpu, g_ref):
    out = {}
    for key, off, shape in LAYOUT:
        n = int(np.prod(shape))
        a, b = g_gpu[off:off + n], g_ref[off:off + n]
        out[key] = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    return out


def random_targets(rng, shape):
    t = rng.uniform(0, 1, shape)
    t[rng.uniform(0, 1, shape) < 0.1] = -1.0          # excluded pixels
    return t


@pytest.mark.parametrize("B,H,W", [(1, 6, 128), (2, 9, 300), (1, 40, 640), (1, 3, 700)])
def test_train_gradients_match_oracle(dags, B, H, W):
    rng = np.random.default_rng(31 + H)
    p = random_params(12)
    x = N.bf16_round(rng.uniform(0, 1, (B, H, W, 8)))
    target = random_targets(rng, (B, H, W))
    wt, master, m, v, feats, tg = train_setup(p, x, target)
    blob0 = wt.clone()
    grad = torch.empty(10881, dtype=torch.float32, device="cuda")
    ctx = dags.Context(16, 16, 16, 1)
    loss = ctx.mpnet_train_step(wt, master, m, v, 1, feats, tg, 0.0, grad=grad)
    torch.cuda.synchronize()
    ctx.check()
    L, g, _ = N.loss_and_grads(x, target, p)
    assert loss.item() == pytest.approx(L, rel=1e-4)
    errs = group_errors(grad.cpu().numpy().astype(np.float64), to_vec(g))
    assert max(errs.values()) <= GRAD_REL, errs
    assert torch.equal(wt, blob0)                        # lr 0 leaves the BF16 weights unchanged


def test_train_adam_step_matches_oracle(dags):
    rng = np.random.default_rng(40)
    B, H, W = 1, 10, 200
    p = random_params(13)
    x = N.bf16_round(rng.uniform(0, 1, (B, H, W, 8)))
    target = random_targets(rng, (B, H, W))
    wt, master, m, v, feats, tg = train_setup(p, x, target)
    m0 = rng.normal(0, 1e-3, 10881).astype(np.float32)
    v0 = rng.uniform(0, 1e-5, 10881).astype(np.float32)
    m.copy_(torch.from_numpy(m0))
    v.copy_(torch.from_numpy(v0))
    w0 = master.cpu().numpy().astype(np.float64)
    grad = torch.empty(10881, dtype=torch.float32, device="cuda")
    ctx = dags.Context(16, 16, 16, 1)
    lr, step = 2e-3, 5
    ctx.mpnet_train_step(wt, master, m, v, step, feats, tg, lr, grad=grad)
    torch.cuda.synchronize()
    ctx.check()
    g = grad.cpu().numpy().astype(np.float64)
    q, mm, vv = N.adam_step({"w": w0}, {"w": g}, {"w": m0.astype(np.float64)}, {"w": v0.astype(np.float64)}, step, lr)
    pad = np.zeros(10881, bool)
    pad[:512] = (np.arange(512) % 16) >= 8
    q["w"][pad] = 0.0
    w1 = master.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(w1, q["w"], rtol=0, atol=1e-4 * lr + 4e-7 * np.abs(w0).max())
    # FP32 moments: a few roundings of the terms' magnitudes (they can cancel)
    scale_m = np.abs(m0) + np.abs(g)
    scale_v = np.abs(v0) + g * g
    assert np.all(np.abs(m.cpu().numpy() - mm["w"]) <= 4 * 2.0 ** -24 * scale_m)
    assert np.all(np.abs(v.cpu().numpy() - vv["w"]) <= 4 * 2.0 ** -24 * scale_v)
    # the blob is the BF16 (weights) / FP32 (biases) copy of the new master
    blob = wt.cpu().numpy()
    mv = master.cpu().numpy()
    np.testing.assert_array_equal(blob[:21568].view(np.uint16), bf16_bits(mv[:10784]))
    np.testing.assert_array_equal(blob[21568:21956].view(np.float32), mv[10784:])


def test_train_reduces_loss_and_agrees_with_oracle(dags):
    # a target that depends on a feature and on its 3x3 neighbourhood: the MP
    # map smoothed and thresholded, masked by the prior channel
    rng = np.random.default_rng(50)
    B, H, W = 2, 24, 160
    x = rng.uniform(0, 1, (B, H, W, 8))
    sm = x[..., 0].copy()
    sm[:, 1:-1, 1:-1] = sum(x[:, 1 + dy:H - 1 + dy, 1 + dx:W - 1 + dx, 0] for dy in (-1, 0, 1) for dx in (-1, 0, 1)) / 9
    target = ((sm > 0.5) & (x[..., 7] > 0.3)).astype(np.float64)
    x = N.bf16_round(x)
    p = N.init_params(21)
    wt, master, m, v, feats, tg = train_setup(p, x, target)
    ctx = dags.Context(16, 16, 16, 1)
    losses = []
    for step in range(1, 301):
        losses.append(ctx.mpnet_train_step(wt, master, m, v, step, feats, tg, 3e-3))
    torch.cuda.synchronize()
    ctx.check()
    losses = [l.item() for l in losses]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    # the trained blob, evaluated by the oracle, gives the loss the kernels report
    blob = wt.cpu().numpy()
    vec = np.zeros(10881)
    vec[:10784] = synth.bf16_bits_to_f32(blob[:21568].view(np.uint16))
    vec[10784:] = blob[21568:21956].view(np.float32)
    L, _, _ = N.loss_and_grads(x, target, from_vec(vec))
    grad = torch.empty(10881, dtype=torch.float32, device="cuda")
    last = ctx.mpnet_train_step(wt, master, m, v, 301, feats, tg, 0.0, grad=grad).item()
    assert last == pytest.approx(L, rel=1e-3)


def test_train_gradients_full_frame(dags):
    # one 640 x 480 frame in the launch configuration of the training step
    # (persistent CTAs over 2400 tiles, several tiles per CTA)
    B, H, W = 1, 480, 640
    rng = np.random.default_rng(77)
    p = random_params(14)
    x = N.bf16_round(rng.uniform(0, 1, (B, H, W, 8)))
    target = random_targets(rng, (B, H, W))
    wt, master, m, v, feats, tg = train_setup(p, x, target)
    grad = torch.empty(10881, dtype=torch.float32, device="cuda")
    ctx = dags.Context(16, 16, 16, 1)
    loss = ctx.mpnet_train_step(wt, master, m, v, 1, feats, tg, 0.0, grad=grad)
    torch.cuda.synchronize()
    ctx.check()
    L, g, _ = N.loss_and_grads(x, target, p)
    assert loss.item() == pytest.approx(L, rel=1e-4)
    errs = group_errors(grad.cpu().numpy().astype(np.float64), to_vec(g))
    assert max(errs.values()) <= GRAD_REL, errs


def test_inference_is_deterministic(dags):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (2, 48, 300, 8)).astype(np.float32)
    feats = to_bf16_tensor(x)
    wt = torch.from_numpy(weight_blob(random_params(5))).cuda()
    ctx = dags.Context(16, 16, 16, 1)
    a = ctx.mpnet_infer(wt, feats).clone()
    b = ctx.mpnet_infer(wt, feats)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
