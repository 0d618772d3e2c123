"""Pins of the learned-MP-network oracle (no GPU)."""
import numpy as np
import pytest

from oracle import mpnet as N


def test_parameter_count():
    p = N.init_params(0)
    assert sum(v.size for v in p.values()) == N.N_PARAMS == 10625


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 1.00390625, 3.1415]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(N.bf16_round(x), ref)


def test_conv3x3_matches_torch_conv2d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    a = rng.normal(0, 1, (2, 7, 9, 32))
    W2 = rng.normal(0, 1, (32, 32, 3, 3))
    ref = torch.nn.functional.conv2d(torch.from_numpy(a).permute(0, 3, 1, 2), torch.from_numpy(W2), padding=1)
    np.testing.assert_allclose(N.conv3x3(a, W2), ref.permute(0, 2, 3, 1).numpy(), rtol=1e-12, atol=1e-12)


def test_forward_matches_torch_modules():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p = N.init_params(3)
    p["b1"] = rng.normal(0, 0.1, 32)
    p["b2"] = rng.normal(0, 0.1, 32)
    x = rng.uniform(0, 1, (1, 6, 5, 8))
    t = lambda v: torch.from_numpy(np.asarray(v, np.float64))
    xt = t(x).permute(0, 3, 1, 2)
    h = torch.relu(torch.nn.functional.conv2d(xt, t(p["W1"])[:, :, None, None], t(p["b1"])))
    h = torch.relu(torch.nn.functional.conv2d(h, t(p["W2"]), t(p["b2"]), padding=1))
    h = torch.relu(torch.nn.functional.conv2d(h, t(p["W3"])[:, :, None, None], t(p["b3"])))
    y = torch.sigmoid(torch.nn.functional.conv2d(h, t(p["w4"])[None, :, None, None], t(p["b4"])))
    f = N.forward(x, p, rounding=False)
    np.testing.assert_allclose(f["y"], y[:, 0].numpy(), rtol=1e-12)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    p = N.init_params(5)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.2, 32)
    x = rng.uniform(0, 1, (2, 5, 6, 8))
    target = rng.uniform(0, 1, (2, 5, 6))
    target[0, 0, 0] = -1.0                      # an invalid pixel
    L, g, f = N.loss_and_grads(x, target, p, rounding=False)
    for key in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        flat = p[key].reshape(-1)
        idx = rng.choice(flat.size, min(12, flat.size), replace=False)
        for i in idx:
            h = 1e-6
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[key].reshape(-1)[i] += h
            pm[key].reshape(-1)[i] -= h
            fd = (N.loss_and_grads(x, target, pp, False)[0] - N.loss_and_grads(x, target, pm, False)[0]) / (2 * h)
            assert g[key].reshape(-1)[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (key, i)


def test_pack_layout():
    p = N.init_params(6)
    w = N.pack_weights(p)
    assert w["W1"].shape == (32, 16) and np.all(w["W1"][:, 8:] == 0)
    o, i, ky, kx = 5, 7, 2, 0
    assert w["W2"][o, (ky * 3 + kx) * 32 + i] == p["W2"][o, i, ky, kx]


def test_adam_first_step_closed_form():
    # after one step, m_hat = g and v_hat = g^2, so every weight moves by
    # lr * g / (|g| + eps)
    rng = np.random.default_rng(8)
    p = {"a": rng.normal(0, 1, 50)}
    g = {"a": rng.normal(0, 1, 50)}
    z = {"a": np.zeros(50)}
    q, m, v = N.adam_step(p, g, z, z, 1, 0.01)
    np.testing.assert_allclose(q["a"], p["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=0, atol=1e-15)


def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    w0 = rng.normal(0, 1, 40)
    gs = [rng.normal(0, 1, 40) for _ in range(5)]
    t = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = {"w": w0.copy()}, {"w": np.zeros(40)}, {"w": np.zeros(40)}
    for k, g in enumerate(gs, start=1):
        t.grad = torch.tensor(g)
        opt.step()
        p, m, v = N.adam_step(p, {"w": g}, m, v, k, 3e-3)
    np.testing.assert_allclose(p["w"], t.detach().numpy(), rtol=0, atol=1e-14)


def test_features_closed_form():
    # three pixels: valid depth, invalid depth (0), and an instance pixel
    table = np.array([[0.1, 0.05], [0.9, 0.8]])
    f = N.features(r_mp=[0.25, 0.0, 0.5], c_rend=[[0.5, 0.5, 0.5], [0.2, 0.3, 0.4], [1, 1, 1]],
                   d_rend=[2.0, 3.0, 1.5], o_rend=[1.0, 0.5, 0.75],
                   c_obs=[[0.75, 0.25, 0.5], [0.2, 0.3, 0.4], [0, 1, 0.5]], d_obs=[2.5, 0.0, 1.0],
                   inst=[0, 0, 1], table=table)
    want = np.array([[0.25, 0.25, 0.25, 0.0, 0.5, 2.5, 1.0, 0.1],
                     [0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.5, 0.1],
                     [0.5, 1.0, 0.0, 0.5, 0.5, 1.0, 0.75, 0.9]])
    np.testing.assert_array_equal(f, N.bf16_round(want))
