"""Pins of the mapping optimiser oracle (Adam on the Gaussian parameters)."""
import numpy as np
import pytest

from oracle import gauss_adam as GA
from paper_2602_21644_gb300 import synth

torch = pytest.importorskip("torch")

LR = {"mean": 1e-3, "opacity": 0.05, "quat": 1e-3, "scale": 5e-3, "colour": 2.5e-3}


def test_matches_torch_adam_over_steps():
    rng = np.random.default_rng(0)
    n = 50
    p0 = rng.normal(size=(n, 15))
    m = np.zeros((n, 15))
    v = np.zeros((n, 15))
    p = p0.copy()
    tp = {k: torch.tensor(p0[:, cols], dtype=torch.float64, requires_grad=True) for k, cols in GA.GROUPS.items()}
    opt = torch.optim.Adam([{"params": [tp[k]], "lr": LR[k]} for k in GA.GROUPS], betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.normal(size=(n, 15))
        p, m, v = GA.adam_step(p, m, v, g, t, LR)
        opt.zero_grad()
        for k, cols in GA.GROUPS.items():
            tp[k].grad = torch.tensor(g[:, cols])
        opt.step()
    for k, cols in GA.GROUPS.items():
        np.testing.assert_allclose(p[:, cols], tp[k].detach().numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(p[:, 11], p0[:, 11])     # the MP slot is not optimised


def test_first_step_moves_each_parameter_by_its_learning_rate():
    # at t = 1, m_hat = g and v_hat = g^2: the step is lr * g / (|g| + eps)
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=(10, 15))
    g = rng.normal(size=(10, 15))
    p, _, _ = GA.adam_step(p0, np.zeros((10, 15)), np.zeros((10, 15)), g, 1, LR)
    for k, cols in GA.GROUPS.items():
        np.testing.assert_allclose(p[:, cols] - p0[:, cols], -LR[k] * g[:, cols] / (np.abs(g[:, cols]) + 1e-8),
                                   rtol=1e-12, atol=1e-15)


def test_colour_refresh_is_bf16_of_the_master():
    sc = synth.tiny_scene(0, n=40)
    master = np.random.default_rng(2).uniform(0, 1, (40, 4)).astype(np.float32)
    params = GA.params_of(sc.records, master)
    rec = GA.records_after(sc.records, params)
    w = rec.view(np.uint32)
    got = np.stack([w[:, 12] & 0xFFFF, w[:, 12] >> 16, w[:, 13] & 0xFFFF], 1).astype(np.uint16)
    ref = torch.from_numpy(master[:, 0:3]).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(rec[:, 0:12], sc.records[:, 0:12])   # params unchanged here: same words
