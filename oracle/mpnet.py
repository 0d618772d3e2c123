"""FP64 oracle of the per-pixel learned MP proposal network.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network is not in the paper; the benchmark spec asks for a small
per-pixel network over rendered MP, colour/depth residuals and depth that
proposes MP between scheduled semantic invocations (the paper's
semantic-on-demand scheduling, Sec. IV-B, reuses a stale prior between
invocations; this network is the learned stand-in for that gap). Layer order
(the reading of "1x1 conv 8 -> 32 -> 32 -> 1 plus one 3x3 conv 32 -> 32"):

    z1 = W1 x + b1            (1x1, 8 -> 32)        a1 = bf16(relu(z1))
    z2 = conv3x3(a1) + b2     (32 -> 32, zero pad)  a2 = bf16(relu(z2))
    z3 = W3 a2 + b3           (1x1, 32 -> 32)       a3 = bf16(relu(z3))
    z4 = w4 . a3 + b4         (1x1, 32 -> 1)        y  = sigmoid(z4)

Weights and inputs are BF16 values, biases FP32 values; sums are exact
(FP64); activations are rounded to BF16 (FP64 -> FP32 -> BF16, each to
nearest, ties to even) where the kernel rounds them. Training loss: mean
binary cross-entropy against a target MP map over valid pixels (target >= 0);
the backward treats the BF16 rounding of activations as the identity.

Input channels (per pixel, `features`): rendered MP, |dR|, |dG|, |dB|,
|dDepth|, observed depth, rendered opacity, prior mask (the MP_ins of the
pixel's instance region, Eq. (2)). Tensors are NHWC.

Training step: Adam (Kingma and Ba, 2015) with beta1 0.9, beta2 0.999,
eps 1e-8 on FP32 master weights; the network's optimiser is not in the paper
and this is the reading taken.

Pins (tests/test_oracle_mpnet.py): conv3x3 against torch.nn.functional.conv2d
in float64, the BF16 rounding against torch's bfloat16 conversion, the
parameter count (10,625), central finite differences of the loss with
rounding off, and Adam against torch.optim.Adam and its first-step closed
form (every parameter moves by lr against the sign of its gradient).
"""
from __future__ import annotations

import numpy as np

C_IN, C_H = 8, 32
N_PARAMS = C_H * C_IN + C_H + C_H * C_H * 9 + C_H + C_H * C_H + C_H + C_H + 1   # 10,625


def bf16_round(x):
    """Round to BF16 (via FP32), each step to nearest, ties to even; float64 out."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(r_mp, c_rend, d_rend, o_rend, c_obs, d_obs, inst, table):
    """Per-pixel input of the network (P x 8, BF16 values): rendered MP,
    |C_obs - C_rend| per channel, |D_obs - D_rend| where the observed depth is
    valid (> 0, else 0), observed depth (0 where invalid), rendered opacity,
    and the prior MP of the pixel's instance region (table[inst, 0], the
    MP_ins of Eq. (2)). Differences are taken in FP32 (the kernel's inputs)
    and rounded to BF16 once."""
    f32 = lambda v: np.asarray(v, np.float32)
    c_rend, c_obs = f32(c_rend).reshape(-1, 3), f32(c_obs).reshape(-1, 3)
    d_rend, d_obs = f32(d_rend).ravel(), f32(d_obs).ravel()
    valid = d_obs > 0
    out = np.zeros((d_obs.size, 8), np.float64)
    out[:, 0] = f32(r_mp).ravel()
    out[:, 1:4] = np.abs(c_obs - c_rend)
    out[:, 4] = np.where(valid, np.abs(d_obs - d_rend), np.float32(0))
    out[:, 5] = np.where(valid, d_obs, np.float32(0))
    out[:, 6] = f32(o_rend).ravel()
    out[:, 7] = np.asarray(table, np.float64).reshape(-1, 2)[np.asarray(inst).astype(np.int64).ravel(), 0]
    return bf16_round(out)


def init_params(seed=0):
    """He-style initial weights rounded to BF16, zero biases except b4."""
    rng = np.random.default_rng(seed)
    p = dict(
        W1=bf16_round(rng.normal(0, np.sqrt(2.0 / C_IN), (C_H, C_IN))),
        b1=np.zeros(C_H),
        W2=bf16_round(rng.normal(0, np.sqrt(2.0 / (9 * C_H)), (C_H, C_H, 3, 3))),   # [out, in, ky, kx]
        b2=np.zeros(C_H),
        W3=bf16_round(rng.normal(0, np.sqrt(2.0 / C_H), (C_H, C_H))),
        b3=np.zeros(C_H),
        w4=bf16_round(rng.normal(0, np.sqrt(1.0 / C_H), C_H)),
        b4=np.array([0.0]),
    )
    return p


def conv3x3(a, W2):
    """Zero-padded 3x3 convolution (cross-correlation) of NHWC a with W2
    [out, in, ky, kx]: out[b, y, x, o] = sum_{i, ky, kx} W2[o, i, ky, kx] *
    a[b, y + ky - 1, x + kx - 1, i]."""
    B, H, W, C = a.shape
    pad = np.zeros((B, H + 2, W + 2, C))
    pad[:, 1:H + 1, 1:W + 1] = a
    out = np.zeros((B, H, W, W2.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += pad[:, ky:ky + H, kx:kx + W] @ W2[:, :, ky, kx].T
    return out


def forward(x, p, rounding=True):
    """Activations of every layer (dict) for NHWC input x (BF16 values)."""
    rnd = bf16_round if rounding else (lambda v: v)
    x = np.asarray(x, np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = conv3x3(a1, p["W2"]) + p["b2"]
    a2 = rnd(np.maximum(z2, 0.0))
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = rnd(np.maximum(z3, 0.0))
    z4 = a3 @ p["w4"] + p["b4"][0]
    y = 1.0 / (1.0 + np.exp(-z4))
    return dict(z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, z4=z4, y=y)


def loss_and_grads(x, target, p, rounding=True):
    """Mean BCE over pixels with target >= 0 and its gradients (dict like p)."""
    f = forward(x, p, rounding)
    t = np.asarray(target, np.float64)
    valid = t >= 0
    nv = max(int(valid.sum()), 1)
    y = np.clip(f["y"], 1e-12, 1 - 1e-12)
    tt = np.where(valid, t, 0.0)
    L = -np.sum(np.where(valid, tt * np.log(y) + (1 - tt) * np.log(1 - y), 0.0)) / nv
    dz4 = np.where(valid, f["y"] - tt, 0.0) / nv
    g = {}
    g["b4"] = np.array([dz4.sum()])
    g["w4"] = np.einsum("bhw,bhwc->c", dz4, f["a3"])
    dz3 = dz4[..., None] * p["w4"] * (f["z3"] > 0)
    g["b3"] = dz3.sum((0, 1, 2))
    g["W3"] = np.einsum("bhwo,bhwi->oi", dz3, f["a2"])
    dz2 = (dz3 @ p["W3"]) * (f["z2"] > 0)
    g["b2"] = dz2.sum((0, 1, 2))
    B, H, W, C = f["a1"].shape
    pad = np.zeros((B, H + 2, W + 2, C))
    pad[:, 1:H + 1, 1:W + 1] = f["a1"]
    g["W2"] = np.zeros_like(p["W2"])
    da1p = np.zeros((B, H + 2, W + 2, C))
    for ky in range(3):
        for kx in range(3):
            g["W2"][:, :, ky, kx] = np.einsum("bhwo,bhwi->oi", dz2, pad[:, ky:ky + H, kx:kx + W])
            da1p[:, ky:ky + H, kx:kx + W] += dz2 @ p["W2"][:, :, ky, kx]
    dz1 = da1p[:, 1:H + 1, 1:W + 1] * (f["z1"] > 0)
    g["b1"] = dz1.sum((0, 1, 2))
    g["W1"] = np.einsum("bhwo,bhwi->oi", dz1, np.asarray(x, np.float64))
    return L, g, f


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015, Algorithm 1) on dicts of arrays:
    first and second moment estimates with bias correction by the step count
    (step >= 1). Returns (params, m, v) as new dicts."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        g = np.asarray(grads[k], np.float64)
        out_m[k] = beta1 * m[k] + (1 - beta1) * g
        out_v[k] = beta2 * v[k] + (1 - beta2) * g * g
        mhat = out_m[k] / (1 - beta1 ** step)
        vhat = out_v[k] / (1 - beta2 ** step)
        out_p[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return out_p, out_m, out_v


def pack_weights(p):
    """The kernel's weight layout (all BF16 values; float64 here):
    W1 [32 x 16] (input channels 8-15 zero), W2 [32 x 288] with column
    index (ky * 3 + kx) * 32 + in, W3 [32 x 32], w4 [32]; biases b1, b2, b3
    [32] and b4 [1] in FP32."""
    W1 = np.zeros((C_H, 16))
    W1[:, :C_IN] = p["W1"]
    W2 = np.transpose(p["W2"], (0, 2, 3, 1)).reshape(C_H, 9 * C_H)
    return dict(W1=W1, W2=W2, W3=p["W3"].copy(), w4=p["w4"].copy(), b1=p["b1"].copy(), b2=p["b2"].copy(),
                b3=p["b3"].copy(), b4=p["b4"].copy())
