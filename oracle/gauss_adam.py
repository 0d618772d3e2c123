"""FP64 oracle of the mapping optimiser step on the Gaussian parameters.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. (27) optimises the Gaussians jointly with the camera poses; the paper
names no optimiser for the map. Reading: Adam (Kingma and Ba, 2015,
Algorithm 1) on every optimised parameter of a record, with one learning rate
per parameter group (mean, opacity logit, quaternion, log-scale, colour) and
the motion probability left to the MP update. The record's FP32 words are the
master copy of the first four groups; the colour is stored BF16 in the record
and kept in FP32 in a separate master copy, from which the record's BF16
colour is refreshed after the step (round to nearest, ties to even).

Record slots: 0-2 mean, 3 opacity logit, 4-7 quaternion, 8-10 log-scale,
11 MP (not optimised), 12-13 BF16 colour. Gradient slots: those of the
record, with 12-14 the colour (r, g, b).

Pins: torch.optim.Adam on the same parameters and gradients (per group),
the first step's closed form (each parameter moves by its learning rate
against the sign of its gradient), the MP slot unchanged, and the BF16
refresh against torch's conversion.
"""
from __future__ import annotations

import numpy as np

GROUPS = {"mean": [0, 1, 2], "opacity": [3], "quat": [4, 5, 6, 7], "scale": [8, 9, 10], "colour": [12, 13, 14]}
SLOTS = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 13, 14]


def bf16_bits(x):
    """uint16 BF16 bits of x (rounded through FP32, to nearest, ties to even)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def bf16_value(bits):
    return (np.asarray(bits, np.uint32) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def params_of(records, colour_master):
    """(n, 15) FP64 parameter vector in gradient slot order; slot 11 = MP."""
    rec = np.asarray(records, np.float32)
    p = np.zeros((rec.shape[0], 15))
    p[:, 0:12] = rec[:, 0:12].astype(np.float64)
    p[:, 12:15] = np.asarray(colour_master, np.float64)[:, 0:3]
    return p


def adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t >= 1 on the slots of SLOTS.

    params, grad: (n, 15) (grad slot order); m, v: (n, 15) moments; lr: a
    dict of group -> learning rate. Returns (params, m, v), new arrays."""
    params, m, v = params.copy(), m.copy(), v.copy()
    g = np.asarray(grad, np.float64)
    for name, cols in GROUPS.items():
        for c in cols:
            m[:, c] = beta1 * m[:, c] + (1.0 - beta1) * g[:, c]
            v[:, c] = beta2 * v[:, c] + (1.0 - beta2) * g[:, c] ** 2
            mhat = m[:, c] / (1.0 - beta1 ** t)
            vhat = v[:, c] / (1.0 - beta2 ** t)
            params[:, c] -= lr[name] * mhat / (np.sqrt(vhat) + eps)
    return params, m, v


def records_after(records, params):
    """The records after a step: FP32 words of slots 0-10, MP unchanged,
    the colour refreshed from the FP32 master as BF16 bits."""
    rec = np.array(records, dtype=np.float32, copy=True)
    rec[:, 0:11] = params[:, 0:11].astype(np.float32)
    w = rec.view(np.uint32)
    b = bf16_bits(params[:, 12:15].astype(np.float32)).astype(np.uint32)
    w[:, 12] = b[:, 0] | (b[:, 1] << 16)
    w[:, 13] = b[:, 2]
    return rec
