"""FP64 CPU oracle of the MP-aware differentiable splatting hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may use this package; the product
package never imports it. It shares no code with the CUDA path: the C part
(``splat_oracle.c``) is compiled here with gcc, the rest is numpy.

Contents
  splat (C, via ctypes)   projection, binning, render, Eq. (20)-(22) loss and
                          the hand-derived adjoint (Gaussians + pose twist)
  pose                    FP64 Adam step on the 6-DoF twist and the SE(3)
                          exponential (Sec. V-A(c) pose refinement)
  mp                      the spatiotemporal MP update, Eqs. (2)-(12), (17)
  splat.render_jac (C)    forward-mode derivative of the rendered colour and
                          depth along the pose twist, and the IRLS normal
                          equations of the MP-weighted L1 loss
  lm                      Levenberg-Marquardt pose refinement (Sec. V-A(c))
  regular                 the MP motion-consistency regulariser, Eqs. (23), (24)
  edge                    the MP-guided edge-warp regulariser, Eqs. (25), (26)
  epipolar                epipolar verification and static recovery, Eqs. (18), (19)
  mpnet                   the small per-pixel MP proposal network
  schedule                the semantic-on-demand trigger, Eqs. (13)-(16)

Parity status of each function is listed in the module that defines it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_splat.so")
_SRC = os.path.join(_HERE, "splat_oracle.c")
_lock = threading.Lock()
_lib = None

# Layout constants mirrored from splat_oracle.c.
G_STRIDE = 15
PJ_STRIDE = 24
PX_STRIDE = 10
PJ = dict(VIS=0, U=1, V=2, Z=3, A=4, B=5, C=6, O=7, SA=8, SB=9, SC=10, LMAX=11, R=12,
          X0=13, Y0=14, X1=15, Y1=16, FLAG=17, PX=18, PY=19, ZKEY=20,
          EX=21, EY=22, CTHR=23)
PX = dict(CR=0, CG=1, CB=2, D=3, O=4, RMP=5, T=6, N=7, LAST=8, W=9)
FLAGS = dict(ZNEAR=1, CLAMP=2, RADIUS=4, RECT=8, OPAC=16, ALPHA=32, AMAX=64, TSTOP=128,
             ZTIE=256, OEPS=512, SIGN=1024)
# Pixel flags that make a pixel's values not decided identically in FP32 and FP64.
PIXEL_DECISION_FLAGS = FLAGS["ALPHA"] | FLAGS["AMAX"] | FLAGS["TSTOP"] | FLAGS["OEPS"]


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_project.argtypes = [I64, P, P, P, P, P]
        lib.oracle_project.restype = None
        lib.oracle_binning.argtypes = [I64, P, P, P, P, I64, P, P, P]
        lib.oracle_binning.restype = I64
        lib.oracle_render.argtypes = [I64, P, P, P, P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P]
        lib.oracle_render.restype = ctypes.c_int
        lib.oracle_render_pixel.argtypes = [I64, P, P, P, P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_render_pixel.restype = ctypes.c_int
        lib.oracle_render_jac.argtypes = [I64, P, P, P, P, P, P, ctypes.c_double, P, P, P, P]
        lib.oracle_render_jac.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- inputs

def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) to float64 (exact)."""
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def params_from_records(rec: np.ndarray) -> np.ndarray:
    """Decode packed 64-byte Gaussian records (n x 16 float32 words) to the
    oracle's FP64 parameter rows (n x 15).

    Record words: 0-2 mean, 3 opacity logit, 4-7 quaternion (w, x, y, z),
    8-10 log-scale, 11 motion probability, 12 = r | g << 16 and 13 = b as
    BF16 bit patterns, 14-15 unused.
    """
    rec = np.ascontiguousarray(rec, dtype=np.float32).reshape(-1, 16)
    n = rec.shape[0]
    G = np.zeros((n, G_STRIDE), dtype=np.float64)
    G[:, 0:12] = rec[:, 0:12].astype(np.float64)
    w = rec[:, 12:14].view(np.uint32)
    G[:, 12] = bf16_bits_to_f64((w[:, 0] & 0xFFFF).astype(np.uint16))
    G[:, 13] = bf16_bits_to_f64((w[:, 0] >> 16).astype(np.uint16))
    G[:, 14] = bf16_bits_to_f64((w[:, 1] & 0xFFFF).astype(np.uint16))
    return G


def camera_vec(fx, fy, cx, cy, width, height) -> np.ndarray:
    """The camera the C ABI receives: its intrinsics are FP32 fields, so the
    oracle evaluates the FP32-rounded values (in FP64 arithmetic)."""
    f32 = lambda x: float(np.float32(x))
    return np.array([f32(fx), f32(fy), f32(cx), f32(cy), width, height], dtype=np.float64)


def raster_vec(tile=16, alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, dilation=0.3,
               z_near=0.2, guard=1.3) -> np.ndarray:
    return np.array([tile, alpha_min, alpha_max, t_min, dilation, z_near, guard], dtype=np.float64)


def loss_vec(lambda_pho=0.9, lambda_depth=0.1, weight_mode=0, weight_grad=0, o_eps=1e-6) -> np.ndarray:
    """Loss constants. lambda_1 = 0.9 and lambda_2 = 0.1 are the paper's
    (Sec. V-A(c)); weight_mode 0 normalises the compositing weights so that
    they sum to one as Eq. (20) states."""
    return np.array([lambda_pho, lambda_depth, weight_mode, weight_grad, o_eps], dtype=np.float64)


# ---------------------------------------------------------------- calls

def project(G, cam, pose, rc=None):
    """Per-Gaussian projection table (n x PJ_STRIDE), see PJ for columns."""
    lib = _load()
    G = _f64(G, (-1, G_STRIDE))
    rc = raster_vec() if rc is None else _f64(rc)
    out = np.zeros((G.shape[0], PJ_STRIDE))
    lib.oracle_project(G.shape[0], _ptr(G), _ptr(_f64(cam)), _ptr(_f64(pose, (12,))), _ptr(rc), _ptr(out))
    return out


def binning(G, cam, pose, rc=None):
    """(tiles, ids, tie_flags) of all (tile, Gaussian) pairs sorted by
    (tile, FP32 depth key, id); tile = ty * tiles_x + tx."""
    lib = _load()
    G = _f64(G, (-1, G_STRIDE))
    rc = raster_vec() if rc is None else _f64(rc)
    args = (G.shape[0], _ptr(G), _ptr(_f64(cam)), _ptr(_f64(pose, (12,))), _ptr(rc))
    total = lib.oracle_binning(*args, 0, None, None, None)
    tiles = np.zeros(max(total, 1), np.int64)
    ids = np.zeros(max(total, 1), np.int64)
    ties = np.zeros(max(total, 1), np.int32)
    lib.oracle_binning(*args, total, _ptr(tiles), _ptr(ids), _ptr(ties))
    return tiles[:total], ids[:total], ties[:total]


def render(G, cam, pose, rc=None, lc=None, targets=None, grads=False, accel=True, wfix=None, upstream=None,
           grad_mag=False):
    """Render one view and, with targets (H*W x 4: r, g, b, depth), the loss
    and, with grads=True, its adjoint. wfix (H*W) freezes the static weight.
    upstream (H*W x 6: dF/d(C_r, C_g, C_b, D, O, R_MP) of a caller's function
    F of the rendered channels) replaces the loss: with grads=True the
    adjoint is that of F, and targets are not used.

    grad_mag=True (with grads) also returns grad_mag (n x 15): per parameter,
    the sum over pixels and 2D words of |term| |d parameter / d word|, the
    magnitude of what the gradient sums (its rounding bound scales with it).

    Returns dict(pix=(H*W x 10), flags=(H*W,), loss=float|None,
    grad=(n x 15)|None, pose_grad=(6,)|None, grad_mag=(n x 15)|None).
    """
    lib = _load()
    G = _f64(G, (-1, G_STRIDE))
    rc = raster_vec() if rc is None else _f64(rc)
    lc = loss_vec() if lc is None else _f64(lc)
    cam = _f64(cam)
    W, H = int(cam[4]), int(cam[5])
    pix = np.zeros((W * H, PX_STRIDE))
    flags = np.zeros(W * H, np.int32)
    loss = np.zeros(1)
    up = None if upstream is None else _f64(upstream, (W * H, 6))
    tg = None if (targets is None or up is not None) else _f64(targets, (W * H, 4))
    gr = np.zeros((G.shape[0], G_STRIDE)) if (grads and (tg is not None or up is not None)) else None
    pg = np.zeros(6) if gr is not None else None
    gm = np.zeros((G.shape[0], G_STRIDE)) if (gr is not None and grad_mag) else None
    rcode = lib.oracle_render(G.shape[0], _ptr(G), _ptr(cam), _ptr(_f64(pose, (12,))), _ptr(rc), _ptr(lc),
                              _ptr(tg), _ptr(None if wfix is None else _f64(wfix, (W * H,))), _ptr(up),
                              int(bool(accel)), _ptr(pix), _ptr(flags),
                              _ptr(loss) if tg is not None else None, _ptr(gr), _ptr(pg), _ptr(gm))
    if rcode != 0:
        raise MemoryError("oracle_render failed")
    return dict(pix=pix, flags=flags, loss=float(loss[0]) if tg is not None else None, grad=gr,
                pose_grad=pg, grad_mag=gm)


def render_pixel(G, cam, pose, i, j, rc=None):
    """One pixel by testing every Gaussian: (values[9], flags)."""
    lib = _load()
    G = _f64(G, (-1, G_STRIDE))
    rc = raster_vec() if rc is None else _f64(rc)
    out = np.zeros(PX_STRIDE)
    fl = lib.oracle_render_pixel(G.shape[0], _ptr(G), _ptr(_f64(cam)), _ptr(_f64(pose, (12,))), _ptr(rc),
                                 int(i), int(j), _ptr(out))
    return out, fl


def render_jac(G, cam, pose, targets, rc=None, lc=None, delta=0.01):
    """Forward-mode pose Jacobian of one view and the IRLS normal equations
    of the MP-weighted L1 loss (w(u) held constant):
      J[u, ch, k] = d(rendered channel ch at pixel u) / d xi_k, ch = r, g, b,
                    depth; xi = (rho, phi), left perturbation
      W = c / max(|r|, delta), H = sum W J J^T, g = sum W r J, L the loss.
    Returns dict(pix, J (H*W x 4 x 6), flags, L, H (6 x 6), g (6,))."""
    lib = _load()
    G = _f64(G, (-1, G_STRIDE))
    rc = raster_vec() if rc is None else _f64(rc)
    lc = loss_vec() if lc is None else _f64(lc)
    cam = _f64(cam)
    W, H = int(cam[4]), int(cam[5])
    pix = np.zeros((W * H, PX_STRIDE))
    J = np.zeros((W * H, 4, 6))
    flags = np.zeros(W * H, np.int32)
    normal = np.zeros(28)
    tg = _f64(targets, (W * H, 4))
    rcode = lib.oracle_render_jac(G.shape[0], _ptr(G), _ptr(cam), _ptr(_f64(pose, (12,))), _ptr(rc), _ptr(lc),
                                  _ptr(tg), float(delta), _ptr(pix), _ptr(J), _ptr(flags), _ptr(normal))
    if rcode != 0:
        raise MemoryError("oracle_render_jac failed")
    Hm, g = unpack_normal(normal)
    return dict(pix=pix, J=J, flags=flags, L=float(normal[0]), H=Hm, g=g, normal=normal)


def unpack_normal(normal):
    """(H 6x6 symmetric, g 6) from the packed (L, upper triangle of H, g)."""
    normal = np.asarray(normal, np.float64)
    Hm = np.zeros((6, 6))
    e = 1
    for k in range(6):
        for m in range(k, 6):
            Hm[k, m] = Hm[m, k] = normal[e]
            e += 1
    return Hm, normal[22:28].copy()
