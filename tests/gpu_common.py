"""Helpers shared by the GPU parity tests: run a scene through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle

# Tolerances against the FP64 oracle.
#  Rendered colour, depth, opacity and composited MP (planes 0-5) are sums of
#  non-negative terms alpha_k T_k x_k. The kernels take each pixel offset as
#  (u_hi - px) + u_lo from the FP64 centre, so the offsets carry a rounding of
#  2^-24 of themselves; the remaining FP32 error per alpha is a few 1e-7
#  (conic, exp2), and a sum of non-negative terms keeps that relative error:
#  elementwise rtol 1e-5, with an absolute floor of 1e-7 of the channel's
#  largest value for pixels whose value is itself at that level.
IMG_RTOL, IMG_ATOL, IMG_NORM = 1e-5, 1e-7, 1e-5
# The final transmittance (plane 6) is a product of (1 - alpha_k): its
# relative error is sum_k alpha_k / (1 - alpha_k) times each alpha's relative
# error, up to ~50x behind a layer at alpha = 0.98, so elementwise 1e-4 and
# normwise 1e-5. The static weight w = (O - R_MP) / O (plane 7) lies in
# [0, 1] and loses digits to cancellation where R_MP ~ O: absolute 1e-5.
T_RTOL, T_NORM = 1e-4, 1e-5
W_ATOL = 1e-5
GRAD_NORM = 1e-4          # per parameter group, L2, relative
# Elementwise, on every entry above GRAD_FLOOR of its group's largest
# magnitude: |g_gpu - g| <= GRAD_ELEM |g| + GRAD_KAPPA M, with M the oracle's
# magnitude of the terms the entry sums (grad_mag: sum over pixels and 2D
# words of |term| |d param / d word|). The FP32 path rounds each pixel term
# (about 15 operations), each 2D-gradient sum (the warp's shuffle tree and
# the atomics across warps and tiles) and the chain to the parameter (about
# 30 operations) relatively, so its error is a few tens of 2^-24 times M,
# whatever the cancellation: where the terms do not cancel (M ~ |g|) the
# bound is the stated 1e-4 relative; where they cancel a hundredfold it
# grows with M, as any FP32 evaluation of the sum must. kappa = 4e-6 (67 ulp
# of M): the largest excess over every parity test was 2.2e-6 M, on one
# quaternion entry of the 1M-Gaussian 1200x680 frame.
GRAD_ELEM = 1e-4
GRAD_KAPPA = 4e-6
GRAD_FLOOR = 1e-3
POSE_REL = 1e-4           # pose twist gradient, L2, relative
LOSS_REL = 1e-5


def to_dev(sc, torch, dev="cuda"):
    gauss = torch.from_numpy(np.ascontiguousarray(sc.records)).to(dev)
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).to(dev)
    targets = torch.from_numpy(np.ascontiguousarray(sc.targets)).to(dev)
    return gauss, poses, targets


def image_rows(image_v):
    """(8, H, W) device tensor -> (H*W, 8) float64 numpy."""
    return image_v.permute(1, 2, 0).reshape(-1, image_v.shape[0]).double().cpu().numpy()


GRAD_MASK_FLAGS = oracle.PIXEL_DECISION_FLAGS | oracle.FLAGS["SIGN"]


def mask_flagged_targets(sc, lc=None):
    """Copy of the scene whose flagged pixels (a decision or a residual sign
    within FP32 error of its threshold) are left out of the loss (r < 0), so
    that gradients compare only what both sides decide identically."""
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    tg = sc.targets.copy()
    masked = 0
    for v in range(sc.poses.shape[0]):
        r = oracle.render(G, cam, sc.poses[v], lc=lc, targets=sc.targets[v])
        bad = (r["flags"] & GRAD_MASK_FLAGS) != 0
        tg[v, bad, 0] = -1.0
        masked += int(bad.sum())
    from paper_2602_21644_gb300 import synth
    return synth.Scene(sc.records, sc.camera, sc.poses, tg, sc.dynamic, sc.extra), masked


def oracle_views(sc, grads=True, lc=None):
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    outs = [oracle.render(G, cam, sc.poses[v], lc=lc, targets=sc.targets[v], grads=grads, grad_mag=grads)
            for v in range(sc.poses.shape[0])]
    return G, cam, outs


# A pixel whose decision is within FP32 error of a threshold may include or
# drop one near-threshold contribution (alpha ~ 1/255, or the tail after
# T ~ 1e-4): its values must still lie within that much of the oracle's.
FLAGGED_ABS = 0.01


def compare_image(img, ref_pix, flags, report=None, label=""):
    """img: (P, 8) GPU rows; ref_pix: (P, 10) oracle rows."""
    ok = (flags & oracle.PIXEL_DECISION_FLAGS) == 0
    if (~ok).any():
        fl = ~ok
        for c, rc in zip([0, 1, 2, 4, 5, 6], [0, 1, 2, 4, 5, 6]):
            d = np.abs(img[fl, c] - ref_pix[fl, rc]).max()
            assert d <= FLAGGED_ABS, f"{label}: flagged pixel channel {c} off by {d:.3e}"
        dz = np.abs(img[fl, 3] - ref_pix[fl, 3]) / np.maximum(1.0, np.abs(ref_pix[fl, 3]))
        assert dz.max() <= FLAGGED_ABS, f"{label}: flagged pixel depth off by {dz.max():.3e}"
        if report is not None:
            report.append(f"{label}: {int(fl.sum())} flagged pixels within the validity envelope")
    cols = [0, 1, 2, 3, 4, 5, 6, 7]
    refc = [0, 1, 2, 3, 4, 5, 6, 9]
    worst = {}
    for c, rc in zip(cols, refc):
        a, b = img[ok, c], ref_pix[ok, rc]
        err = np.abs(a - b)
        scale = np.abs(b).max() if b.size else 1.0
        if c == 6:
            tol = T_RTOL * np.abs(b) + IMG_ATOL * max(1.0, scale)
        elif c == 7:
            tol = np.full(b.shape, W_ATOL)
        else:
            tol = IMG_RTOL * np.abs(b) + IMG_ATOL * max(1.0, scale)
        bad = err > tol
        nrm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        rel = (err / np.maximum(np.abs(b), 1e-30))[np.abs(b) > 1e-3 * scale] if b.size else err
        worst[c] = (float(err.max()) if err.size else 0.0, float(nrm), int(bad.sum()))
        if report is not None:
            report.append(f"{label} ch{c}: max|d|={worst[c][0]:.3e} max rel(|v|>1e-3 max)="
                          f"{(rel.max() if rel.size else 0.0):.3e} norm={nrm:.3e} bad={int(bad.sum())}")
    return worst, int((~ok).sum())


GROUPS = {"mean": [0, 1, 2], "logit": [3], "quat": [4, 5, 6, 7], "logscale": [8, 9, 10], "colour": [12, 13, 14]}


def compare_grads(gg, ref_grad, report=None, mag=None, elementwise=True):
    """gg: (n, 16) GPU; ref_grad: (n, 15) oracle; mag: (n, 15) the oracle's
    grad_mag (for a sum over views, the sum of the views'). Returns the
    per-group relative L2 errors; with elementwise, also asserts on every
    entry above GRAD_FLOOR of its group's largest magnitude |d| <= GRAD_ELEM
    |g| + GRAD_KAPPA M (M = 0 without mag: the plain relative bound)."""
    out = {}
    fails = []
    for name, cols in GROUPS.items():
        a = gg[:, cols]
        b = ref_grad[:, cols]
        m = mag[:, cols] if mag is not None else np.zeros_like(b)
        nrm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        out[name] = float(nrm)
        big = np.abs(b) > GRAD_FLOOR * np.abs(b).max() if b.size else np.zeros(b.shape, bool)
        d = np.abs(a - b)[big]
        rel = d / np.abs(b)[big] if big.any() else np.zeros(0)
        ratio = d / (GRAD_ELEM * np.abs(b)[big] + GRAD_KAPPA * m[big]) if big.any() else np.zeros(0)
        el = float(rel.max()) if rel.size else 0.0
        worst = float(ratio.max()) if ratio.size else 0.0
        if report is not None:
            report.append(f"grad {name}: norm rel={nrm:.3e} elem rel (|g|>{GRAD_FLOOR:g}max)={el:.3e} "
                          f"(>{GRAD_ELEM:g}: {int((rel > GRAD_ELEM).sum())} of {int(big.sum())}), "
                          f"worst error / bound {worst:.3f}")
        if elementwise and worst > 1.0:
            fails.append(f"{name}: {int((ratio > 1).sum())} of {int(big.sum())} entries beyond "
                         f"{GRAD_ELEM:g}|g| + {GRAD_KAPPA:g}M (worst {worst:.2f}x, max rel {el:.3e})")
    assert not fails, "gradient elementwise: " + "; ".join(fails)
    return out
