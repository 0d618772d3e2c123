"""Helpers shared by the GPU parity tests: run a scene through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle

# Tolerances (derivation in the design notes, "Parity tolerances"):
#  FP32 pixel coordinates near x ~ W carry an absolute rounding of about
#  ulp(W) ~ 2^-24 W; at the alpha = 1/255 edge of a Gaussian whose smallest
#  2D std is ~0.55 px (0.3 px^2 dilation) that moves the exponent by up to
#  ~6 ulp(W) px / px, i.e. a relative alpha error up to ~1e-4 at W = 640.
#  Elementwise rendered values therefore get rtol 2e-4 with a small absolute
#  floor; the image as a whole (per channel, L2) must agree to 1e-5.
IMG_RTOL, IMG_ATOL, IMG_NORM = 2e-4, 2e-6, 1e-5
# The final transmittance is a product of (1 - alpha) factors: its relative
# error is the sum of alpha/(1 - alpha) times each alpha's relative error,
# up to ~1e-4 behind a few near-opaque layers; normwise it gets 1e-4.
T_NORM = 1e-4
GRAD_NORM = 1e-4          # per parameter group, L2, relative
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
    outs = [oracle.render(G, cam, sc.poses[v], lc=lc, targets=sc.targets[v], grads=grads)
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
        tol = IMG_RTOL * np.abs(b) + IMG_ATOL * max(1.0, scale)
        bad = err > tol
        nrm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        worst[c] = (float(err.max()) if err.size else 0.0, float(nrm), int(bad.sum()))
        if report is not None:
            report.append(f"{label} ch{c}: max|d|={worst[c][0]:.3e} norm={nrm:.3e} bad={int(bad.sum())}")
    return worst, int((~ok).sum())


GROUPS = {"mean": [0, 1, 2], "logit": [3], "quat": [4, 5, 6, 7], "logscale": [8, 9, 10], "colour": [12, 13, 14]}


def compare_grads(gg, ref_grad, report=None):
    """gg: (n, 16) GPU; ref_grad: (n, 15) oracle. Per-group relative L2."""
    out = {}
    for name, cols in GROUPS.items():
        a = gg[:, cols]
        b = ref_grad[:, cols]
        nrm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        out[name] = float(nrm)
        if report is not None:
            big = np.abs(b) > 1e-3 * np.abs(b).max()
            el = (np.abs(a - b)[big] / np.abs(b)[big]).max() if big.any() else 0.0
            report.append(f"grad {name}: norm rel={nrm:.3e} elem rel (|g|>1e-3max)={el:.3e}")
    return out
