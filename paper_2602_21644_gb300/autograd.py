"""torch.autograd wrappers of the splatting path: SplatLoss, whose forward
kernels render and reduce the MP-weighted loss of Eqs. (20)-(22), and
SplatRender, which returns the rendered channels for a caller's own loss; the
hand-written adjoint kernels give the gradients with respect to the Gaussian
records and to the camera poses. No arithmetic of the path runs here: both directions call the
library through the C ABI.

Pose gradient convention: the poses are world-to-camera T_CW (V x 12
doubles); their gradient is taken with respect to a left-perturbation twist
xi = (rho, phi) applied as T <- exp(xi^) T, evaluated at xi = 0. The twist is
therefore an explicit input that must be zero when the loss is evaluated
(pose_step applies a step and folds it back into T).
"""
from __future__ import annotations

import torch

from . import dags


class SplatLoss(torch.autograd.Function):
    """loss = SplatLoss.apply(gauss, xi, ctx, cam, poses, targets, rcfg, lcfg)

    gauss   [N, 16] float32 CUDA records (gradient: same slots, see dags.h)
    xi      [V, 6] float64 CUDA twist, all zero (gradient: dL/dxi)
    ctx     dags.Context; cam dags.Camera; poses [V, 12] float64 CUDA
    targets [V, H*W, 4] float32 CUDA; rcfg / lcfg optional configs
    Returns the loss as a [1] float64 tensor."""

    @staticmethod
    def forward(fctx, gauss, xi, ctx, cam, poses, targets, rcfg=None, lcfg=None):
        image, last, loss = ctx.forward(gauss, cam, poses, targets, rcfg=rcfg, lcfg=lcfg)
        fctx.save_for_backward(gauss, poses, targets, image, last)
        fctx.dags_ctx, fctx.cam, fctx.rcfg, fctx.lcfg = ctx, cam, rcfg, lcfg
        return loss

    @staticmethod
    def backward(fctx, gloss):
        gauss, poses, targets, image, last = fctx.saved_tensors
        flags = 0
        if fctx.needs_input_grad[0]:
            flags |= dags.GRAD_GAUSS
        if fctx.needs_input_grad[1]:
            flags |= dags.GRAD_POSE
        gg = gp = None
        if flags:
            gg, gp = fctx.dags_ctx.backward(gauss, fctx.cam, poses, targets, image, last, flags=flags,
                                            rcfg=fctx.rcfg, lcfg=fctx.lcfg)
        s = gloss.reshape(())
        if gg is not None:
            gg = gg * s.to(gg.dtype)
        if gp is not None:
            gp = gp * s
        return gg, gp, None, None, None, None, None, None


class SplatRender(torch.autograd.Function):
    """C, D, O, R_MP = SplatRender.apply(gauss, xi, ctx, cam, poses, rcfg)

    The rendered channels themselves, for a caller's own loss: C [V, 3, H, W],
    D, O and R_MP [V, H, W] float32. Their gradients go back through the
    library's adjoint (splat_backward_upstream) to the records and the pose
    twist xi ([V, 6] float64, all zero)."""

    @staticmethod
    def forward(fctx, gauss, xi, ctx, cam, poses, rcfg=None):
        image, last, _ = ctx.forward(gauss, cam, poses, None, rcfg=rcfg)
        fctx.save_for_backward(gauss, poses, image, last)
        fctx.dags_ctx, fctx.cam, fctx.rcfg = ctx, cam, rcfg
        fctx.mark_non_differentiable(last)
        return image[:, 0:3], image[:, 3], image[:, 4], image[:, 5]

    @staticmethod
    def backward(fctx, gC, gD, gO, gR):
        gauss, poses, image, last = fctx.saved_tensors
        V, _, H, W = image.shape
        up = torch.zeros((V, 6, H, W), dtype=torch.float32, device=image.device)
        if gC is not None:
            up[:, 0:3] = gC
        for k, g in ((3, gD), (4, gO), (5, gR)):
            if g is not None:
                up[:, k] = g
        flags = 0
        if fctx.needs_input_grad[0]:
            flags |= dags.GRAD_GAUSS
        if fctx.needs_input_grad[1]:
            flags |= dags.GRAD_POSE
        gg = gp = None
        if flags:
            gg, gp = fctx.dags_ctx.backward_upstream(gauss, fctx.cam, poses, image, last, up, flags=flags,
                                                     rcfg=fctx.rcfg)
        return gg, gp, None, None, None, None


def splat_render(ctx, cam, gauss, poses, xi=None, rcfg=None):
    """Differentiable rendering: returns (C, D, O, R_MP); pass xi (zeros,
    requires_grad) to get the pose-twist gradient of a loss on them."""
    if xi is None:
        xi = torch.zeros((poses.shape[0], 6), dtype=torch.float64, device=poses.device)
    return SplatRender.apply(gauss, xi, ctx, cam, poses, rcfg)


def splat_loss(ctx, cam, gauss, poses, targets, xi=None, rcfg=None, lcfg=None):
    """Differentiable MP-weighted loss; pass xi (zeros, requires_grad) to get
    the pose-twist gradient."""
    if xi is None:
        xi = torch.zeros((poses.shape[0], 6), dtype=torch.float64, device=poses.device)
    return SplatLoss.apply(gauss, xi, ctx, cam, poses, targets, rcfg, lcfg)


class MPConsistency(torch.autograd.Function):
    """loss = MPConsistency.apply(gauss, ctx, prev, lam, rel_pose)

    lambda * L_MP of Eqs. (23), (24) over all Gaussians, with its gradient
    with respect to the means (record words 0-2; the MP word is held
    constant). prev: the records after the previous mapping update. Returns a
    [1] float64 tensor."""

    @staticmethod
    def forward(fctx, gauss, ctx, prev, lam, rel_pose=None):
        loss = ctx.mp_consistency(gauss, prev, lam, rel_pose=rel_pose)
        fctx.save_for_backward(gauss, prev)
        fctx.dags_ctx, fctx.lam, fctx.rel_pose = ctx, lam, rel_pose
        return loss

    @staticmethod
    def backward(fctx, gloss):
        gauss, prev = fctx.saved_tensors
        grad = torch.zeros_like(gauss)
        fctx.dags_ctx.mp_consistency(gauss, prev, fctx.lam, rel_pose=fctx.rel_pose, grad=grad, want_loss=False)
        return grad * gloss.reshape(()).to(grad.dtype), None, None, None, None


def mp_consistency(ctx, gauss, prev, lam=500.0, rel_pose=None):
    """Differentiable lambda * L_MP (Sec. IV-D): add it to splat_loss's value
    for the mapping objective of Eq. (27)."""
    return MPConsistency.apply(gauss, ctx, prev, lam, rel_pose)
