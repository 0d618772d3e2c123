"""Thin ctypes binding of libdags.so (C ABI in include/dags.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Tensors are torch CUDA tensors; their data pointers and torch's
current CUDA stream are handed to the C entry points. If the library is
missing this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdags.so")

IMG_CHANNELS = 8
GRAD_WORDS = 16
RECORD_WORDS = 16
GRAD_GAUSS = 1
GRAD_POSE = 2

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "pair capacity exceeded",
          -4: "device wait timed out", -5: "workspace allocation failed",
          -6: "backward does not follow its forward", -7: "index check failed (DAGS_CHECK build)"}


class DagsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class CCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class CRasterCfg(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("dilation", ctypes.c_float), ("z_near", ctypes.c_float),
                ("guard", ctypes.c_float)]


class CLossCfg(ctypes.Structure):
    _fields_ = [("lambda_pho", ctypes.c_float), ("lambda_depth", ctypes.c_float), ("weight_mode", ctypes.c_int32),
                ("weight_grad", ctypes.c_int32), ("o_eps", ctypes.c_float)]


class CMpCfg(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("kappa_c", "lam", "sigma_min", "e_floor", "sigma_g", "sigma_c",
                                              "lam_u", "eps", "alpha_min", "alpha_max", "rho", "r_s", "sigma_w",
                                              "vis_tol", "z_near", "tau_floor")] + [("fusion_mode", ctypes.c_int32),
                                                                                    ("scales", ctypes.c_int32)]


class CSchedCfg(ctypes.Structure):
    _fields_ = [("w_u", ctypes.c_double), ("w_r", ctypes.c_double), ("theta", ctypes.c_double),
                ("e_ref", ctypes.c_double), ("n_max", ctypes.c_int32)]


class CEdgeCfg(ctypes.Structure):
    _fields_ = [("edge_rel", ctypes.c_float), ("huber", ctypes.c_float), ("z_near", ctypes.c_float),
                ("literal", ctypes.c_int32)]


class CLmCfg(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("mu0", "mu_min", "mu_max", "down", "up", "delta", "floor")]


LM_NORMAL = 28
LM_STATE = 48
MP_STATS_HEAD = 6
MPNET_WEIGHT_BYTES = 22016
MPNET_ACT_WORDS = 96
MPNET_PARAMS = 10881


class CGaussAdamCfg(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("lr_mean", "lr_opacity", "lr_quat", "lr_scale", "lr_colour", "beta1",
                                              "beta2", "eps")]


class CPoseCfg(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double * 6), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


EXPORTS = ["dags_create", "dags_destroy", "dags_status_string", "dags_abi_version", "dags_sync_status",
           "dags_default_raster_cfg", "dags_default_loss_cfg", "dags_default_pose_cfg", "splat_forward",
           "splat_backward", "pose_step", "dags_copy_bins", "dags_timing_enable", "dags_timing_read",
           "splat_track", "splat_forward_static", "dags_default_mp_cfg", "mp_update", "mpnet_features", "mpnet_infer",
           "mpnet_train_step", "dags_selftest_timeout", "dags_default_sched_cfg", "semantic_trigger",
           "dags_default_lm_cfg", "splat_normal_equations", "lm_init", "lm_pose_step", "splat_track_lm",
           "splat_mp_consistency", "dags_default_edge_cfg", "splat_edge_warp",
           "epipolar_verify", "dags_eval_counting", "dags_eval_read", "dags_measure_alu", "dags_measure_mma",
           "splat_backward_upstream", "dags_default_gauss_adam_cfg", "gauss_adam_init", "gauss_adam_step"]

KERNELS = ["preprocess", "emit", "tile_sort", "render_fwd", "render_bwd", "preprocess_bwd", "pose_step",
           "mp_pixel", "mp_gauss", "mpnet", "mpnet_train", "pose_tangent", "render_jac", "lm_step",
           "regulariser", "epipolar", "gauss_adam"]

_lib = None


def measure_alu(kind: int, iters: int = 1 << 14):
    """Measured lane operations per second of the current device's FP32 FMA
    (kind 0) or ex2.approx (kind 1) pipe, and the timed launch's ms."""
    lib = load()
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.dags_measure_alu(int(kind), int(iters), ctypes.byref(ops), ctypes.byref(ms)), "dags_measure_alu")
    return ops.value, ms.value


def measure_mma(n_cols: int, groups: int, reps: int = 256, m_rows: int = 128):
    """Measured tensor-core rate (multiply-adds per SM cycle) of back-to-back
    M = m_rows, N = n_cols, K = 16 BF16 MMAs issued by `groups` warpgroups of
    one CTA, and the issue cycles per MMA of one issuing thread."""
    lib = load()
    mac, cyc = ctypes.c_double(), ctypes.c_double()
    _check(lib.dags_measure_mma(int(m_rows), int(n_cols), int(groups), int(reps), ctypes.byref(mac),
                                ctypes.byref(cyc)), "dags_measure_mma")
    return mac.value, cyc.value


def load(path: str = LIB_PATH):
    """Load libdags.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdags.so not found at {path}; build it with "
                           "`python -m paper_2602_21644_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.dags_create.argtypes = [ctypes.POINTER(P), I64, I32, I32, I32, I64]
    lib.dags_create.restype = ctypes.c_int
    lib.dags_destroy.argtypes = [P]
    lib.dags_destroy.restype = None
    lib.dags_status_string.argtypes = [ctypes.c_int]
    lib.dags_status_string.restype = ctypes.c_char_p
    lib.dags_abi_version.argtypes = []
    lib.dags_abi_version.restype = ctypes.c_int
    lib.dags_sync_status.argtypes = [P, ctypes.POINTER(I64)]
    lib.dags_sync_status.restype = ctypes.c_int
    lib.dags_default_raster_cfg.argtypes = [ctypes.POINTER(CRasterCfg)]
    lib.dags_default_loss_cfg.argtypes = [ctypes.POINTER(CLossCfg)]
    lib.dags_default_pose_cfg.argtypes = [ctypes.POINTER(CPoseCfg)]
    lib.splat_forward.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, I32, P, ctypes.POINTER(CRasterCfg),
                                  ctypes.POINTER(CLossCfg), P, P, P, P]
    lib.splat_forward.restype = ctypes.c_int
    lib.splat_backward.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, I32, P, ctypes.POINTER(CRasterCfg),
                                   ctypes.POINTER(CLossCfg), P, P, U32, P, P, P]
    lib.splat_backward.restype = ctypes.c_int
    lib.splat_backward_upstream.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, I32,
                                            ctypes.POINTER(CRasterCfg), P, P, P, U32, P, P, P]
    lib.splat_backward_upstream.restype = ctypes.c_int
    lib.dags_default_gauss_adam_cfg.argtypes = [ctypes.POINTER(CGaussAdamCfg)]
    lib.dags_default_gauss_adam_cfg.restype = None
    lib.gauss_adam_init.argtypes = [P, P, I64, P, P, P, P]
    lib.gauss_adam_init.restype = ctypes.c_int
    lib.gauss_adam_step.argtypes = [P, P, I64, P, P, P, P, I64, ctypes.POINTER(CGaussAdamCfg), P]
    lib.gauss_adam_step.restype = ctypes.c_int
    lib.pose_step.argtypes = [P, P, P, P, I32, ctypes.POINTER(CPoseCfg), P]
    lib.pose_step.restype = ctypes.c_int
    lib.dags_copy_bins.argtypes = [P, P, I64, P, I64, ctypes.POINTER(I64)]
    lib.dags_copy_bins.restype = ctypes.c_int
    lib.dags_timing_enable.argtypes = [P, ctypes.c_int]
    lib.dags_timing_enable.restype = ctypes.c_int
    lib.dags_timing_read.argtypes = [P, P, P, I32]
    lib.dags_timing_read.restype = ctypes.c_int
    lib.dags_eval_counting.argtypes = [P, I32]
    lib.dags_eval_counting.restype = ctypes.c_int
    lib.dags_eval_read.argtypes = [P, P]
    lib.dags_eval_read.restype = ctypes.c_int
    lib.dags_measure_alu.argtypes = [I32, I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.dags_measure_alu.restype = ctypes.c_int
    lib.dags_measure_mma.argtypes = [I32, I32, I32, I32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.dags_measure_mma.restype = ctypes.c_int
    lib.splat_track.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, P, ctypes.POINTER(CRasterCfg),
                                ctypes.POINTER(CLossCfg), ctypes.POINTER(CPoseCfg), I32, P, P, P, P, P, I32, P]
    lib.splat_track.restype = ctypes.c_int
    lib.splat_forward_static.argtypes = [P, I64, ctypes.POINTER(CCamera), P, P, ctypes.POINTER(CRasterCfg),
                                         ctypes.POINTER(CLossCfg), P, P, P, P, P]
    lib.splat_forward_static.restype = ctypes.c_int
    lib.dags_default_mp_cfg.argtypes = [ctypes.POINTER(CMpCfg)]
    lib.mp_update.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, P, P, P, P, I32, ctypes.POINTER(CMpCfg), I32, P,
                              P, P, P, P]
    lib.mpnet_features.argtypes = [P, P, P, P, P, I32, I32, I32, P, P]
    lib.mpnet_features.restype = ctypes.c_int
    lib.mp_update.restype = ctypes.c_int
    lib.mpnet_infer.argtypes = [P, P, P, I32, I32, I32, P, P, P]
    lib.mpnet_infer.restype = ctypes.c_int
    lib.mpnet_train_step.argtypes = [P, P, P, P, P, I32, P, P, I32, I32, I32, ctypes.c_float, P, P, P]
    lib.mpnet_train_step.restype = ctypes.c_int
    lib.dags_selftest_timeout.argtypes = [P, I64, P]
    lib.dags_default_sched_cfg.argtypes = [ctypes.POINTER(CSchedCfg)]
    lib.dags_default_sched_cfg.restype = None
    lib.semantic_trigger.argtypes = [P, P, ctypes.POINTER(CSchedCfg), I32, P, P, P]
    lib.semantic_trigger.restype = ctypes.c_int
    lib.dags_default_lm_cfg.argtypes = [ctypes.POINTER(CLmCfg)]
    lib.dags_default_lm_cfg.restype = None
    lib.splat_normal_equations.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, P, ctypes.POINTER(CRasterCfg),
                                           ctypes.POINTER(CLossCfg), ctypes.c_double, P, P, P, P, P]
    lib.splat_normal_equations.restype = ctypes.c_int
    lib.lm_init.argtypes = [P, P, ctypes.POINTER(CLmCfg), P, P, P]
    lib.lm_init.restype = ctypes.c_int
    lib.lm_pose_step.argtypes = [P, P, ctypes.POINTER(CLmCfg), P, P, P, P]
    lib.lm_pose_step.restype = ctypes.c_int
    lib.splat_track_lm.argtypes = [P, P, I64, ctypes.POINTER(CCamera), P, P, ctypes.POINTER(CRasterCfg),
                                   ctypes.POINTER(CLossCfg), ctypes.POINTER(CLmCfg), I32, P, I32, P]
    lib.splat_track_lm.restype = ctypes.c_int
    lib.splat_mp_consistency.argtypes = [P, P, I64, P, P, ctypes.c_float, P, P, P]
    lib.splat_mp_consistency.restype = ctypes.c_int
    lib.dags_default_edge_cfg.argtypes = [ctypes.POINTER(CEdgeCfg)]
    lib.dags_default_edge_cfg.restype = None
    lib.splat_edge_warp.argtypes = [P, ctypes.POINTER(CCamera), P, P, P, P, P, ctypes.POINTER(CEdgeCfg),
                                    ctypes.c_float, P, P]
    lib.splat_edge_warp.restype = ctypes.c_int
    lib.epipolar_verify.argtypes = [P, ctypes.POINTER(CCamera), P, P, P, P, P, I64, P, I64, P, ctypes.c_float,
                                    ctypes.c_float, P, P, P]
    lib.epipolar_verify.restype = ctypes.c_int
    lib.dags_selftest_timeout.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise DagsError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def c(self) -> CCamera:
        return CCamera(self.fx, self.fy, self.cx, self.cy, self.width, self.height)


def default_raster_cfg() -> CRasterCfg:
    c = CRasterCfg()
    load().dags_default_raster_cfg(ctypes.byref(c))
    return c


def default_loss_cfg(**kw) -> CLossCfg:
    c = CLossCfg()
    load().dags_default_loss_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_pose_cfg(lr=None, **kw) -> CPoseCfg:
    c = CPoseCfg()
    load().dags_default_pose_cfg(ctypes.byref(c))
    if lr is not None:
        for k in range(6):
            c.lr[k] = float(lr[k] if hasattr(lr, "__len__") else lr)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_gauss_adam_cfg(**kw) -> CGaussAdamCfg:
    c = CGaussAdamCfg()
    load().dags_default_gauss_adam_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_mp_cfg(**kw) -> CMpCfg:
    c = CMpCfg()
    load().dags_default_mp_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_sched_cfg(**kw) -> CSchedCfg:
    c = CSchedCfg()
    load().dags_default_sched_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_edge_cfg(**kw) -> CEdgeCfg:
    c = CEdgeCfg()
    load().dags_default_edge_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def default_lm_cfg(**kw) -> CLmCfg:
    c = CLmCfg()
    load().dags_default_lm_cfg(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _need(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


class Context:
    """Owns a dags_ctx (device workspace) on the current CUDA device."""

    def __init__(self, max_gaussians: int, max_width: int, max_height: int, max_views: int = 1,
                 max_pairs: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.dags_create(ctypes.byref(h), int(max_gaussians), int(max_width), int(max_height),
                                    int(max_views), int(max_pairs)), "dags_create")
        self.h = h
        self.max = (max_gaussians, max_width, max_height, max_views)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dags_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self):
        """(status_code, required_pairs); synchronises the last stream."""
        req = ctypes.c_int64(0)
        code = self.lib.dags_sync_status(self.h, ctypes.byref(req))
        return code, req.value

    def check(self):
        code, req = self.sync_status()
        if code != 0:
            raise DagsError(code, f"device status (required pairs {req})")

    def timing(self, enable: bool):
        _check(self.lib.dags_timing_enable(self.h, int(bool(enable))), "dags_timing_enable")

    def timing_read(self):
        """{kernel: (total_ms, launches)} accumulated since the last read."""
        import numpy as np
        k = len(KERNELS)
        ms = np.zeros(k, np.float64)
        n = np.zeros(k, np.int64)
        _check(self.lib.dags_timing_read(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                         n.ctypes.data_as(ctypes.c_void_p), k), "dags_timing_read")
        return {KERNELS[i]: (float(ms[i]), int(n[i])) for i in range(k)}

    def eval_counting(self, enable: bool):
        """Count the compositing kernels' evaluations (see eval_read)."""
        _check(self.lib.dags_eval_counting(self.h, int(bool(enable))), "dags_eval_counting")

    def eval_read(self):
        """{fwd_eval, fwd_contrib, bwd_eval, bwd_contrib} accumulated since the last read."""
        import numpy as np
        c = np.zeros(4, np.int64)
        _check(self.lib.dags_eval_read(self.h, c.ctypes.data_as(ctypes.c_void_p)), "dags_eval_read")
        return dict(zip(("fwd_eval", "fwd_contrib", "bwd_eval", "bwd_contrib"), (int(x) for x in c)))

    def copy_bins(self, views: int, cam: Camera):
        """(tile_start [views*T+1] uint32, ids [pairs] uint32) of the last forward."""
        import numpy as np
        T = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
        start = np.zeros(views * T + 1, np.uint32)
        npairs = ctypes.c_int64(0)
        _check(self.lib.dags_copy_bins(self.h, start.ctypes.data_as(ctypes.c_void_p), start.size, None, 0,
                                       ctypes.byref(npairs)), "dags_copy_bins")
        ids = np.zeros(max(1, npairs.value), np.uint32)
        _check(self.lib.dags_copy_bins(self.h, start.ctypes.data_as(ctypes.c_void_p), start.size,
                                       ids.ctypes.data_as(ctypes.c_void_p), ids.size, ctypes.byref(npairs)),
               "dags_copy_bins")
        return start, ids[:npairs.value]

    # ------------------------------------------------------------ splatting

    def forward(self, gauss, cam: Camera, poses, targets=None, rcfg=None, lcfg=None, image=None, last=None,
                loss=None, want_loss=True):
        """Returns (image [V,8,H,W] f32, last [V,H,W] i32, loss [1] f64 or None)."""
        _need(gauss, torch.float32, "gauss")
        _need(poses, torch.float64, "poses")
        n = gauss.shape[0]
        V = poses.shape[0]
        H, W = cam.height, cam.width
        dev = gauss.device
        if targets is not None:
            _need(targets, torch.float32, "targets")
        if image is None:
            image = torch.empty((V, IMG_CHANNELS, H, W), dtype=torch.float32, device=dev)
        if last is None:
            last = torch.empty((V, H, W), dtype=torch.int32, device=dev)
        if loss is None and targets is not None and want_loss:
            loss = torch.empty(1, dtype=torch.float64, device=dev)
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        lc = lcfg if lcfg is not None else default_loss_cfg()
        _check(self.lib.splat_forward(self.h, _ptr(gauss), n, ctypes.byref(c), _ptr(poses), V, _ptr(targets),
                                      ctypes.byref(rc), ctypes.byref(lc), _ptr(image), _ptr(last),
                                      _ptr(loss if targets is not None else None), _stream()), "splat_forward")
        return image, last, loss

    def backward(self, gauss, cam: Camera, poses, targets, image, last, flags=GRAD_POSE, rcfg=None, lcfg=None,
                 grad_gauss=None, grad_pose=None):
        """Returns (grad_gauss [n,16] f32 or None, grad_pose [V,6] f64 or None)."""
        n = gauss.shape[0]
        V = poses.shape[0]
        dev = gauss.device
        if flags & GRAD_GAUSS and grad_gauss is None:
            grad_gauss = torch.empty((n, GRAD_WORDS), dtype=torch.float32, device=dev)
        if flags & GRAD_POSE and grad_pose is None:
            grad_pose = torch.empty((V, 6), dtype=torch.float64, device=dev)
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        lc = lcfg if lcfg is not None else default_loss_cfg()
        _check(self.lib.splat_backward(self.h, _ptr(gauss), n, ctypes.byref(c), _ptr(poses), V, _ptr(targets),
                                       ctypes.byref(rc), ctypes.byref(lc), _ptr(image), _ptr(last), int(flags),
                                       _ptr(grad_gauss if flags & GRAD_GAUSS else None),
                                       _ptr(grad_pose if flags & GRAD_POSE else None), _stream()), "splat_backward")
        return (grad_gauss if flags & GRAD_GAUSS else None), (grad_pose if flags & GRAD_POSE else None)

    def gauss_adam_state(self, gauss):
        """(colour master [n,4] f32, m [n,16], v [n,16]) initialised for gauss_adam_step."""
        n = gauss.shape[0]
        dev = gauss.device
        colour = torch.empty((n, 4), dtype=torch.float32, device=dev)
        m = torch.empty((n, GRAD_WORDS), dtype=torch.float32, device=dev)
        v = torch.empty((n, GRAD_WORDS), dtype=torch.float32, device=dev)
        _check(self.lib.gauss_adam_init(self.h, _ptr(gauss), n, _ptr(colour), _ptr(m), _ptr(v), _stream()),
               "gauss_adam_init")
        return colour, m, v

    def gauss_adam_step(self, gauss, state, grad, step, cfg=None):
        """One Adam step (step >= 1) of the Gaussian parameters in place."""
        colour, m, v = state
        c = cfg if cfg is not None else default_gauss_adam_cfg()
        _check(self.lib.gauss_adam_step(self.h, _ptr(gauss), gauss.shape[0], _ptr(colour), _ptr(m), _ptr(v),
                                        _ptr(grad), int(step), ctypes.byref(c), _stream()), "gauss_adam_step")

    def backward_upstream(self, gauss, cam: Camera, poses, image, last, grad_image, flags=GRAD_POSE, rcfg=None,
                          grad_gauss=None, grad_pose=None):
        """Backward of a caller's function of the rendered channels: grad_image
        [V, 6, H, W] f32 holds its gradients with respect to image planes 0-5
        (C_r, C_g, C_b, D, O, R_MP). Returns (grad_gauss, grad_pose) as backward."""
        _need(grad_image, torch.float32, "grad_image")
        n = gauss.shape[0]
        V = poses.shape[0]
        if tuple(grad_image.shape) != (V, 6, cam.height, cam.width):
            raise ValueError(f"grad_image must be [{V}, 6, {cam.height}, {cam.width}]")
        dev = gauss.device
        if flags & GRAD_GAUSS and grad_gauss is None:
            grad_gauss = torch.empty((n, GRAD_WORDS), dtype=torch.float32, device=dev)
        if flags & GRAD_POSE and grad_pose is None:
            grad_pose = torch.empty((V, 6), dtype=torch.float64, device=dev)
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        _check(self.lib.splat_backward_upstream(self.h, _ptr(gauss), n, ctypes.byref(c), _ptr(poses), V,
                                                ctypes.byref(rc), _ptr(image), _ptr(last), _ptr(grad_image),
                                                int(flags), _ptr(grad_gauss if flags & GRAD_GAUSS else None),
                                                _ptr(grad_pose if flags & GRAD_POSE else None), _stream()),
               "splat_backward_upstream")
        return (grad_gauss if flags & GRAD_GAUSS else None), (grad_pose if flags & GRAD_POSE else None)

    def track(self, gauss, cam: Camera, pose, targets, iters, adam_state, image, last, loss, grad_pose,
              rcfg=None, lcfg=None, pcfg=None, use_graph=True):
        """iters tracking iterations (forward, pose backward, pose step) enqueued
        by the library; pose and adam_state are updated in place."""
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        lc = lcfg if lcfg is not None else default_loss_cfg()
        pc = pcfg if pcfg is not None else default_pose_cfg()
        _check(self.lib.splat_track(self.h, _ptr(gauss), gauss.shape[0], ctypes.byref(c), _ptr(pose), _ptr(targets),
                                    ctypes.byref(rc), ctypes.byref(lc), ctypes.byref(pc), int(iters),
                                    _ptr(adam_state), _ptr(image), _ptr(last), _ptr(loss), _ptr(grad_pose),
                                    int(bool(use_graph)), _stream()), "splat_track")

    def normal_equations(self, gauss, cam: Camera, pose, targets, delta=0.01, rcfg=None, lcfg=None, jac=False,
                         image=None, last=None, normal=None):
        """IRLS normal equations of the MP-weighted L1 loss at pose (Levenberg-
        Marquardt linearisation). Returns (normal float64 [28]: L, upper
        triangle of H, g; jac float32 [H*W, 4, 6] or None)."""
        _need(gauss, torch.float32, "gauss")
        _need(targets, torch.float32, "targets")
        _need(pose, torch.float64, "pose")
        dev = gauss.device
        if normal is None:
            normal = torch.empty(LM_NORMAL, dtype=torch.float64, device=dev)
        J = torch.empty((cam.width * cam.height, 4, 6), dtype=torch.float32, device=dev) if jac else None
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        lc = lcfg if lcfg is not None else default_loss_cfg()
        _check(self.lib.splat_normal_equations(self.h, _ptr(gauss), gauss.shape[0], ctypes.byref(c), _ptr(pose),
                                               _ptr(targets), ctypes.byref(rc), ctypes.byref(lc), float(delta),
                                               _ptr(normal), _ptr(J), _ptr(image), _ptr(last), _stream()),
               "splat_normal_equations")
        return normal, J

    def lm_init(self, pose, state, pose_try, cfg=None):
        lc = cfg if cfg is not None else default_lm_cfg()
        _check(self.lib.lm_init(self.h, _ptr(pose), ctypes.byref(lc), _ptr(state), _ptr(pose_try), _stream()),
               "lm_init")

    def lm_step(self, normal, state, pose_try, pose_best, cfg=None):
        """One LM decision and damped step (FP64) from the normal equations."""
        lc = cfg if cfg is not None else default_lm_cfg()
        _check(self.lib.lm_pose_step(self.h, _ptr(normal), ctypes.byref(lc), _ptr(state), _ptr(pose_try),
                                     _ptr(pose_best), _stream()), "lm_pose_step")

    def track_lm(self, gauss, cam: Camera, pose, targets, iters, state=None, cfg=None, rcfg=None, lcfg=None,
                 use_graph=True):
        """iters Levenberg-Marquardt iterations from pose (in place: the best
        pose). Returns the state tensor (float64 [48])."""
        _need(gauss, torch.float32, "gauss")
        _need(targets, torch.float32, "targets")
        _need(pose, torch.float64, "pose")
        if state is None:
            state = torch.empty(LM_STATE, dtype=torch.float64, device=gauss.device)
        c = cam.c()
        rc = rcfg if rcfg is not None else default_raster_cfg()
        lc = lcfg if lcfg is not None else default_loss_cfg()
        mc = cfg if cfg is not None else default_lm_cfg()
        _check(self.lib.splat_track_lm(self.h, _ptr(gauss), gauss.shape[0], ctypes.byref(c), _ptr(pose), _ptr(targets),
                                       ctypes.byref(rc), ctypes.byref(lc), ctypes.byref(mc), int(iters), _ptr(state),
                                       int(bool(use_graph)), _stream()), "splat_track_lm")
        return state

    def mp_consistency(self, gauss, prev, lam=500.0, rel_pose=None, grad=None, loss=None, want_loss=True):
        """MP motion-consistency regulariser lambda * L_MP (Eqs. (23), (24)).
        prev: the records after the previous mapping update (n x 16 float32).
        grad (n x 16 float32, optional) receives d/d mean added into words
        0-2. Returns the loss tensor (float64 [1]) or None."""
        _need(gauss, torch.float32, "gauss")
        _need(prev, torch.float32, "prev")
        if prev.shape != gauss.shape:
            raise ValueError("prev must have the records' shape")
        if grad is not None:
            _need(grad, torch.float32, "grad")
        if rel_pose is not None:
            _need(rel_pose, torch.float64, "rel_pose")
        if loss is None and want_loss:
            loss = torch.empty(1, dtype=torch.float64, device=gauss.device)
        _check(self.lib.splat_mp_consistency(self.h, _ptr(gauss), gauss.shape[0], _ptr(prev), _ptr(rel_pose),
                                             float(lam), _ptr(grad), _ptr(loss), _stream()), "splat_mp_consistency")
        return loss

    def edge_warp(self, cam: Camera, depth_i, depth_j, weight_j, pose_i, pose_j, lam=300.0, cfg=None, out=None):
        """Edge-warp regulariser from frame i to frame j (Eqs. (25), (26)).
        depth_*, weight_j: float32 [H*W] device tensors; poses float64 [12].
        Returns float64 [13]: lambda L_edge, d/d xi_i (6), d/d xi_j (6)."""
        for name, t in (("depth_i", depth_i), ("depth_j", depth_j), ("weight_j", weight_j)):
            _need(t, torch.float32, name)
            if t.numel() < cam.width * cam.height:
                raise ValueError(f"{name} must hold H*W floats")
        _need(pose_i, torch.float64, "pose_i")
        _need(pose_j, torch.float64, "pose_j")
        if out is None:
            out = torch.empty(13, dtype=torch.float64, device=depth_i.device)
        c = cam.c()
        ec = cfg if cfg is not None else default_edge_cfg()
        _check(self.lib.splat_edge_warp(self.h, ctypes.byref(c), _ptr(depth_i), _ptr(depth_j), _ptr(weight_j),
                                        _ptr(pose_i), _ptr(pose_j), ctypes.byref(ec), float(lam), _ptr(out),
                                        _stream()), "splat_edge_warp")
        return out

    def epipolar_verify(self, cam: Camera, pose_1, pose_2, p1, p2, gid, gauss, labels, eps=1.0, m_static=0.1,
                        want_d=True, want_dbar=True):
        """Epipolar verification and static recovery (Eqs. (18), (19)); gauss's
        MP words and labels are updated in place. p1, p2: float32 [m, 2];
        gid: int32 [m]. Returns (d float32 [m] or None, dbar float32 [n] or None)."""
        _need(gauss, torch.float32, "gauss")
        _need(labels, torch.uint8, "labels")
        _need(pose_1, torch.float64, "pose_1")
        _need(pose_2, torch.float64, "pose_2")
        m = int(gid.shape[0])
        if m:
            _need(p1, torch.float32, "p1")
            _need(p2, torch.float32, "p2")
            _need(gid, torch.int32, "gid")
        dev = gauss.device
        d = torch.empty(m, dtype=torch.float32, device=dev) if want_d else None
        dbar = torch.empty(gauss.shape[0], dtype=torch.float32, device=dev) if want_dbar else None
        c = cam.c()
        _check(self.lib.epipolar_verify(self.h, ctypes.byref(c), _ptr(pose_1), _ptr(pose_2), _ptr(p1) if m else None,
                                        _ptr(p2) if m else None, _ptr(gid) if m else None, m, _ptr(gauss),
                                        gauss.shape[0], _ptr(labels), float(eps), float(m_static), _ptr(d), _ptr(dbar),
                                        _stream()), "epipolar_verify")
        return d, dbar

    def mp_update(self, gauss, cam: Camera, pose, targets, image, inst, table, labels, cfg=None, seg_refreshed=True,
                  stats=None, mp_map=None, mp_pixel=None):
        """Spatiotemporal MP update of one view; gauss's MP words and labels are
        updated in place. mp_map (float32 [H*W], optional) replaces the fused
        per-pixel M_p in the association; mp_pixel (float32 [H*W], optional)
        receives the fused M_p. Returns the stats tensor (float64)."""
        for name, t in (("mp_map", mp_map), ("mp_pixel", mp_pixel)):
            if t is not None:
                _need(t, torch.float32, name)
                if t.numel() != cam.width * cam.height:
                    raise ValueError(f"{name} must hold H*W floats")
        _need(gauss, torch.float32, "gauss")
        _need(inst, torch.uint8, "inst")
        _need(labels, torch.uint8, "labels")
        _need(table, torch.float32, "table")
        nreg = table.shape[0]
        if stats is None:
            stats = torch.empty(MP_STATS_HEAD + 4 * nreg, dtype=torch.float64, device=gauss.device)
        c = cam.c()
        mc = cfg if cfg is not None else default_mp_cfg()
        _check(self.lib.mp_update(self.h, _ptr(gauss), gauss.shape[0], ctypes.byref(c), _ptr(pose), _ptr(targets),
                                  _ptr(image), _ptr(inst), _ptr(table), nreg, ctypes.byref(mc), int(bool(seg_refreshed)),
                                  _ptr(labels), _ptr(stats), _ptr(mp_map), _ptr(mp_pixel), _stream()), "mp_update")
        return stats

    def semantic_trigger(self, stats, state, seg_refreshed, cfg=None, score=None):
        """Semantic-on-demand trigger of one frame (Eqs. (13)-(16)) from the
        frame's mp_update stats. state: int32 [2] device tensor (frames since
        the last refresh; out: 1 if the next frame should refresh). score:
        optional float64 [3] (e_bar, R, S). Returns score (or None)."""
        _need(stats, torch.float64, "stats")
        _need(state, torch.int32, "state")
        if state.numel() < 2:
            raise ValueError("state must hold 2 int32")
        if score is not None:
            _need(score, torch.float64, "score")
            if score.numel() < 3:
                raise ValueError("score must hold 3 doubles")
        sc = cfg if cfg is not None else default_sched_cfg()
        _check(self.lib.semantic_trigger(self.h, _ptr(stats), ctypes.byref(sc), int(bool(seg_refreshed)), _ptr(state),
                                         _ptr(score), _stream()), "semantic_trigger")
        return score

    def mpnet_features(self, image, targets, inst, table, cam: Camera, out=None):
        """8-channel bfloat16 network input [H, W, 8] of one view."""
        _need(image, torch.float32, "image")
        _need(targets, torch.float32, "targets")
        _need(inst, torch.uint8, "inst")
        _need(table, torch.float32, "table")
        if out is None:
            out = torch.empty((cam.height, cam.width, 8), dtype=torch.bfloat16, device=image.device)
        _check(self.lib.mpnet_features(self.h, _ptr(image), _ptr(targets), _ptr(inst), _ptr(table), table.shape[0],
                                       cam.width, cam.height, _ptr(out), _stream()), "mpnet_features")
        return out

    def mpnet_infer(self, weights, feats, out=None, acts=None):
        """feats: [B, H, W, 8] bfloat16 CUDA tensor; weights: uint8 blob of
        MPNET_WEIGHT_BYTES. Returns the [B, H, W] float MP map."""
        B, H, W, C = feats.shape
        if C != 8 or feats.dtype != torch.bfloat16 or not feats.is_contiguous():
            raise ValueError("feats must be a contiguous [B, H, W, 8] bfloat16 tensor")
        if out is None:
            out = torch.empty((B, H, W), dtype=torch.float32, device=feats.device)
        _check(self.lib.mpnet_infer(self.h, _ptr(weights), _ptr(feats), B, W, H, _ptr(out), _ptr(acts), _stream()),
               "mpnet_infer")
        return out

    def mpnet_train_step(self, weights, master, adam_m, adam_v, step, feats, target, lr, loss=None, grad=None):
        """One training step (BCE + Adam) of the MP network; updates weights,
        master, adam_m and adam_v in place. master/adam_m/adam_v/grad: float32
        CUDA tensors of MPNET_PARAMS; target: [B, H, W] float32 (negative =
        excluded). Returns the loss (float64 CUDA tensor of 1) at the weights
        before the step."""
        B, H, W, C = feats.shape
        if C != 8 or feats.dtype != torch.bfloat16 or not feats.is_contiguous():
            raise ValueError("feats must be a contiguous [B, H, W, 8] bfloat16 tensor")
        if tuple(target.shape) != (B, H, W):
            raise ValueError("target must be [B, H, W]")
        _need(target, torch.float32, "target")
        for name, t in (("master", master), ("adam_m", adam_m), ("adam_v", adam_v)) + \
                ((("grad", grad),) if grad is not None else ()):
            _need(t, torch.float32, name)
            if t.numel() != MPNET_PARAMS:
                raise ValueError(f"{name} must hold {MPNET_PARAMS} floats")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=feats.device)
        _check(self.lib.mpnet_train_step(self.h, _ptr(weights), _ptr(master), _ptr(adam_m), _ptr(adam_v), int(step),
                                         _ptr(feats), _ptr(target), B, W, H, float(lr), _ptr(loss), _ptr(grad),
                                         _stream()), "mpnet_train_step")
        return loss

    def selftest_timeout(self, spins: int = 1000):
        """Run the failure-path self-test (a bounded wait that runs out); the
        next check() raises with DAGS_E_TIMEOUT."""
        _check(self.lib.dags_selftest_timeout(self.h, int(spins), _stream()), "dags_selftest_timeout")

    def pose_step(self, poses, grad_pose, adam_state, cfg=None):
        _need(poses, torch.float64, "poses")
        _need(grad_pose, torch.float64, "grad_pose")
        _need(adam_state, torch.float64, "adam_state")
        c = cfg if cfg is not None else default_pose_cfg()
        _check(self.lib.pose_step(self.h, _ptr(poses), _ptr(grad_pose), _ptr(adam_state), poses.shape[0],
                                  ctypes.byref(c), _stream()), "pose_step")
