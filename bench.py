#!/usr/bin/env python
"""Benchmark of the MP-aware splatting hot path on GB300.

Metric: splat fwd+bwd iterations/s at 300k Gaussians, 640x480 (the tracking
workload: one step = one tracking frame = `--iters` (100) pose-only
forward + backward + FP64 pose-step iterations through the C ABI, plus the
per-frame MP update), and the fraction of the HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0). With N > 1 (torchrun) every rank runs an
independent replica of the workload (the path does not shard across GPUs);
value = iterations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "splat fwd+bwd iters/s (300k Gaussians, 640×480) and % of GB300 HBM roofline"
UNIT = "iters/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--iters", type=int, default=100, help="fwd+bwd iterations per tracking frame")
    ap.add_argument("--gaussians", type=int, default=300_000)
    ap.add_argument("--width", type=int, default=640)
    ap.add_argument("--height", type=int, default=480)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gain", action="store_true",
                    help="skip the learned-vs-plain MP comparisons (train + held-out evaluation, ~1 min)")
    return ap.parse_args(argv)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle arm

def oracle_baseline(args, budget_s):
    """The FP64 oracle, as it stands, on the host cores: full-image fwd+bwd
    (pose gradient) iterations of the same frame, as many as fit the budget."""
    import oracle
    from paper_2602_21644_gb300 import synth
    sc = synth.tracking_scene(args.gaussians, frame=10, width=args.width, height=args.height)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    oracle.render(G, cam, sc.poses[0], targets=sc.targets[0], grads=True)     # build + page in
    t0 = time.perf_counter()
    it = 0
    while True:
        oracle.render(G, cam, sc.poses[0], targets=sc.targets[0], grads=True)
        it += 1
        if time.perf_counter() - t0 >= budget_s and it >= 2:
            break
    dt = time.perf_counter() - t0
    return {"value": it / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{it} full-image fwd+bwd iterations (pose gradient) of the {args.gaussians}-Gaussian "
                      f"{args.width}x{args.height} tracking frame, single-threaded FP64 C, {dt:.1f} s"}


def _oracle_worker(gaussians, width, height, budget_s):
    """One host core's share of the all-cores oracle baseline: the same frame,
    full-image fwd+bwd iterations for budget_s seconds (scene set-up and one
    warm-up iteration excluded). Runs in a spawn-started process."""
    import oracle
    from paper_2602_21644_gb300 import synth
    sc = synth.tracking_scene(gaussians, frame=10, width=width, height=height)
    G = oracle.params_from_records(sc.records)
    cam = oracle.camera_vec(*sc.camera.as_tuple())
    oracle.render(G, cam, sc.poses[0], targets=sc.targets[0], grads=True)
    t0 = time.perf_counter()
    it = 0
    while True:
        oracle.render(G, cam, sc.poses[0], targets=sc.targets[0], grads=True)
        it += 1
        if time.perf_counter() - t0 >= budget_s and it >= 1:
            break
    return it, time.perf_counter() - t0


def oracle_baseline_all_cores(args, budget_s):
    """The oracle, as it stands, on every host core at once: one process per
    core (spawn: the bench process already holds a CUDA context), each running
    whole iterations of the frame; throughput = all iterations / the slowest
    process's time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, [args.gaussians] * cores, [args.width] * cores, [args.height] * cores,
                          [budget_s] * cores))
    its = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": its / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{its} full-image fwd+bwd iterations (pose gradient) of the {args.gaussians}-Gaussian "
                      f"{args.width}x{args.height} tracking frame in {cores} processes (one per host core), FP64 C, "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = oracle_baseline_all_cores(args, max(5.0, args.cpu_seconds))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MAX_FRAMES = 50   # frames 10-59 of the 60-frame sequence


def workload_config(args):
    F = max(1, min(args.steps, MAX_FRAMES))
    return {"workload": f"tracking frames 10-{9 + F} of a synthetic room sequence (two objects at 0.3 m/s, "
                        f"30 Hz): {args.gaussians} Gaussians, {args.width}x{args.height} RGB-D, {args.iters} "
                        f"pose-only fwd+bwd iterations with FP64 pose steps and one MP update per frame (step)",
            "gaussians": args.gaussians, "width": args.width, "height": args.height,
            "iters_per_step": args.iters,
            "l2": "flushed between steps by a 256 MiB write, then a 256 MiB read of a never-written buffer (L2 left clean); inside a step the iterations re-read the "
                  "L2-resident map as the tracking loop does",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------------------------ ranks

def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of the ranks' values (the slowest rank's time); the
    value itself on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(iters_per_step: int, steps: int, world: int, t_ms_max: float) -> float:
    """Whole-job iterations per second: every replica runs the same steps;
    the job takes the slowest rank's time."""
    return iters_per_step * steps * world / (t_ms_max / 1e3)


# ------------------------------------------------------------------ our arm

def algorithmic_bytes(n, nv, K, P):
    """Compulsory bytes per stage of one pose-only iteration: each stage
    reads its inputs and writes its outputs once (the method's stages,
    whatever kernels run them)."""
    return {"preprocess": 64 * n + 48 * nv,
            "emit": 12 * K,
            "tile_sort": 24 * K,
            "render_fwd": 52 * K + 16 * P + 32 * P,
            "render_bwd": 52 * K + 48 * P + 24 * nv,
            "preprocess_bwd": 64 * nv + 24 * nv,
            "pose_step": 6 * 8 + 13 * 8 * 2 + 12 * 8 * 2}


def kernel_bytes(n, nv, K, P):
    """Compulsory bytes per launch of the tracking loop's kernels: the
    preprocess reads every record and writes the projected records and the
    keys into the tile buckets; the forward sorts its keys (read 8, write 4
    bytes per pair), reads each pair's projected record and the targets, and
    writes the image (8 planes) and last; the adjoint reads each pair's id
    and record, the targets, the image and last, and adds the 2D gradients
    (6 words per visible Gaussian); the pose chain reads the records and 2D
    gradients of the visible Gaussians."""
    return {"preprocess": 64 * n + 48 * nv + 8 * K,
            "render_fwd": 12 * K + 52 * K + 16 * P + 36 * P,
            "render_bwd": 52 * K + 16 * P + 36 * P + 24 * nv,
            "preprocess_bwd": 64 * nv + 24 * nv}


# FP32 lane operations of the compositing loops (the method's arithmetic; an
# exp2 or a reciprocal counts as one), per evaluated exponent: the pixel
# offset 2, the quadratic form 6 and the alpha_min test 1; per contribution
# (alpha >= alpha_min): forward alpha, its clamp, 1 - alpha, the new T and its
# test, the weight and six accumulations (12); backward alpha, its clamp,
# 1/(1 - alpha), the transmittance recovery, the weight, dL/dalpha over six
# channels with its suffix term, the chain to centre, conic and depth, the
# suffix update and the warp sums of the six gradient words (39). The
# evaluation and contribution counts are counted by the kernels themselves.
OPS_EVAL, OPS_FWD_CONTRIB, OPS_BWD_CONTRIB = 9, 12, 39
# special-function operations per contribution: forward exp2; backward exp2
# and the reciprocal of 1 - alpha
SFU_FWD_CONTRIB, SFU_BWD_CONTRIB = 1, 2
# the LM Jacobian compositing, per listed evaluation: the forward's 16, 10
# shared per evaluation (exponent gradient, squared offsets, ln2 alpha) and 14
# per twist direction (the exponent's tangent 5, alpha' 1, the weight's
# tangent 2, four channel accumulations 5, T' 1) over six directions
OPS_JAC = 16 + 10 + 6 * 14
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
# the tracking iteration's kernels as the traffic file names them
TRAFFIC_NAMES = {"preprocess": "preprocess_cull_kernel", "render_fwd": "render_fwd_kernel",
                 "render_bwd": "render_bwd_kernel<pose-only>", "preprocess_bwd": "preprocess_bwd_kernel<pose-only>"}


def source_digest(paths: str) -> str:
    """SHA-256 (first 16 hex digits) of the concatenated bytes of the
    '+'-separated source files (paths relative to the repository root)."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths.split("+"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summary, or (None, why) when there is no capture or one of
    the kernel's source files has changed since it was taken (the file
    records the SHA-256 of the sources the kernel compiles from)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no committed capture"
    for line in open(TRAFFIC_FILE):
        if line.startswith("#") or "|" not in line:
            continue
        f = [x.strip() for x in line.split("|")]
        if len(f) < 5 or f[0] != kernel or f[1] != workload:
            continue
        missing = [rel for rel in f[3].split("+") if not os.path.exists(os.path.join(ROOT, rel))]
        if missing:
            return None, f"source {missing[0]} missing"
        sha = source_digest(f[3])
        if sha != f[4]:
            return None, f"{f[3]} changed since the capture"
        return int(f[2]), f"ncu capture of this source ({f[3]} sha256 {sha}; cold caches)"
    return None, "no committed capture of this kernel and workload"


ALU_LANES = 152 * 128          # FP32 lanes: 152 SMs x 128
MPNET_FLOP_PER_PX = 2 * (8 * 32 + 288 * 32 + 32 * 32 + 32)   # 21,056: the network's multiply-adds x 2


class L2Flush:
    """Between timed iterations: write a 256 MiB buffer (twice the 129 MB L2),
    then read a second, never-written 256 MiB buffer, so that L2 holds clean
    lines and the timed work does not pay the write-back of the flush."""

    def __init__(self, torch, dev):
        self.torch = torch
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.out = None

    def fill_(self, v):
        self.w.fill_(v)
        self.out = self.r.sum()


def learned_mp_section(args, ctx, dags, synth, image, targets, inst, table, cam, flush, stream):
    """Learned MP proposal at its inference batch: 16 frames of 640x480 per
    launch. The network input is assembled by the library from the frame's
    render (mpnet_features), one copy per frame; weights are a seeded draw.
    Also one training step (BCE + Adam) on the same batch against the frame's
    rendered MP. Times are CUDA events around each launch, L2 flushed before."""
    import torch
    B = 16
    P = cam.width * cam.height
    f1 = ctx.mpnet_features(image[0].reshape(dags.IMG_CHANNELS, P), targets, inst, table, cam)
    feats = f1[None].repeat(B, 1, 1, 1).contiguous()
    blob, master = synth.mpnet_init(1)
    blob = torch.from_numpy(blob).cuda()
    master = torch.from_numpy(master).cuda()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    target = image[0, 5][None].repeat(B, 1, 1).contiguous()
    out = torch.empty((B, cam.height, cam.width), dtype=torch.float32, device=feats.device)
    step = [0]

    def infer():
        ctx.mpnet_infer(blob, feats, out=out)

    def train():
        step[0] += 1
        ctx.mpnet_train_step(blob, master, m, v, step[0], feats, target, 1e-4)

    def time_it(fn, reps):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)) * 1e3

    t_inf = time_it(infer, 20)
    t_tr = time_it(train, 10)
    torch.cuda.synchronize()
    ctx.check()
    flop = MPNET_FLOP_PER_PX * B * P
    return {"workload": f"{B} frames of {cam.width}x{cam.height} x 8 BF16 features per launch",
            "infer_us": round(t_inf, 2), "infer_frames_per_s": round(B / (t_inf * 1e-6), 1),
            "infer_tflops": round(flop / (t_inf * 1e-6) / 1e12, 2), "alg_flop_per_launch": flop,
            "train_step_us": round(t_tr, 2), "gpu_launches_infer": 1, "gpu_launches_train": 6}


def mp_section(ctx, dags, gauss, cam, poses, targets, image, inst, table, labels, mp_stats, flush, stream):
    """The per-frame MP update (Sec. IV-A) on the tracking frame, with the
    association over 1, 2 and 3 pyramid levels (Eq. (1)): CUDA events around
    each call, L2 flushed before. The Gaussians' MP words and labels are put
    back afterwards."""
    import torch
    mp0 = gauss[:, 11].clone()
    lab0 = labels.clone()
    out = {}
    for S in (1, 2, 3):
        cfg = dags.default_mp_cfg(scales=S)
        for _ in range(3):
            ctx.mp_update(gauss, cam, poses, targets, image, inst, table, labels, cfg, stats=mp_stats)
        ts = []
        for _ in range(10):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.mp_update(gauss, cam, poses, targets, image, inst, table, labels, cfg, stats=mp_stats)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[f"scales_{S}_us"] = round(float(np.median(ts)) * 1e3, 2)
    gauss[:, 11].copy_(mp0)
    labels.copy_(lab0)
    torch.cuda.synchronize()
    ctx.check()
    out["workload"] = f"{gauss.shape[0]} Gaussians, {cam.width}x{cam.height}, one view"
    return out


def lm_section(args, ctx, dags, gauss, cam, targets0, pose0, gt_pose, pcfg, flush, stream, alu_peak):
    """Levenberg-Marquardt pose refinement (the second-order tracker) on the
    bench's first tracking frame (300k Gaussians, 640x480, its ray-cast
    target): device time per LM iteration through the captured loop (graph
    replay, L2 flushed before every timed call) and per kernel (direct
    launches with CUDA events). Then convergence on the same map with a
    self-consistent target (the map rendered at the ground-truth pose; the
    ray-cast target's loss minimum lies centimetres from the ground truth for
    any optimiser): pose error after 15 LM iterations against 100 iterations
    of the first-order tracker, and the device time of each."""
    import torch
    iters = 15
    P = cam.width * cam.height
    pose = pose0.clone().contiguous()
    state = torch.empty(dags.LM_STATE, dtype=torch.float64, device=gauss.device)

    def run_lm(tg, graph=True):
        pose.copy_(pose0)
        ctx.track_lm(gauss, cam, pose, tg, iters, state=state, use_graph=graph)

    def time_it(fn, reps):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_frame = time_it(lambda: run_lm(targets0), 10)
    ctx.timing_read()
    ctx.timing(True)
    for _ in range(3):
        run_lm(targets0, graph=False)
    torch.cuda.synchronize()
    ctx.timing(False)
    kt = ctx.timing_read()
    kern = {}
    for name in ("preprocess", "emit", "pose_tangent", "render_jac", "lm_step"):
        ms, cnt = kt.get(name, (0.0, 0))
        if cnt:
            kern[name] = {"launches": cnt, "avg_us": round(1e3 * ms / cnt, 3)}
    # evaluations of one Jacobian compositing launch at the starting pose
    last = torch.empty(P, dtype=torch.int32, device=gauss.device)
    ctx.normal_equations(gauss, cam, pose0.contiguous(), targets0, last=last)
    E = int(last.to(torch.int64).sum().item())
    jac_us = kern["render_jac"]["avg_us"]
    jac_tops = E * OPS_JAC / (jac_us * 1e-6) / 1e12
    roof = {"kernel": "render_jac", "bound": "alu", "achieved": round(jac_tops, 3), "peak": round(alu_peak, 2),
            "unit": "TFLOP/s", "frac": round(jac_tops / alu_peak, 4), "ops_per_evaluation": OPS_JAC,
            "evaluations_per_launch": E}

    # convergence against a self-consistent target
    image = torch.empty((1, dags.IMG_CHANNELS, cam.height, cam.width), dtype=torch.float32, device=gauss.device)
    lastf = torch.empty((1, cam.height, cam.width), dtype=torch.int32, device=gauss.device)
    ctx.forward(gauss, cam, gt_pose[None].contiguous(), None, image=image, last=lastf)
    tg2 = torch.empty_like(targets0)
    im = image[0].reshape(dags.IMG_CHANNELS, P)
    tg2[:, 0:4] = im[0:4].t()
    tg2[:, 3] = torch.where(im[4] > 0.5, im[3], torch.zeros_like(im[3]))
    t_lm = time_it(lambda: run_lm(tg2), 5)
    torch.cuda.synchronize()
    e_lm = pose_error(pose.cpu().numpy(), gt_pose.cpu().numpy())
    pa = pose0[None].clone().contiguous()
    adam = torch.zeros((1, 13), dtype=torch.float64, device=gauss.device)
    loss = torch.empty(1, dtype=torch.float64, device=gauss.device)
    gp = torch.empty((1, 6), dtype=torch.float64, device=gauss.device)
    tgb = tg2[None].contiguous()

    def run_adam():
        pa.copy_(pose0[None])
        adam.zero_()
        ctx.track(gauss, cam, pa, tgb, 100, adam, image, lastf, loss, gp, pcfg=pcfg)

    t_adam = time_it(run_adam, 5)
    torch.cuda.synchronize()
    e_adam = pose_error(pa[0].cpu().numpy(), gt_pose.cpu().numpy())
    e0 = pose_error(pose0.cpu().numpy(), gt_pose.cpu().numpy())
    ctx.check()
    return {"workload": "tracking frame 10: 300k Gaussians, 640x480, 15 LM iterations per frame",
            "us_per_iter": round(1e3 * t_frame / iters, 3), "iters_per_s": round(iters / (t_frame * 1e-3), 1),
            "kernels": kern, "roofline": roof,
            "gpu_launches_per_iter": 3,
            "convergence": {"target": "the map rendered at the ground-truth pose",
                            "start_error": {"mm": round(1e3 * e0[0], 4), "deg": round(float(np.degrees(e0[1])), 5)},
                            "lm_15_iters": {"mm": round(1e3 * e_lm[0], 4), "deg": round(float(np.degrees(e_lm[1])), 5),
                                            "ms": round(t_lm, 3), "accepted": int(state[41].item())},
                            "adam_100_iters": {"mm": round(1e3 * e_adam[0], 4),
                                               "deg": round(float(np.degrees(e_adam[1])), 5), "ms": round(t_adam, 3)}}}


def edge_section(ctx, dags, gauss, cam, tg_all, pose_all, flush, stream):
    """The edge-warp regulariser (Eqs. (25), (26)) between the sequence's
    first two frames at 640x480: the observed depths of frames 10 and 11, the
    static weight w^j of frame 11's render (channel 7), their starting poses;
    CUDA events around the launch, L2 flushed before each. One thread per
    pixel of frame i: the edge test reads four neighbours, the warp and the
    bilinear samples touch the few edge pixels, so the launch is latency-bound
    (about 1.2 MB of depth read)."""
    import torch
    P = cam.width * cam.height
    Di = tg_all[0, 0, :, 3].contiguous()
    Dj = tg_all[1, 0, :, 3].contiguous()
    image, _, _ = ctx.forward(gauss, cam, pose_all[1].contiguous(), tg_all[1].contiguous())
    wj = image[0, 7].reshape(P).contiguous()
    pi = pose_all[0, 0].contiguous()
    pj = pose_all[1, 0].contiguous()
    out = torch.empty(13, dtype=torch.float64, device=gauss.device)
    fn = lambda: ctx.edge_warp(cam, Di, Dj, wj, pi, pj, 300.0, out=out)
    for _ in range(3):
        fn()
    ts = []
    for _ in range(20):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.check()
    return {"workload": f"frames 10 -> 11, {cam.width}x{cam.height}, w^j from frame 11's render",
            "us": round(1e3 * float(np.median(ts)), 3), "loss": round(float(out[0].item()), 4),
            "bound": "latency (one pass over the depth image; edge pixels only beyond the test)"}


def epipolar_section(dags, flush, stream):
    """Epipolar verification and static recovery (Eqs. (18), (19)) on the
    synthetic matches of frames 11 and 16 (300k-Gaussian map, 20k Gaussians
    with 4 matches each, 0.3 px noise): CUDA events around the call (seven
    launches: distances, three scan kernels, scatter, medians; one memset),
    L2 flushed before each; and what the recovery does."""
    import torch
    from paper_2602_21644_gb300 import synth
    d = synth.epipolar_matches()
    cam = dags.Camera(*d["camera"].as_tuple())
    n = d["records"].shape[0]
    ctx = dags.Context(n, cam.width, cam.height, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g0, lab0 = t(d["records"]), t(d["labels"])
    g, lab = g0.clone(), lab0.clone()
    args = (cam, t(d["pose_1"].ravel()), t(d["pose_2"].ravel()), t(d["p1"]), t(d["p2"]), t(d["gid"]))
    ctx.epipolar_verify(*args, g, lab)
    torch.cuda.synchronize()
    restored = ((lab0 == 1) & (lab == 0)).cpu().numpy()
    ts = []
    for _ in range(20):
        g.copy_(g0)
        lab.copy_(lab0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.epipolar_verify(*args, g, lab, want_d=False, want_dbar=False)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.check()
    ctx.close()
    moving = d["moving"]
    return {"workload": f"{len(d['gid'])} matches of {len(np.unique(d['gid']))} Gaussians, frames 11 -> 16, "
                        f"{n} Gaussians",
            "us": round(1e3 * float(np.median(ts)), 3), "gpu_launches": 7,
            "restored_static": int((restored & ~moving).sum()), "restored_moving": int((restored & moving).sum()),
            "suppressed_static": int(((d["labels"] == 1) & ~moving).sum())}


def pose_error(T, T_gt):
    """(camera-centre distance in m, rotation angle in rad) of world-to-camera poses."""
    T = np.asarray(T, np.float64).reshape(3, 4)
    T_gt = np.asarray(T_gt, np.float64).reshape(3, 4)
    c = -T[:, :3].T @ T[:, 3]
    c_gt = -T_gt[:, :3].T @ T_gt[:, 3]
    R = T[:, :3] @ T_gt[:, :3].T
    return float(np.linalg.norm(c - c_gt)), float(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))


def gain_section(dags):
    """What the learned proposal gains over the method without it, on the
    library's own kernels (paper_2602_21644_gb300.mp_eval): trained on a
    synthetic 60-frame sequence at 320x240 (80k Gaussians, semantic refresh
    every 10 frames), evaluated on a held-out 40-frame one. Means over the
    frames between refreshes: per-pixel MP MAE and IoU(M > 0.5) against the
    fresh-prior arm, static/dynamic label IoU with the fresh-prior labels and
    with the ground-truth moving Gaussians."""
    import time
    from paper_2602_21644_gb300 import mp_eval
    t0 = time.time()
    ex = mp_eval.experiment(dags)
    m = mp_eval.metrics(ex)
    out = {"workload": "train 60 + held-out 40 frames, 320x240, 80k Gaussians, refresh every 10, 1000 Adam steps"}
    for key, (a, b) in {"mp_mae": ("mae_s", "mae_l"), "mp_iou": ("iou_s", "iou_l"),
                        "label_iou_vs_fresh_prior": ("agree_s", "agree_l"),
                        "label_iou_vs_ground_truth": ("gt_s", "gt_l")}.items():
        out[key] = {"stale_prior": round(m[a], 4), "learned": round(m[b], 4)}
    out["label_iou_vs_ground_truth"]["fresh_prior"] = round(m["gt_j"], 4)
    out["train_loss"] = {"first": round(m["loss_first"], 4), "last": round(m["loss_last"], 4)}
    # the semantic-on-demand trigger (Eqs. (13)-(16)) against the fixed cadence, over frames 1-39
    out["semantic_schedule"] = {k: {a: (round(b, 4) if isinstance(b, float) else b) for a, b in v.items()}
                                for k, v in mp_eval.schedule_metrics(ex).items()}
    out["seconds"] = round(time.time() - t0, 1)
    return out


def gain_rendered_section(dags):
    """The same comparison with the network trained on 10,000 frames the
    plain method generates on the mapping room at 640x480 (observations
    rendered by the library: mp_eval.rendered_training_set), 3000 Adam steps
    of 16 frames, evaluated on a held-out ray-cast 640x480 sequence (200k
    Gaussians, 40 frames)."""
    import time
    from paper_2602_21644_gb300 import mp_eval
    t0 = time.time()
    ex = mp_eval.experiment_rendered(dags, n_frames=10_000, steps=3000)
    m = mp_eval.metrics(ex)
    out = {"workload": "train: 10,000 rendered frames of the 200k-Gaussian mapping room at 640x480, 3000 Adam "
                       "steps x 16 frames; held-out: 40 ray-cast frames at 640x480, refresh every 10",
           "generate_s": round(ex["t_gen"], 1), "train_s": round(ex["t_train"], 1)}
    for key, (a, b) in {"mp_mae": ("mae_s", "mae_l"), "mp_iou": ("iou_s", "iou_l"),
                        "label_iou_vs_fresh_prior": ("agree_s", "agree_l")}.items():
        out[key] = {"stale_prior": round(m[a], 4), "learned": round(m[b], 4)}
    out["train_loss"] = {"first": round(m["loss_first"], 4), "last": round(m["loss_last"], 4)}
    out["seconds"] = round(time.time() - t0, 1)
    return out


def splat_variants_section(args, ctx, dags, synth, gauss, cam, targets, poses, flush, stream):
    """The other two splatting workloads, each timed with CUDA events around
    direct launches, L2 flushed before every timed iteration:
    - the full-parameter fwd+bwd variant at the tracking size (one view;
      gradients of every Gaussian parameter and of the pose);
    - the mapping step: 200k Gaussians, 8 keyframes of 640x480, one iteration
      = render + backward of all 8 views w.r.t. all parameters, plus the
      lambda_3 L_MP gradient;
    - the L_MP regulariser alone at the tracking map's size."""
    import torch

    def time_it(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    flags = dags.GRAD_GAUSS | dags.GRAD_POSE

    def full_iter():
        image, last, _ = ctx.forward(gauss, cam, poses, targets)
        ctx.backward(gauss, cam, poses, targets, image, last, flags)

    t_full = time_it(full_iter)
    ms = synth.mapping_scene(200_000, views=8, width=args.width, height=args.height)
    mcam = dags.Camera(*ms.camera.as_tuple())
    mg = torch.from_numpy(ms.records).cuda()
    mp = torch.from_numpy(np.ascontiguousarray(ms.poses)).cuda()
    mt = torch.from_numpy(np.ascontiguousarray(ms.targets)).cuda()
    mctx = dags.Context(mg.shape[0], mcam.width, mcam.height, ms.poses.shape[0])

    mprev = mg.clone()          # the records after the previous mapping update (Eq. (23))
    mstate = mctx.gauss_adam_state(mg)
    mstep = [0]

    def map_iter():
        # Eq. (27) without the edge term: MP-weighted L1 of every view,
        # lambda_3 L_MP added into the Gaussian gradient, then the Adam step
        # on the Gaussian parameters
        image, last, _ = mctx.forward(mg, mcam, mp, mt)
        gg, _ = mctx.backward(mg, mcam, mp, mt, image, last, flags)
        mctx.mp_consistency(mg, mprev, 500.0, grad=gg, want_loss=False)
        mstep[0] += 1
        mctx.gauss_adam_step(mg, mstate, gg, mstep[0])

    t_map = time_it(map_iter)
    # the regulariser alone at the tracking map's size: HBM-bound, 80 bytes
    # per Gaussian (two float4 of the record, one of the snapshot, the
    # gradient's first float4 read and written)
    prev = gauss.clone()
    greg = torch.zeros_like(gauss)
    t_reg = time_it(lambda: ctx.mp_consistency(gauss, prev, 500.0, grad=greg), reps=20)
    reg_bytes = 80 * gauss.shape[0]
    hbm = float(load_peaks()[0]["hbm_gbs"])
    torch.cuda.synchronize()
    ctx.check()
    mctx.check()
    mctx.close()
    # the tiny scene (2,000 Gaussians, 160x120): fwd+bwd of all parameters
    # and the pose on the GPU, and 100 iterations of the FP64 oracle on one
    # host core, as the same units
    ts = synth.tiny_scene(0)
    tcam = dags.Camera(*ts.camera.as_tuple())
    tgx = torch.from_numpy(ts.records).cuda()
    tpx = torch.from_numpy(np.ascontiguousarray(ts.poses)).cuda()
    ttx = torch.from_numpy(np.ascontiguousarray(ts.targets)).cuda()
    tctx = dags.Context(tgx.shape[0], tcam.width, tcam.height, 1)

    def tiny_iter():
        image, last, _ = tctx.forward(tgx, tcam, tpx, ttx)
        tctx.backward(tgx, tcam, tpx, ttx, image, last, flags)

    t_tiny = time_it(tiny_iter, reps=20)
    torch.cuda.synchronize()
    tctx.check()
    tctx.close()
    tiny = {"workload": "2000 Gaussians, 160x120, one view, gradients of all Gaussian parameters and the pose",
            "ms_per_iter": round(t_tiny, 4), "iters_per_s": round(1e3 / t_tiny, 2)}
    if not args.no_cpu_baseline:
        import oracle
        G = oracle.params_from_records(ts.records)
        ocam = oracle.camera_vec(*ts.camera.as_tuple())
        oracle.render(G, ocam, ts.poses[0], targets=ts.targets[0], grads=True)
        t0 = time.perf_counter()
        for _ in range(100):
            oracle.render(G, ocam, ts.poses[0], targets=ts.targets[0], grads=True)
        dt = time.perf_counter() - t0
        tiny["cpu_baseline"] = {"value": round(100 / dt, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"100 fwd+bwd iterations (all gradients) of the tiny scene, FP64 C, "
                                          f"{dt:.2f} s"}
    return {"tiny": tiny,
            "full_param_fwd_bwd": {"workload": f"{gauss.shape[0]} Gaussians, {cam.width}x{cam.height}, one view, "
                                               "gradients of all Gaussian parameters and the pose",
                                   "ms_per_iter": round(t_full, 4), "iters_per_s": round(1e3 / t_full, 2)},
            "mapping": {"workload": f"200000 Gaussians, 8 keyframes of {mcam.width}x{mcam.height}, render + "
                                    "backward of all views w.r.t. all parameters",
                        "ms_per_iter": round(t_map, 4), "iters_per_s": round(1e3 / t_map, 2),
                        "includes": "lambda_3 L_MP gradient (Eqs. (23), (24)) and the Adam step on the "
                                    "Gaussian parameters"},
            "mp_consistency": {"workload": f"lambda_3 L_MP and its gradient over {gauss.shape[0]} Gaussians",
                               "us": round(1e3 * t_reg, 3), "alg_bytes": reg_bytes,
                               "hbm_frac": round(reg_bytes / (t_reg * 1e-3) / 1e9 / hbm, 4)}}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2602_21644_gb300 import dags, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # frames 10 .. 10 + F - 1 of the sequence; step k tracks frame k mod F
    # (its RGB-D target, instance prior and starting pose, all resident on
    # the device and copied into the working buffers as the step begins)
    F = max(1, min(args.steps, MAX_FRAMES))
    records, scam, seq, sx = synth.tracking_sequence(args.gaussians, frames=range(10, 10 + F), width=args.width,
                                                     height=args.height)
    cam = dags.Camera(*scam.as_tuple())
    n = records.shape[0]
    P = cam.width * cam.height
    gauss = torch.from_numpy(records).to(dev)
    tg_all = torch.from_numpy(np.stack([f["target"] for f in seq])[:, None]).to(dev)       # F x 1 x P x 4
    pose_all = torch.from_numpy(np.stack([f["pose"] for f in seq])[:, None]).to(dev)      # F x 1 x 3 x 4
    inst_all = torch.from_numpy(np.stack([f["instance"] for f in seq])).to(dev)           # F x P
    targets = tg_all[0].clone()
    poses = pose_all[0].clone()
    inst = inst_all[0].clone()
    fidx = [0]
    state = torch.zeros((1, 13), dtype=torch.float64, device=dev)
    image = torch.empty((1, dags.IMG_CHANNELS, cam.height, cam.width), dtype=torch.float32, device=dev)
    last = torch.empty((1, cam.height, cam.width), dtype=torch.int32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gpose = torch.empty((1, 6), dtype=torch.float64, device=dev)
    ctx = dags.Context(n, cam.width, cam.height, 1)
    pcfg = dags.default_pose_cfg(lr=[1e-3, 1e-3, 1e-3, 5e-4, 5e-4, 5e-4])
    # per-frame MP update inputs: the frame's instance prior and class table
    table = torch.tensor([[0.1, 0.05]] + [[0.9, 0.8]] * sx["n_instances"], dtype=torch.float32, device=dev)
    labels = torch.zeros(n, dtype=torch.uint8, device=dev)
    mp_stats = torch.empty(dags.MP_STATS_HEAD + 4 * table.shape[0], dtype=torch.float64, device=dev)
    flush = L2Flush(torch, dev)

    def frame(use_graph=True):
        k = fidx[0] % F
        fidx[0] += 1
        targets.copy_(tg_all[k])
        poses.copy_(pose_all[k])
        inst.copy_(inst_all[k])
        state.zero_()
        ctx.track(gauss, cam, poses, targets, args.iters, state, image, last, loss, gpose, pcfg=pcfg,
                  use_graph=use_graph)
        ctx.mp_update(gauss, cam, poses, targets, image, inst, table, labels, stats=mp_stats)

    # warm-up (captures the iteration graph; checks the device status once)
    for _ in range(max(1, args.warmup)):
        frame()
    frame(use_graph=False)
    torch.cuda.synchronize()
    ctx.check()
    # the pairs K and visible Gaussians N_v at the frame's final pose (a
    # plain forward: the tracking loop keeps its lists in the fixed-bucket
    # layout)
    ctx.forward(gauss, cam, poses, targets, image=image, last=last, loss=loss)
    start_bins, ids = ctx.copy_bins(1, cam)
    K = int(len(ids))
    nv = int(len(np.unique(ids)))
    # measured FP32 FMA and ex2 lane rates (T ops/s) for the ALU roofline
    alu_peak = max(dags.measure_alu(0, 1 << 15)[0] for _ in range(3)) / 1e12
    sfu_peak = max(dags.measure_alu(1, 1 << 13)[0] for _ in range(3)) / 1e12

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)

    def timed(steps, fn, timing=False):
        ctx.timing(timing)
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        ctx.timing(False)
        return tot

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_ms = timed(args.steps, frame)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = max_over_ranks(t_ms, world, dev)
    if world > 1:
        dist.barrier()
    value = replica_throughput(args.iters, args.steps, world, t_ms)

    # per-kernel device times: the same steps with every kernel launched
    # directly (no graph) between a pair of CUDA events on its stream; the
    # compositing kernels also count the exponents they evaluate and the
    # contributions among them (one atomic per warp and counter)
    ctx.timing_read()
    t_direct = timed(args.steps, lambda: frame(use_graph=False), timing=True)
    kt = ctx.timing_read()
    # the compositing kernels' evaluation counts, in a pass of their own (the
    # counting variants of the kernels are not the timed ones)
    ctx.eval_read()
    ctx.eval_counting(True)
    n_count = min(args.steps, 5)
    for _ in range(n_count):
        frame(use_graph=False)
    ctx.eval_counting(False)
    evals = ctx.eval_read()
    count_launches = n_count * args.iters

    # e2e: public API with host buffers; every step copies the frame (RGB-D
    # target) and the starting pose from pinned host memory and reads back the
    # refined pose and the loss
    tg_host = torch.from_numpy(np.stack([f["target"] for f in seq])[:, None]).pin_memory()
    pose_host = torch.from_numpy(np.stack([f["pose"] for f in seq])[:, None]).pin_memory()
    inst_host = torch.from_numpy(np.stack([f["instance"] for f in seq])).pin_memory()
    pose_out = torch.empty_like(pose_host[0]).pin_memory()
    loss_out = torch.empty(1, dtype=torch.float64).pin_memory()

    def frame_e2e():
        k = fidx[0] % F
        fidx[0] += 1
        targets.copy_(tg_host[k], non_blocking=True)
        poses.copy_(pose_host[k], non_blocking=True)
        inst.copy_(inst_host[k], non_blocking=True)
        state.zero_()
        ctx.track(gauss, cam, poses, targets, args.iters, state, image, last, loss, gpose, pcfg=pcfg)
        ctx.mp_update(gauss, cam, poses, targets, image, inst, table, labels, stats=mp_stats)
        pose_out.copy_(poses, non_blocking=True)
        loss_out.copy_(loss, non_blocking=True)

    t_e2e = max_over_ranks(timed(args.steps, frame_e2e), world, dev)
    h2d = tg_host[0].numel() * 4 + pose_host[0].numel() * 8 + inst_host[0].numel()
    d2h = pose_out.numel() * 8 + 8

    mp_upd = mp_section(ctx, dags, gauss, cam, poses, targets, image, inst, table, labels, mp_stats, flush, stream)
    learned = learned_mp_section(args, ctx, dags, synth, image, targets, inst, table, cam, flush, stream)
    if not args.no_gain and rank == 0:
        learned["gain"] = gain_section(dags)
        learned["gain_10k"] = gain_rendered_section(dags)
    variants = splat_variants_section(args, ctx, dags, synth, gauss, cam, targets, poses, flush, stream)
    lm = lm_section(args, ctx, dags, gauss, cam, tg_all[0, 0].contiguous(), pose_all[0, 0].contiguous(),
                    torch.from_numpy(np.ascontiguousarray(seq[0]["gt_pose"])).to(dev), pcfg, flush, stream,
                    alu_peak)

    peaks, src = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    ab = kernel_bytes(n, nv, K, P)
    kernels = {}
    kt_total = sum(ms for ms, _ in kt.values())
    for name, (ms, cnt) in kt.items():
        if cnt:
            avg_us = 1e3 * ms / cnt
            kernels[name] = {"launches": cnt, "avg_us": round(avg_us, 3), "share": round(ms / max(kt_total, 1e-9), 4)}
            if name in ab:
                kernels[name]["alg_bytes"] = ab[name]
                kernels[name]["hbm_frac"] = round(ab[name] / (avg_us * 1e-6) / 1e9 / hbm, 4)
                tr, _ = committed_traffic(TRAFFIC_NAMES.get(name, name), f"tracking {args.gaussians // 1000}k "
                                                                        f"{args.width}x{args.height}")
                kernels[name]["dram_bytes"] = tr
    # the compositing kernels are ALU-bound: per launch, E_eval evaluated
    # exponents and E_contrib contributions (counted by the kernels), OPS_*
    # FP32 lane operations per unit, against the measured FMA lane rate;
    # E_listed (every list entry up to each pixel's last contributor) is
    # reported beside them
    E_listed = int(last.to(torch.int64).sum().item())
    # the forward's units are its evaluations and contributions, the
    # adjoint's its own (the kernels count them)
    fe, fc = evals["fwd_eval"] / count_launches, evals["fwd_contrib"] / count_launches
    be, bc = evals["bwd_eval"] / count_launches, evals["bwd_contrib"] / count_launches
    per = {"render_fwd": (fe, fc, OPS_FWD_CONTRIB, SFU_FWD_CONTRIB),
           "render_bwd": (be, bc, OPS_BWD_CONTRIB, SFU_BWD_CONTRIB)}
    for name, (ee, ec, oc, sc) in per.items():
        if name in kernels:
            t_s = kernels[name]["avg_us"] * 1e-6
            ops = OPS_EVAL * ee + oc * ec
            kernels[name].update({"evaluations_performed": int(round(ee)), "contributions": int(round(ec)),
                                  "evaluations_listed": E_listed, "alg_ops": int(round(ops)),
                                  "alu_tops": round(ops / t_s / 1e12, 3),
                                  "alu_frac": round(ops / t_s / 1e12 / alu_peak, 4),
                                  "sfu_frac": round(sc * ec / t_s / 1e12 / sfu_peak, 4)})
    modelled = [k for k in kernels if k in ab]
    dom = max(modelled, key=lambda k: kt[k][0]) if modelled else None
    roof = None
    workload = f"tracking {args.gaussians // 1000}k {args.width}x{args.height}"
    if dom in ("render_fwd", "render_bwd"):
        ach = kernels[dom]["alu_tops"]
        traffic, tnote = committed_traffic(TRAFFIC_NAMES[dom], workload)
        ee, ec, oc, _ = per[dom]
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / alu_peak, 4), "traffic": traffic, "traffic_source": tnote,
                "peak_source": "measured in this run: FP32 FMA lane operations/s (dags_measure_alu), "
                               "one FMA counted as one operation",
                "alg_ops_per_launch": kernels[dom]["alg_ops"], "ops_per_evaluation": OPS_EVAL,
                "ops_per_contribution": oc, "evaluations_performed": int(round(ee)),
                "contributions": int(round(ec)), "evaluations_listed": E_listed,
                "alg_bytes_per_launch": ab[dom], "hbm_frac": kernels[dom].get("hbm_frac"),
                "sfu_frac": kernels[dom]["sfu_frac"], "sfu_peak": round(sfu_peak, 2)}
    elif dom:
        avg_s = kernels[dom]["avg_us"] * 1e-6
        ach = ab[dom] / avg_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 2), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": None, "peak_source": f"{src} hbm_gbs (copy)",
                "alg_bytes_per_launch": ab[dom]}
    iter_bytes = sum(algorithmic_bytes(n, nv, K, P).values())
    iter_us = 1e3 * t_ms / (args.iters * args.steps)
    # kernels per step: per iteration the preprocess (with direct binning),
    # the forward, the adjoint and the pose chain (pose step fused); per frame
    # the culling and the MP update's 9 kernels (pixel sum, pixel var, pixel map, gauss,
    # apply, 2 select levels, labels, region stats)
    gpu_launches = args.steps * (args.iters * 4 + 9 + 1)   # + the frame's culling
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args),
            "iteration_hbm_roofline": {"alg_bytes": iter_bytes, "us_per_iter": round(iter_us, 3),
                                       "frac": round(iter_bytes / (iter_us * 1e-6) / 1e9 / hbm, 4),
                                       "peak_gbs": hbm, "pairs_K": K, "visible_Nv": nv, "pixels_P": P},
            "roofline": roof, "kernels": kernels, "gpu_launches": gpu_launches,
            "alu_peaks_measured": {"fp32_fma_tops": round(alu_peak, 3), "ex2_tops": round(sfu_peak, 3),
                                   "derived_fp32_lanes_at_max_clock": round(ALU_LANES * float(
                                       peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12, 3)},
            "kernel_timing": {"how": "same steps, kernels launched directly by the library with a CUDA event "
                                     "pair around each on its stream; value above is from CUDA-graph replay",
                              "ms_per_step_direct": round(t_direct / args.steps, 4)},
            "e2e": {"value": round(replica_throughput(args.iters, args.steps, world, t_e2e), 2), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clk}
    bf16 = float(peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    learned["roofline"] = {"bound": "tensor", "achieved": learned["infer_tflops"], "peak": bf16, "unit": "TFLOP/s",
                           "frac": round(learned["infer_tflops"] / bf16, 4),
                           "peak_source": f"{src} bf16_tflops (burst: the launch is timed alone)"}
    # the tensor core's rate by MMA width (the network's layers are 32
    # channels wide: its MMAs are M = 128 pixels x N = 32 x K = 16), measured
    # on this device by the library's probe
    rates = {}
    for n_cols, groups in ((32, 4), (64, 4), (128, 4), (256, 2)):
        rates[n_cols] = max(dags.measure_mma(n_cols, groups, 512)[0] for _ in range(2))
    # M = 64, the training step's weight-gradient MMAs (33 real rows)
    m64 = {n_cols: max(dags.measure_mma(n_cols, 4, 512, m_rows=64)[0] for _ in range(2)) for n_cols in (32, 64)}
    top = max(rates.values())
    # the probe's rates as TFLOP/s of the whole device at the maximum SM clock
    sms = int(torch.cuda.get_device_properties(0).multi_processor_count)
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n32_tflops = rates[32] * 2 * sms * mhz * 1e6 / 1e12
    learned["roofline"]["mma_rate_by_n"] = {
        "mac_per_sm_cycle": {str(k): round(v, 1) for k, v in rates.items()},
        "mac_per_sm_cycle_m64": {str(k): round(v, 1) for k, v in m64.items()},
        "n32_frac_of_best": round(rates[32] / top, 4),
        "n32_ceiling_tflops": round(n32_tflops, 1),
        "best_tflops": round(top * 2 * sms * mhz * 1e6 / 1e12, 1),
        "frac_of_n32_ceiling": round(learned["infer_tflops"] / n32_tflops, 4),
        "how": "dags_measure_mma: one CTA, back-to-back BF16 MMAs (M 128, K 16) from 4 warpgroups (2 at N 256); "
               "TFLOP/s = MAC/cycle x 2 x SMs x the maximum SM clock"}
    line["mp_update"] = mp_upd
    line["learned_mp"] = learned
    line["splat_variants"] = variants
    line["lm_tracking"] = lm
    if F >= 2:
        variants["edge_warp"] = edge_section(ctx, dags, gauss, cam, tg_all, pose_all, flush, stream)
    variants["epipolar_verify"] = epipolar_section(dags, flush, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline_all_cores(args, args.cpu_seconds)
        line["cpu_baseline"]["single_core"] = oracle_baseline(args, min(args.cpu_seconds, 10.0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
