"""Learned MP proposal against the method without it (used by the tests and
the bench).

Between scheduled semantic invocations (every REFRESH frames) the plain
update reuses the last instance prior (stale) with its rate scaled by rho,
Eq. (17). The learned network proposes the per-pixel MP from the frame's
rendered MP, residuals, depth, opacity and the stale prior. The fresh-prior arm is the
plain method itself with a fresh prior at every frame. The network is trained
on the GPU, by the library's own kernels, on the fresh-prior arm's per-pixel maps of a
training sequence, then evaluated on a held-out sequence with other
Gaussians, other noise and other object motions. Both the plain and the
learned arm also run with the semantic-on-demand trigger of Eqs. (13)-(16)
deciding the refreshes instead of the fixed cadence.

Synthetic stand-in for an indoor RGB-D sequence: the analytic room of
synth.room_scene at 320 x 240 (f = 262.5, the 640 x 480 field of view), two
moving ellipsoids at 0.3 m/s at 30 Hz, the map holding the objects at their
frame-0 positions, the camera on synth.camera_path at the ground-truth pose,
instance masks of the moving objects with 5% pixel flips.
"""
from __future__ import annotations

import numpy as np
import torch

from . import synth

W, H = 320, 240
N_GAUSS = 80_000
REFRESH = 10
TABLE = np.array([[0.1, 0.05], [0.9, 0.8], [0.9, 0.8]], np.float32)


def objects(velocities):
    objs = synth.default_objects()
    for ob, v in zip(objs, velocities):
        ob.velocity = np.asarray(v, np.float64)
    return objs


class Sequence:
    """Frames of the room with moving objects: observed RGB-D and noisy
    instance masks (label k for the k-th moving object)."""

    def __init__(self, seed, velocities, n_frames, width=W, height=H, n_gauss=N_GAUSS):
        self.width, self.height, self.n = width, height, n_gauss
        self.objs = objects(velocities)
        self.rec, self.oid, _ = synth.room_scene(n_gauss, seed, objects=self.objs)
        self.rec[:, 11] = 0.2                      # uninformed initial MP
        moving = [k for k, ob in enumerate(self.objs) if np.any(ob.velocity != 0)]
        self.dynamic = np.isin(self.oid, moving)
        self.velocity = np.zeros((n_gauss, 3), np.float32)
        for k, ob in enumerate(self.objs):
            self.velocity[self.oid == k] = ob.velocity
        f = 525.0 * width / 640.0                  # the 640x480 rig's field of view
        self.cam = synth.Camera(f, f, width / 2.0, height / 2.0, width, height)
        self.poses = synth.camera_path(n_frames)
        rng = np.random.default_rng(seed + 100)
        self.obs, self.inst = [], []
        for f in range(n_frames):
            tg, hit = synth.raycast(self.cam, self.poses[f], self.objs, f / 30.0, 0.01, rng)
            tg[(tg[:, 3] < 0.5) | (tg[:, 3] > 5.0), 3] = 0.0
            inst = np.zeros(hit.shape, np.uint8)
            for lab, k in enumerate(moving, start=1):
                inst[hit == k] = lab
            fl = rng.random(inst.shape) < 0.05
            repl = rng.integers(0, len(moving) + 1, inst.shape).astype(np.uint8)
            same = repl == inst
            repl[same] = (repl[same] + 1) % (len(moving) + 1)
            self.obs.append(tg)
            self.inst.append(np.where(fl, repl, inst).astype(np.uint8))


class Runner:
    """One sequence through the library: render, MP update (fresh, stale or
    learned), network features and inference."""

    def __init__(self, dags, seq, mp_cfg=None):
        self.d, self.seq = dags, seq
        self.mp_cfg = mp_cfg
        self.cam = dags.Camera(*seq.cam.as_tuple())
        self.ctx = dags.Context(seq.n, seq.width, seq.height, 1)
        self.table = torch.from_numpy(TABLE).cuda()
        self.P = seq.width * seq.height

    def frame_inputs(self, f):
        pose = torch.from_numpy(np.ascontiguousarray(self.seq.poses[f])[None]).cuda()
        tg = torch.from_numpy(self.seq.obs[f]).cuda()
        return pose, tg

    def render(self, gauss, pose):
        image, _, _ = self.ctx.forward(gauss, self.cam, pose)
        return image[0].reshape(8, self.P).contiguous()

    def fresh_map(self, gauss, pose, tg, image, f):
        """The fresh-prior arm's per-pixel M_p (fresh prior) at frame f."""
        g = gauss.clone()
        lab = torch.zeros(self.seq.n, dtype=torch.uint8, device="cuda")
        out = torch.empty(self.P, dtype=torch.float32, device="cuda")
        inst = torch.from_numpy(self.seq.inst[f]).cuda()
        self.ctx.mp_update(g, self.cam, pose, tg, image, inst, self.table, lab, mp_pixel=out, cfg=self.mp_cfg)
        return out

    def run(self, mode, net=None, collect=False, schedule=None, follow=False, score_only=False):
        """mode: 'fresh' (fresh prior every frame), 'stale' (the method without
        the network), 'learned' (network proposal between refreshes).
        Refreshes come every REFRESH frames, or from the semantic-on-demand
        trigger (Eqs. (13)-(16)) when schedule (a dags_sched_cfg) is given.
        follow: the map's moving-object Gaussians are placed at their frame's
        positions before each frame (a map that mapping keeps up to date), so
        that the frame's residuals come from the observation noise only.
        score_only (with schedule): the trigger scores every frame but the
        refreshes keep the fixed cadence."""
        gauss = torch.from_numpy(self.seq.rec.copy()).cuda()
        base = gauss[:, 0:3].clone()
        vel = torch.from_numpy(self.seq.velocity).cuda()
        labels = torch.zeros(self.seq.n, dtype=torch.uint8, device="cuda")
        state = torch.zeros(2, dtype=torch.int32, device="cuda")
        score = torch.zeros(3, dtype=torch.float64, device="cuda")
        hist = []
        nxt, last_ref = True, 0
        for f in range(len(self.seq.poses)):
            pose, tg = self.frame_inputs(f)
            if follow:
                gauss[:, 0:3] = base + vel * (f / 30.0)
            image = self.render(gauss, pose)
            if mode == "fresh":
                refreshed = True
            elif schedule is not None and not score_only:
                refreshed = nxt
            else:
                refreshed = f % REFRESH == 0
            if refreshed:
                last_ref = f
            inst = torch.from_numpy(self.seq.inst[last_ref]).cuda()
            rec = {"refreshed": refreshed}
            if collect or (mode == "learned" and not refreshed):
                feats = self.ctx.mpnet_features(image, tg, inst, self.table, self.cam)
                rec["feats"] = feats
            if collect:
                rec["target"] = self.fresh_map(gauss, pose, tg, image, f)
            mp_map = None
            if mode == "learned" and not refreshed:
                mp_map = self.ctx.mpnet_infer(net, rec["feats"][None]).reshape(-1)
                rec["net"] = mp_map
            stale_px = torch.empty(self.P, dtype=torch.float32, device="cuda")
            stats = self.ctx.mp_update(gauss, self.cam, pose, tg, image, inst, self.table, labels,
                                       seg_refreshed=refreshed, mp_map=mp_map, mp_pixel=stale_px, cfg=self.mp_cfg)
            if schedule is not None:
                self.ctx.semantic_trigger(stats, state, refreshed, cfg=schedule, score=score)
                nxt = bool(state[1].item())
                rec["score"] = score.clone()
            rec["pixel"] = stale_px
            rec["labels"] = labels.clone()
            hist.append(rec)
        torch.cuda.synchronize()
        self.ctx.check()
        return hist


def train_net(dags, runner, steps=1000, lr=2e-3, batch=16, seed=0, follow=False):
    """Adam training on the fresh-prior maps of the runner's sequence; returns
    (weight blob, per-step losses)."""
    hist = runner.run("stale", collect=True, follow=follow)
    feats = torch.stack([h["feats"] for h in hist])                    # [T, H, W, 8]
    target = torch.stack([h["target"].reshape(runner.seq.height, runner.seq.width) for h in hist])
    return train_on(runner.ctx, feats, target, steps, lr, batch, seed)


def train_on(ctx, feats, target, steps=1000, lr=2e-3, batch=16, seed=0):
    """Adam training of a seeded network on (feats [T, H, W, 8] bf16, target
    [T, H, W] f32), batches of `batch` frames drawn without replacement per
    step; returns (weight blob, per-step losses)."""
    blob, vec = synth.mpnet_init(seed)
    net = torch.from_numpy(blob).cuda()
    master = torch.from_numpy(vec).cuda()
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    gen = torch.Generator().manual_seed(seed)
    losses = []
    for step in range(1, steps + 1):
        idx = torch.randperm(feats.shape[0], generator=gen)[:batch].cuda()
        fb = feats.index_select(0, idx).contiguous()
        tb = target.index_select(0, idx).contiguous()
        losses.append(ctx.mpnet_train_step(net, master, m, v, step, fb, tb, lr))
    torch.cuda.synchronize()
    ctx.check()
    return net, [l.item() for l in losses]


def iou(a, b):
    u = np.logical_or(a, b).sum()
    return np.logical_and(a, b).sum() / u if u else 1.0


def calibrate_schedule(dags, runner, follow=False):
    """The trigger's constants (Eqs. (14)-(16)) fitted to a training sequence
    run with the fixed cadence: e_ref is twice the largest mean background
    residual at any prior age, so that R = e_bar / e_ref stays below 1/2
    and follows the residual instead of saturating; theta lies halfway
    between the mean score S of the frames with a fresh prior and of those
    REFRESH - 1 frames after a refresh, so that the trigger fires once the
    stale prior has cost half of what a full interval costs. Returns
    (dags_sched_cfg, dict of the fitted statistics)."""
    base = dags.default_sched_cfg()
    hist = runner.run("stale", schedule=base, score_only=True, follow=follow)
    age = np.array([f % REFRESH for f in range(len(hist))])
    e_bar = np.array([h["score"][0].item() for h in hist])
    e_ref = 2.0 * max(e_bar[age == a].mean() for a in range(REFRESH))
    cfg = dags.default_sched_cfg(e_ref=float(e_ref))
    hist = runner.run("stale", schedule=cfg, score_only=True, follow=follow)
    S = np.array([h["score"][2].item() for h in hist])
    s0, s9 = S[age == 0].mean(), S[age == REFRESH - 1].mean()
    cfg.theta = float(s0 + 0.5 * (s9 - s0))
    return cfg, {"e_ref": float(e_ref), "theta": cfg.theta, "S_fresh": float(s0), "S_stale": float(s9)}


def experiment(dags, steps=1000, follow=False, mp_cfg=None):
    """Train on one sequence, run fresh / stale / learned on the held-out one.
    follow: the map keeps its moving objects at their current positions (see
    Runner.run), in training and evaluation; mp_cfg: the MP update's
    constants (default dags_default_mp_cfg)."""
    train_seq = Sequence(seed=11, velocities=[(0.0, 0.0, 0.3), (-0.3, 0.0, 0.0)], n_frames=60)
    tr = Runner(dags, train_seq, mp_cfg)
    net, losses = train_net(dags, tr, steps=steps, follow=follow)
    cal, cal_stats = calibrate_schedule(dags, tr, follow=follow)
    tr.ctx.close()
    eval_seq = Sequence(seed=12, velocities=[(0.3, 0.0, 0.0), (0.0, 0.0, 0.3)], n_frames=40)
    ev = Runner(dags, eval_seq, mp_cfg)
    sc = dags.default_sched_cfg()
    out = dict(losses=losses, fresh=ev.run("fresh", follow=follow), stale=ev.run("stale", follow=follow),
               learned=ev.run("learned", net=net, follow=follow),
               scheduled=ev.run("stale", schedule=sc, follow=follow),
               scheduled_learned=ev.run("learned", net=net, schedule=sc, follow=follow),
               calibrated=ev.run("stale", schedule=cal, follow=follow),
               calibrated_learned=ev.run("learned", net=net, schedule=cal, follow=follow),
               calibration=cal_stats, seq=eval_seq)
    ev.ctx.close()
    return out


def metrics(ex):
    """Means over the held-out frames between refreshes: per-pixel MP against
    the fresh-prior map (MAE, IoU of M > 0.5) and dynamic-label IoU with the
    fresh-prior labels and with the ground-truth dynamic Gaussians."""
    j, s, l = ex["fresh"], ex["stale"], ex["learned"]
    gt = ex["seq"].dynamic
    acc = {k: [] for k in ("mae_s", "mae_l", "iou_s", "iou_l", "agree_s", "agree_l", "gt_j", "gt_s", "gt_l")}
    for f in range(len(j)):
        if f % REFRESH == 0:
            continue
        ref = j[f]["pixel"].cpu().numpy()
        ps = s[f]["pixel"].cpu().numpy()
        pl = l[f]["net"].cpu().numpy()
        acc["mae_s"].append(np.abs(ps - ref).mean())
        acc["mae_l"].append(np.abs(pl - ref).mean())
        acc["iou_s"].append(iou(ps > 0.5, ref > 0.5))
        acc["iou_l"].append(iou(pl > 0.5, ref > 0.5))
        lj = j[f]["labels"].cpu().numpy() == 1
        ls = s[f]["labels"].cpu().numpy() == 1
        ll = l[f]["labels"].cpu().numpy() == 1
        acc["agree_s"].append(iou(ls, lj))
        acc["agree_l"].append(iou(ll, lj))
        acc["gt_j"].append(iou(lj, gt))
        acc["gt_s"].append(iou(ls, gt))
        acc["gt_l"].append(iou(ll, gt))
    m = {k: float(np.mean(v)) for k, v in acc.items()}
    L = ex["losses"]
    m["loss_first"] = float(np.mean(L[:5]))
    m["loss_last"] = float(np.mean(L[-20:]))
    return m


def schedule_metrics(ex):
    """The semantic-on-demand trigger against the fixed cadence on the
    held-out sequence: segmentation calls, and over frames 1.. the per-pixel
    MP MAE against the fresh-prior arm and the label IoU with the fresh-prior labels (the
    learned proposal's map where it stands in for M_p)."""
    j = ex["fresh"]
    out = {}
    for name in ("stale", "scheduled", "learned", "scheduled_learned", "calibrated", "calibrated_learned"):
        if name not in ex:
            continue
        h = ex[name]
        mae, agree = [], []
        for f in range(1, len(j)):
            ref = j[f]["pixel"].cpu().numpy()
            px = (h[f]["net"] if "net" in h[f] else h[f]["pixel"]).cpu().numpy()
            mae.append(np.abs(px - ref).mean())
            agree.append(iou(h[f]["labels"].cpu().numpy() == 1, j[f]["labels"].cpu().numpy() == 1))
        out[name] = {"calls": int(sum(r["refreshed"] for r in h)), "mp_mae": float(np.mean(mae)),
                     "label_iou_vs_fresh_prior": float(np.mean(agree))}
        if "score" in h[0]:
            out[name]["mean_S"] = float(np.mean([r["score"][2].item() for r in h]))
    return out


def rendered_training_set(dags, n_frames=10_000, n_gauss=200_000, width=640, height=480, seed=0, flip=0.05,
                          max_stale=9, fps=30.0):
    """Training frames the plain method generates on the mapping room (200k
    Gaussians, 640x480), with the observations rendered by the library
    instead of ray-cast (ray-casting 10k frames on the host would take hours).

    Per frame, seeded: a viewpoint inside the room looking across it; an
    object time t (the two moving objects displaced by v t) and a stale time
    t - k / fps, k in 1..max_stale (the prior of the last refresh);
      observation  the render of the displaced scene, colour + N(0, 0.01),
                   depth x (1 + N(0, 0.01)) where opacity > 0.5 and depth in
                   0.5-5 m (else invalid)
      instance maps renders whose MP channel carries the object label (fresh
                   at t, stale at t - k / fps), `flip` pixel flips
      map render   the map as the tracker holds it (objects at their t = 0
                   positions) with per-frame MP words (0.2 plus a random
                   separation of the moving objects' Gaussians)
      target       the plain method's fused M_p with the fresh prior
                   (mp_update's per-pixel output)
      features     mpnet_features with the stale prior.
    Returns (feats [T, H, W, 8] bf16, target [T, H, W] f32), on the device."""
    rec, oid, objs = synth.room_scene(n_gauss, seed)
    cam_s = synth.room_camera(width, height)
    cam = dags.Camera(*cam_s.as_tuple())
    P = width * height
    moving = [k for k, ob in enumerate(objs) if np.any(ob.velocity != 0)]
    L = len(moving)
    dev = "cuda"
    base = torch.from_numpy(rec).to(dev)
    idx = [torch.from_numpy(np.nonzero(oid == k)[0]).to(dev) for k in moving]
    vel = [torch.tensor(objs[k].velocity, dtype=torch.float32, device=dev) for k in moving]
    dyn = torch.from_numpy(np.isin(oid, moving)).to(dev)
    table = torch.from_numpy(np.array([[0.1, 0.05]] + [[0.9, 0.8]] * L, np.float32)).to(dev)
    ctx = dags.Context(n_gauss, width, height, 1)
    feats = torch.empty((n_frames, height, width, 8), dtype=torch.bfloat16, device=dev)
    target = torch.empty((n_frames, height, width), dtype=torch.float32, device=dev)
    work = base.clone()
    labels = torch.zeros(n_gauss, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(seed + 4242)
    gen = torch.Generator(device=dev).manual_seed(seed + 4243)

    def displaced(t, label_mp):
        work.copy_(base)
        if label_mp:
            work[:, 11] = 0.0
        for j in range(L):
            work[idx[j], 0:3] += vel[j] * t
            if label_mp:
                work[idx[j], 11] = (j + 1) / L
        return work

    def instance(t):
        im, _, _ = ctx.forward(displaced(t, True), cam, pose_d[None], want_loss=False)
        o = im[0, 4].reshape(P)
        lab = torch.where(o > 0.5, torch.round(im[0, 5].reshape(P) / o.clamp_min(1e-6) * L), torch.zeros_like(o))
        lab = lab.clamp(0, L).to(torch.uint8)
        fl = torch.rand(P, generator=gen, device=dev) < flip
        repl = torch.randint(0, L + 1, (P,), generator=gen, device=dev, dtype=torch.uint8)
        repl = torch.where(repl == lab, (repl + 1) % (L + 1), repl)
        return torch.where(fl, repl, lab).contiguous()

    for f in range(n_frames):
        a = rng.uniform(0, 2 * np.pi)
        r = rng.uniform(1.0, 1.8)
        eye = np.array([r * np.cos(a), rng.uniform(-0.5, 0.1), r * np.sin(a)])
        b = a + rng.uniform(-0.6, 0.6)
        look = np.array([-0.6 * np.cos(b), rng.uniform(0.2, 0.6), -0.6 * np.sin(b)])
        pose_d = torch.from_numpy(synth.look_at_pose(eye, look)).to(dev)
        t = rng.uniform(0.2, 3.0)
        t_stale = t - rng.integers(1, max_stale + 1) / fps
        # observation of the displaced scene
        im, _, _ = ctx.forward(displaced(t, False), cam, pose_d[None], want_loss=False)
        c = im[0, 0:3].reshape(3, P).t()
        d = im[0, 3].reshape(P)
        o = im[0, 4].reshape(P)
        tg = torch.empty((P, 4), dtype=torch.float32, device=dev)
        tg[:, 0:3] = (c + 0.01 * torch.randn((P, 3), generator=gen, device=dev)).clamp(0, 1)
        dn = d * (1 + 0.01 * torch.randn(P, generator=gen, device=dev))
        tg[:, 3] = torch.where((o > 0.5) & (dn > 0.5) & (dn < 5.0), dn, torch.zeros_like(dn))
        inst_fresh = instance(t)
        inst_stale = instance(t_stale)
        # the map as tracked, its MP words, its render
        work.copy_(base)
        sep = float(rng.uniform(0.0, 0.7))
        work[:, 11] = (0.2 + sep * dyn.float() + 0.1 * torch.randn(n_gauss, generator=gen, device=dev)).clamp(0, 1)
        image, _, _ = ctx.forward(work, cam, pose_d[None], want_loss=False)
        img = image[0].reshape(dags.IMG_CHANNELS, P)
        ctx.mpnet_features(img, tg, inst_stale, table, cam, out=feats[f])
        ctx.mp_update(work, cam, pose_d[None], tg, img, inst_fresh, table, labels, mp_pixel=target[f].reshape(P))
    torch.cuda.synchronize()
    ctx.check()
    ctx.close()
    return feats, target


def experiment_rendered(dags, n_frames=10_000, steps=3000, lr=2e-3, batch=16, width=640, height=480,
                        eval_frames=40):
    """Train on `n_frames` rendered training frames (rendered_training_set),
    then run fresh / stale / learned on a held-out ray-cast sequence at the
    same resolution (other Gaussians, other object motions)."""
    import time
    t0 = time.perf_counter()
    feats, target = rendered_training_set(dags, n_frames, width=width, height=height)
    t_gen = time.perf_counter() - t0
    tctx = dags.Context(16, width, height, 1)
    t0 = time.perf_counter()
    net, losses = train_on(tctx, feats, target, steps, lr, batch)
    t_train = time.perf_counter() - t0
    tctx.close()
    del feats, target
    torch.cuda.empty_cache()
    eval_seq = Sequence(seed=12, velocities=[(0.3, 0.0, 0.0), (0.0, 0.0, 0.3)], n_frames=eval_frames,
                        width=width, height=height, n_gauss=200_000)
    ev = Runner(dags, eval_seq)
    out = dict(losses=losses, fresh=ev.run("fresh"), stale=ev.run("stale"), learned=ev.run("learned", net=net),
               seq=eval_seq, t_gen=t_gen, t_train=t_train)
    ev.ctx.close()
    return out
