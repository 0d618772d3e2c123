"""What the learned MP proposal gains over the method without it.

Between scheduled semantic invocations (every 10 frames) the plain update
reuses the last instance prior (stale) with its rate scaled by rho, Eq. (17).
The learned network proposes the per-pixel MP from the frame's rendered MP,
residuals, depth, opacity and the stale prior. The judge is the plain method
itself with a fresh prior at every frame. The network is trained (on the GPU,
by the project's own kernels) on the judge's per-pixel maps of a training
sequence, then evaluated on a held-out sequence with other Gaussians, other
noise and other object motions.

Synthetic stand-in for an indoor RGB-D sequence: the analytic room of
synth.room_scene at 320 x 240 (f = 262.5, the 640 x 480 field of view), two
moving ellipsoids at 0.3 m/s at 30 Hz, the map holding the objects at their
frame-0 positions, the camera on synth.camera_path at the ground-truth pose,
instance masks of the moving objects with 5% pixel flips."""
import numpy as np
import pytest

from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W, H, F = 320, 240, 262.5
N_GAUSS = 80_000
REFRESH = 10
TABLE = np.array([[0.1, 0.05], [0.9, 0.8], [0.9, 0.8]], np.float32)


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def objects(velocities):
    objs = synth.default_objects()
    for ob, v in zip(objs, velocities):
        ob.velocity = np.asarray(v, np.float64)
    return objs


class Sequence:
    """Frames of the room with moving objects: observed RGB-D and noisy
    instance masks (label k for the k-th moving object)."""

    def __init__(self, seed, velocities, n_frames):
        self.objs = objects(velocities)
        self.rec, self.oid, _ = synth.room_scene(N_GAUSS, seed, objects=self.objs)
        self.rec[:, 11] = 0.2                      # uninformed initial MP
        moving = [k for k, ob in enumerate(self.objs) if np.any(ob.velocity != 0)]
        self.dynamic = np.isin(self.oid, moving)
        self.cam = synth.Camera(F, F, W / 2.0, H / 2.0, W, H)
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
    def __init__(self, dags, seq):
        self.d, self.seq = dags, seq
        self.cam = dags.Camera(*seq.cam.as_tuple())
        self.ctx = dags.Context(N_GAUSS, W, H, 1)
        self.table = torch.from_numpy(TABLE).cuda()
        self.P = W * H

    def frame_inputs(self, f):
        pose = torch.from_numpy(np.ascontiguousarray(self.seq.poses[f])[None]).cuda()
        tg = torch.from_numpy(self.seq.obs[f]).cuda()
        return pose, tg

    def render(self, gauss, pose):
        image, _, _ = self.ctx.forward(gauss, self.cam, pose)
        return image[0].reshape(8, self.P).contiguous()

    def fresh_map(self, gauss, pose, tg, image, f):
        """The judge's per-pixel M_p (fresh prior) at frame f."""
        g = gauss.clone()
        lab = torch.zeros(N_GAUSS, dtype=torch.uint8, device="cuda")
        out = torch.empty(self.P, dtype=torch.float32, device="cuda")
        inst = torch.from_numpy(self.seq.inst[f]).cuda()
        self.ctx.mp_update(g, self.cam, pose, tg, image, inst, self.table, lab, mp_pixel=out)
        return out

    def run(self, mode, net=None, collect=False):
        """mode: 'judge' (fresh prior every frame), 'stale' (the method without
        the network), 'learned' (network proposal between refreshes)."""
        gauss = torch.from_numpy(self.seq.rec.copy()).cuda()
        labels = torch.zeros(N_GAUSS, dtype=torch.uint8, device="cuda")
        hist = []
        for f in range(len(self.seq.poses)):
            pose, tg = self.frame_inputs(f)
            image = self.render(gauss, pose)
            refreshed = f % REFRESH == 0 or mode == "judge"
            inst = torch.from_numpy(self.seq.inst[f if refreshed else f - f % REFRESH]).cuda()
            rec = {}
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
            self.ctx.mp_update(gauss, self.cam, pose, tg, image, inst, self.table, labels,
                               seg_refreshed=refreshed, mp_map=mp_map, mp_pixel=stale_px)
            rec["pixel"] = stale_px
            rec["labels"] = labels.clone()
            hist.append(rec)
        torch.cuda.synchronize()
        self.ctx.check()
        return hist


def train_net(dags, runner, steps=1000, lr=2e-3, batch=16, seed=0):
    from oracle import mpnet as N          # initial weights only (a seeded draw)
    hist = runner.run("stale", collect=True)
    feats = torch.stack([h["feats"] for h in hist])                    # [T, H, W, 8]
    target = torch.stack([h["target"].reshape(H, W) for h in hist])    # [T, H, W]
    p = N.init_params(seed)
    w = N.pack_weights(p)
    blob = np.zeros(22016, np.uint8)
    blob[0:1024] = synth.f32_to_bf16_bits(np.asarray(w["W1"], np.float32)).view(np.uint8).ravel()
    blob[1024:19456] = synth.f32_to_bf16_bits(np.asarray(w["W2"], np.float32)).view(np.uint8).ravel()
    blob[19456:21504] = synth.f32_to_bf16_bits(np.asarray(w["W3"], np.float32)).view(np.uint8).ravel()
    blob[21504:21568] = synth.f32_to_bf16_bits(np.asarray(w["w4"], np.float32)).view(np.uint8).ravel()
    vec = np.zeros(10881, np.float32)
    vec[0:512] = np.asarray(w["W1"], np.float32).ravel()
    vec[512:9728] = np.asarray(w["W2"], np.float32).ravel()
    vec[9728:10752] = np.asarray(w["W3"], np.float32).ravel()
    vec[10752:10784] = np.asarray(w["w4"], np.float32).ravel()
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
        losses.append(runner.ctx.mpnet_train_step(net, master, m, v, step, fb, tb, lr))
    torch.cuda.synchronize()
    runner.ctx.check()
    return net, [l.item() for l in losses]


def iou(a, b):
    u = np.logical_or(a, b).sum()
    return np.logical_and(a, b).sum() / u if u else 1.0


@pytest.fixture(scope="module")
def experiment(dags):
    train_seq = Sequence(seed=11, velocities=[(0.0, 0.0, 0.3), (-0.3, 0.0, 0.0)], n_frames=60)
    tr = Runner(dags, train_seq)
    net, losses = train_net(dags, tr)
    eval_seq = Sequence(seed=12, velocities=[(0.3, 0.0, 0.0), (0.0, 0.0, 0.3)], n_frames=40)
    ev = Runner(dags, eval_seq)
    judge = ev.run("judge")
    stale = ev.run("stale")
    learned = ev.run("learned", net=net)
    return dict(losses=losses, judge=judge, stale=stale, learned=learned, seq=eval_seq)


def test_training_converges(experiment):
    L = experiment["losses"]
    assert np.mean(L[-20:]) < 0.9 * np.mean(L[:5]), (L[:5], L[-20:])


def test_learned_map_closer_to_judge_than_stale_prior(experiment):
    # per-pixel MP between refreshes against the judge's fresh-prior map
    j, s, l = experiment["judge"], experiment["stale"], experiment["learned"]
    mae_s, mae_l, iou_s, iou_l = [], [], [], []
    for f in range(len(j)):
        if f % REFRESH == 0:
            continue
        ref = j[f]["pixel"].cpu().numpy()
        ps = s[f]["pixel"].cpu().numpy()
        pl = l[f]["net"].cpu().numpy()
        mae_s.append(np.abs(ps - ref).mean())
        mae_l.append(np.abs(pl - ref).mean())
        iou_s.append(iou(ps > 0.5, ref > 0.5))
        iou_l.append(iou(pl > 0.5, ref > 0.5))
    print(f"\npixel MP vs judge between refreshes: MAE stale {np.mean(mae_s):.4f} learned {np.mean(mae_l):.4f}; "
          f"IoU(>0.5) stale {np.mean(iou_s):.4f} learned {np.mean(iou_l):.4f}")
    assert np.mean(mae_l) < np.mean(mae_s)
    assert np.mean(iou_l) > np.mean(iou_s)


def test_label_agreement_and_ground_truth_iou(experiment):
    # static/dynamic labels of the Gaussians: agreement with the judge and IoU
    # against the synthetic ground-truth dynamic set, between refreshes
    j, s, l = experiment["judge"], experiment["stale"], experiment["learned"]
    gt = experiment["seq"].dynamic
    agree_s, agree_l, gt_j, gt_s, gt_l = [], [], [], [], []
    for f in range(len(j)):
        if f % REFRESH == 0:
            continue
        lj = j[f]["labels"].cpu().numpy() == 1
        ls = s[f]["labels"].cpu().numpy() == 1
        ll = l[f]["labels"].cpu().numpy() == 1
        agree_s.append(iou(ls, lj))
        agree_l.append(iou(ll, lj))
        gt_j.append(iou(lj, gt))
        gt_s.append(iou(ls, gt))
        gt_l.append(iou(ll, gt))
    print(f"\ndynamic-label IoU with the judge: stale {np.mean(agree_s):.4f} learned {np.mean(agree_l):.4f}; "
          f"vs ground truth: judge {np.mean(gt_j):.4f} stale {np.mean(gt_s):.4f} learned {np.mean(gt_l):.4f}")
    # the labels integrate the map over frames through Eq. (9) and the median
    # threshold, so the per-pixel gain shows only weakly here: it must not
    # lose agreement (training is not bit-reproducible: FP32 atomics)
    assert np.mean(agree_l) >= np.mean(agree_s) - 0.02
