"""The seeded input generators (paper_2602_21644_gb300/synth.py) that both the
CUDA path's tests and the oracle's consume: determinism per seed, the stated
recipe (surfaces, speeds, flip rate, field of view, the closed camera loop),
and the conventions the generator shares with the oracle (ray-cast depth is
camera z; a noise-free static match lies on its epipolar line, Eq. (18))."""
import numpy as np

from oracle import epipolar as E
from paper_2602_21644_gb300 import synth


def same(a, b):
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(same(a[k], b[k]) for k in a)
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    if isinstance(a, synth.Camera):
        return a.as_tuple() == b.as_tuple()
    if isinstance(a, np.ndarray):
        return a.dtype == b.dtype and np.array_equal(a, b)
    if isinstance(a, synth.Ellipsoid):
        return all(np.array_equal(getattr(a, f), getattr(b, f)) for f in ("center", "axes", "velocity"))
    return a == b


def test_generators_are_deterministic_per_seed():
    small = dict(n=20_000, width=96, height=72)
    cases = [
        lambda s: synth.tiny_scene(s).records,
        lambda s: synth.tiny_scene(s).targets,
        lambda s: synth.room_scene(20_000, s)[:2],
        lambda s: synth.tracking_scene(frame=3, seed=s, **small).targets,
        lambda s: synth.tracking_sequence(frames=range(2, 4), seed=s, **small)[2],
        lambda s: synth.full_loop_sequence(frames=range(0, 2), seed=s, n=20_000, width=120, height=68)[2],
        lambda s: synth.epipolar_matches(seed=s, n=20_000, n_sample=300),
        lambda s: synth.spline_path(12, seed=s),
        lambda s: synth.mpnet_init(s),
    ]
    for k, make in enumerate(cases):
        assert same(make(0), make(0)), f"case {k} differs between two calls with one seed"
        assert not same(make(0), make(1)), f"case {k} ignores its seed"


def test_room_gaussians_lie_on_their_surfaces():
    rec, oid, objs = synth.room_scene(30_000, 2)
    assert rec.shape == (30_000, 16) and rec.dtype == np.float32
    mu = rec[:, 0:3].astype(np.float64)
    walls = oid < 0
    # a wall Gaussian has one coordinate on the room's boundary
    on = np.abs(np.abs(mu[walls]) - synth.ROOM_HALF) <= 1e-6 * synth.ROOM_HALF
    assert np.all(on.any(axis=1))
    assert np.all(np.abs(mu[walls]) <= synth.ROOM_HALF * (1 + 1e-6))
    for j, ob in enumerate(objs):
        q = (mu[oid == j] - ob.center) / ob.axes
        assert np.abs(np.sum(q * q, axis=1) - 1.0).max() < 1e-5
    # unit quaternions, MP 0.9 on the moving objects and 0.1 elsewhere, colours in [0, 1]
    assert np.allclose(np.linalg.norm(rec[:, 4:8], axis=1), 1.0, atol=1e-6)
    moving = np.array([np.any(ob.velocity != 0) for ob in objs])
    dyn = (oid >= 0) & moving[np.maximum(oid, 0)]
    assert np.all(rec[dyn, 11] == np.float32(0.9)) and np.all(rec[~dyn, 11] == np.float32(0.1))
    rgb = synth.record_rgb(rec)
    assert rgb.min() >= 0.0 and rgb.max() <= 1.0
    # the default objects: two move at 0.3 m/s, one is static
    speeds = sorted(float(np.linalg.norm(ob.velocity)) for ob in objs)
    assert np.allclose(speeds, [0.0, 0.3, 0.3])


def test_raycast_depth_is_camera_z():
    # a camera at the room's centre looking along +z sees only the far wall
    # (z = 3 m) at 640x480, f = 525: every pixel's depth is exactly 3
    cam = synth.room_camera()
    pose = synth.look_at_pose([0.0, 0.0, 0.0], [0.0, 0.0, 1.0])
    tg, hit = synth.raycast(cam, pose, [], 0.0)
    assert np.all(hit == -1)
    np.testing.assert_allclose(tg[:, 3], 3.0, rtol=0, atol=1e-6)
    # moved 1 m towards the wall, the depth drops by 1 m everywhere
    pose2 = synth.look_at_pose([0.0, 0.0, 1.0], [0.0, 0.0, 2.0])
    tg2, _ = synth.raycast(cam, pose2, [], 0.0)
    np.testing.assert_allclose(tg2[:, 3], 2.0, rtol=0, atol=1e-6)


def test_tracking_frames_and_flip_rate():
    small = dict(n=20_000, width=160, height=120)
    rec, cam, seq, ex = synth.tracking_sequence(frames=range(4, 7), **small)
    for a, b in zip(seq[:-1], seq[1:]):
        assert np.array_equal(b["pose"], a["gt_pose"])        # each frame starts from the previous pose
    one = synth.tracking_scene(frame=5, **small)
    assert np.array_equal(one.targets[0], seq[1]["target"]) and np.array_equal(one.extra["instance"], seq[1]["instance"])
    # 5 % of the instance labels are flipped, each to another label
    clean = synth.tracking_scene(frame=5, flip=0.0, **small).extra["instance"]
    frac = np.mean(clean != one.extra["instance"])
    assert abs(frac - 0.05) < 0.008
    assert set(np.unique(one.extra["instance"])) <= set(range(ex["n_instances"] + 1))


def test_full_loop_camera_and_objects():
    rec, cam, seq, ex = synth.full_loop_sequence(frames=range(0, 2), n=20_000, width=1200, height=680)
    # the 640x480 rig's horizontal field of view at 1200 px
    assert cam.as_tuple() == (525.0 * 1200 / 640, 525.0 * 1200 / 640, 600.0, 340.0, 1200, 680)
    assert ex["n_instances"] == 3 and len(ex["objects"]) == 4
    assert np.array_equal(ex["dynamic"], np.isin(ex["object_id"], [0, 1, 2]))
    assert seq[0]["target"].shape == (1200 * 680, 4)


def test_spline_path_closes_after_ten_seconds():
    poses = synth.spline_path(301)                             # 30 fps: frame 300 is t = 10 s
    np.testing.assert_allclose(poses[300], poses[0], rtol=0, atol=1e-12)
    assert not np.allclose(poses[150], poses[0])
    for T in poses[::37]:
        R = T[:, :3]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)


def test_noise_free_static_matches_lie_on_their_epipolar_lines():
    m = synth.epipolar_matches(n=40_000, n_sample=2_000, noise_px=0.0, suppressed=0.0)
    cam = m["camera"].as_tuple()
    d = E.distances(E.fundamental(cam, m["pose_1"], m["pose_2"]), m["p1"].astype(np.float64),
                    m["p2"].astype(np.float64))
    static = ~m["moving"][m["gid"]]
    assert static.sum() > 1000 and (~static).sum() > 0
    # only the float32 rounding of the pixel coordinates remains
    assert d[static].max() < 1e-3
    # the moving objects' matches leave their lines (5 frames at 0.3 m/s)
    assert np.median(d[~static]) > 0.5
    # 4 matches per Gaussian; labels: the moving ones dynamic, none suppressed
    assert np.all(np.bincount(m["gid"])[np.unique(m["gid"])] == 4)
    assert np.array_equal(m["labels"].astype(bool), m["moving"])
