"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by
the oracle's tests.

This module holds none of the method's arithmetic: it samples Gaussians,
packs them into the 64-byte record format, builds camera poses, and makes
ground-truth RGB-D frames by ray-casting the analytic scene (planes and
ellipsoids) that the Gaussians were sampled from. It never splats.

The paper evaluates on the TUM RGB-D and BONN sequences (Sec. V-A(a));
neither is available here, so these scenes stand in for them: 640x480
RGB-D frames with fx = fy = 525 of an indoor room with moving objects.

Record layout (16 x 32-bit words, 64 bytes, little endian):
  0-2 mean (m, world), 3 opacity logit, 4-7 rotation quaternion (w, x, y, z;
  any norm), 8-10 natural-log scale per axis, 11 motion probability,
  12 = bf16(r) | bf16(g) << 16, 13 = bf16(b), 14-15 zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RECORD_WORDS = 16


# ------------------------------------------------------------------ packing

def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest, ties to even); uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b).astype(np.uint32) << 16).view(np.float32)


def pack_records(means, logits, quats, logscales, mp, rgb) -> np.ndarray:
    """Pack per-Gaussian arrays into n x 16 float32 records (colours to BF16)."""
    n = means.shape[0]
    rec = np.zeros((n, RECORD_WORDS), dtype=np.float32)
    rec[:, 0:3] = means
    rec[:, 3] = logits
    rec[:, 4:8] = quats
    rec[:, 8:11] = logscales
    rec[:, 11] = mp
    bits = f32_to_bf16_bits(np.asarray(rgb, dtype=np.float32)).astype(np.uint32)
    words = rec.view(np.uint32)
    words[:, 12] = bits[:, 0] | (bits[:, 1] << 16)
    words[:, 13] = bits[:, 2]
    return rec


def record_rgb(rec: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(rec).view(np.uint32)
    r = bf16_bits_to_f32((w[:, 12] & 0xFFFF).astype(np.uint16))
    g = bf16_bits_to_f32((w[:, 12] >> 16).astype(np.uint16))
    b = bf16_bits_to_f32((w[:, 13] & 0xFFFF).astype(np.uint16))
    return np.stack([r, g, b], axis=1)


# ------------------------------------------------------------------ cameras

@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_tuple(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


def identity_pose() -> np.ndarray:
    p = np.zeros((3, 4))
    p[:, :3] = np.eye(3)
    return p


def look_at_pose(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World-to-camera 3x4 pose of a camera at eye looking at target
    (camera x right, y down, z forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, dtype=np.float64), f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=0)          # rows: camera axes in world
    pose = np.zeros((3, 4))
    pose[:, :3] = R
    pose[:, 3] = -R @ eye
    return pose


def rotmat_to_quat(R: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) of rotation matrices (..., 3, 3)."""
    R = np.asarray(R, dtype=np.float64)
    m00, m11, m22 = R[..., 0, 0], R[..., 1, 1], R[..., 2, 2]
    tr = m00 + m11 + m22
    q = np.zeros(R.shape[:-2] + (4,))
    c0 = tr > 0
    s = np.sqrt(np.maximum(tr + 1.0, 1e-12)) * 2
    q0 = np.stack([0.25 * s, (R[..., 2, 1] - R[..., 1, 2]) / s, (R[..., 0, 2] - R[..., 2, 0]) / s,
                   (R[..., 1, 0] - R[..., 0, 1]) / s], -1)
    c1 = (~c0) & (m00 > m11) & (m00 > m22)
    s1 = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 1e-12)) * 2
    q1 = np.stack([(R[..., 2, 1] - R[..., 1, 2]) / s1, 0.25 * s1, (R[..., 0, 1] + R[..., 1, 0]) / s1,
                   (R[..., 0, 2] + R[..., 2, 0]) / s1], -1)
    c2 = (~c0) & (~c1) & (m11 > m22)
    s2 = np.sqrt(np.maximum(1.0 + m11 - m00 - m22, 1e-12)) * 2
    q2 = np.stack([(R[..., 0, 2] - R[..., 2, 0]) / s2, (R[..., 0, 1] + R[..., 1, 0]) / s2, 0.25 * s2,
                   (R[..., 1, 2] + R[..., 2, 1]) / s2], -1)
    s3 = np.sqrt(np.maximum(1.0 + m22 - m00 - m11, 1e-12)) * 2
    q3 = np.stack([(R[..., 1, 0] - R[..., 0, 1]) / s3, (R[..., 0, 2] + R[..., 2, 0]) / s3,
                   (R[..., 1, 2] + R[..., 2, 1]) / s3, 0.25 * s3], -1)
    q = np.where(c0[..., None], q0, np.where(c1[..., None], q1, np.where(c2[..., None], q2, q3)))
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


# ------------------------------------------------------------------ tiny

@dataclass
class Scene:
    records: np.ndarray                 # n x 16 float32
    camera: Camera
    poses: np.ndarray                   # V x 3 x 4 float64 (world -> camera)
    targets: np.ndarray                 # V x H*W x 4 float32 (r, g, b, depth; depth 0 = invalid)
    dynamic: np.ndarray = None          # n bool: Gaussian belongs to a moving object
    extra: dict = field(default_factory=dict)


def tiny_scene(seed: int = 0, n: int = 2000, width: int = 160, height: int = 120, f: float = 120.0,
               dyn_frac: float = 0.2) -> Scene:
    """2,000 anisotropic Gaussians: means U([-1,1]x[-1,1]x[1,4]) m, log-scales
    N(-3, 0.5), random unit quaternions, RGB U[0,1], opacity logit N(0,1); the
    first 20% re-drawn inside a 'dynamic' box with MP 0.9, the rest MP 0.1;
    one pinhole camera fx = fy = 120 at 160x120, identity pose; target RGB
    U[0,1] and depth U[1,4] per pixel."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 4, n)], 1)
    logscales = rng.normal(-3.0, 0.5, (n, 3))
    q = rng.normal(0, 1, (n, 4))
    quats = q / np.linalg.norm(q, axis=1, keepdims=True)
    rgb = rng.uniform(0, 1, (n, 3))
    logits = rng.normal(0, 1, n)
    nd = int(round(dyn_frac * n))
    means[:nd] = np.stack([rng.uniform(0.2, 0.8, nd), rng.uniform(-0.3, 0.3, nd), rng.uniform(1.5, 2.5, nd)], 1)
    mp = np.full(n, 0.1)
    mp[:nd] = 0.9
    dyn = np.zeros(n, bool)
    dyn[:nd] = True
    rec = pack_records(means, logits, quats, logscales, mp, rgb)
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    tg = np.zeros((1, width * height, 4), np.float32)
    tg[0, :, 0:3] = rng.uniform(0, 1, (width * height, 3))
    tg[0, :, 3] = rng.uniform(1, 4, width * height)
    return Scene(rec, cam, identity_pose()[None], tg, dyn)


# ------------------------------------------------------------------ room

ROOM_HALF = np.array([3.0, 1.5, 3.0])   # x, y (down), z half-extents: 6 x 3 x 6 m


@dataclass
class Ellipsoid:
    center: np.ndarray
    axes: np.ndarray
    velocity: np.ndarray      # m/s; zero for static objects

    def center_at(self, t: float) -> np.ndarray:
        return self.center + self.velocity * t


def default_objects(n_moving: int = 2, n_static: int = 1):
    objs = []
    cs = [np.array([-1.2, 0.6, 0.8]), np.array([1.0, 0.5, -0.6]), np.array([0.2, 0.9, 1.6])]
    ax = [np.array([0.35, 0.5, 0.3]), np.array([0.4, 0.3, 0.45]), np.array([0.5, 0.25, 0.2])]
    vs = [np.array([0.3, 0.0, 0.0]), np.array([0.0, 0.0, 0.3])]
    for k in range(n_moving + n_static):
        v = vs[k] if k < n_moving else np.zeros(3)
        objs.append(Ellipsoid(cs[k % 3].copy(), ax[k % 3].copy(), v.copy()))
    return objs


def texture(p: np.ndarray) -> np.ndarray:
    """Smooth colour field of the room surfaces (RGB in [0.1, 0.9])."""
    r = 0.5 + 0.3 * np.sin(2.1 * p[..., 0] + 0.7 * p[..., 2]) * np.cos(1.3 * p[..., 1])
    g = 0.5 + 0.3 * np.sin(1.7 * p[..., 2] - 1.1 * p[..., 1] + 0.4)
    b = 0.5 + 0.3 * np.cos(2.5 * p[..., 0] - 1.9 * p[..., 2] + 1.3 * p[..., 1])
    return np.stack([r, g, b], -1)


def _frames_from_normals(nrm: np.ndarray) -> np.ndarray:
    """Rotation matrices whose third column is the given unit normal."""
    helper = np.where(np.abs(nrm[:, 1:2]) < 0.9, np.array([[0.0, 1.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = np.cross(helper, nrm)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    return np.stack([t1, t2, nrm], axis=2)


def _jittered_grid(m: int, ex: float, ey: float, rng) -> np.ndarray:
    """m points covering [-ex, ex] x [-ey, ey] on a jittered grid (one
    point per cell, no holes), extra points uniform."""
    nx = max(1, int(np.floor(np.sqrt(m * ex / ey))))
    ny = max(1, m // nx)
    gx, gy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    px = (gx.ravel() + rng.uniform(0.1, 0.9, nx * ny)) / nx * 2 * ex - ex
    py = (gy.ravel() + rng.uniform(0.1, 0.9, nx * ny)) / ny * 2 * ey - ey
    extra = m - nx * ny
    if extra > 0:
        px = np.concatenate([px, rng.uniform(-ex, ex, extra)])
        py = np.concatenate([py, rng.uniform(-ey, ey, extra)])
    return np.stack([px[:m], py[:m]], 1)


def _fibonacci_sphere(m: int, rng) -> np.ndarray:
    k = np.arange(m) + 0.5
    z = 1 - 2 * k / m
    phi = np.pi * (1 + 5 ** 0.5) * k + rng.uniform(0, 2 * np.pi)
    r = np.sqrt(np.maximum(0.0, 1 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def room_scene(n: int, seed: int = 0, objects=None, opacity_logit=(4.0, 0.5), mp_static=0.1,
               mp_dynamic=0.9):
    """n Gaussians covering the 6 x 6 x 3 m room's walls, floor and ceiling
    and the objects' ellipsoidal surfaces, area-proportionally, on jittered
    grids (Fibonacci lattices on the ellipsoids) so that the surfaces have no
    holes, as in a converged map. Disc-like Gaussians: tangent sigma = 0.7 x
    mean spacing, normal sigma = 2 mm; opacity logit N(4, 0.5).
    Returns (records, object_id per Gaussian (-1 = room), objects)."""
    rng = np.random.default_rng(seed)
    objects = default_objects() if objects is None else objects
    hx, hy, hz = ROOM_HALF
    planes = [  # (axis, sign): wall at coordinate sign * half on that axis
        (0, -1), (0, 1), (2, -1), (2, 1), (1, -1), (1, 1)]
    areas = []
    for axis, _ in planes:
        o = [a for a in range(3) if a != axis]
        areas.append(4 * ROOM_HALF[o[0]] * ROOM_HALF[o[1]])
    for ob in objects:
        a, b, c = ob.axes
        p = 1.6075
        areas.append(4 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p))
    areas = np.array(areas)
    counts = np.floor(n * areas / areas.sum()).astype(int)
    counts[0] += n - counts.sum()
    spacing = np.sqrt(areas.sum() / n)
    pts, nrms, oid = [], [], []
    for k, (axis, sgn) in enumerate(planes):
        m = counts[k]
        o = [a for a in range(3) if a != axis]
        p = np.zeros((m, 3))
        p[:, o] = _jittered_grid(m, ROOM_HALF[o[0]], ROOM_HALF[o[1]], rng)
        p[:, axis] = sgn * ROOM_HALF[axis]
        nv = np.zeros((m, 3))
        nv[:, axis] = -sgn
        pts.append(p); nrms.append(nv); oid.append(np.full(m, -1))
    for j, ob in enumerate(objects):
        m = counts[len(planes) + j]
        d = _fibonacci_sphere(m, rng)
        p = ob.center + d * ob.axes
        nv = d / ob.axes
        nv /= np.linalg.norm(nv, axis=1, keepdims=True)
        pts.append(p); nrms.append(nv); oid.append(np.full(m, j))
    pts = np.concatenate(pts); nrms = np.concatenate(nrms); oid = np.concatenate(oid)
    quats = rotmat_to_quat(_frames_from_normals(nrms))
    sig_t = 0.7 * spacing
    logscales = np.stack([np.log(sig_t) + rng.normal(0, 0.1, n), np.log(sig_t) + rng.normal(0, 0.1, n),
                          np.full(n, np.log(0.002))], 1)
    rgb = np.clip(texture(pts) + rng.uniform(-0.05, 0.05, (n, 3)), 0, 1)
    logits = rng.normal(opacity_logit[0], opacity_logit[1], n)
    moving = np.array([np.any(ob.velocity != 0) for ob in objects] + [False])
    mp = np.where((oid >= 0) & moving[np.where(oid >= 0, oid, len(objects))], mp_dynamic, mp_static)
    rec = pack_records(pts, logits, quats, logscales, mp, rgb)
    return rec, oid, objects


def raycast(cam: Camera, pose: np.ndarray, objects, t: float = 0.0, depth_noise: float = 0.0,
            rng=None):
    """Ground-truth RGB-D of the analytic room at time t: per pixel (r, g, b,
    depth) with depth = camera z of the first hit, and the index of the hit
    object (-1 = room). Depth noise is multiplicative N(0, depth_noise)."""
    W, H = cam.width, cam.height
    jj, ii = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    dc = np.stack([(ii - cam.cx) / cam.fx, (jj - cam.cy) / cam.fy, np.ones_like(ii)], -1).reshape(-1, 3)
    R, tr = pose[:, :3], pose[:, 3]
    dw = dc @ R                                # rows: R^T d
    ow = -R.T @ tr
    best = np.full(dw.shape[0], np.inf)
    hit = np.full(dw.shape[0], -1)
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            with np.errstate(divide="ignore", invalid="ignore"):
                s = (sgn * ROOM_HALF[axis] - ow[axis]) / dw[:, axis]
            ok = (s > 1e-6) & (s < best)
            best = np.where(ok, s, best)
            hit = np.where(ok, -1, hit)
    for j, ob in enumerate(objects):
        c = ob.center_at(t)
        oc = (ow - c) / ob.axes
        dd = dw / ob.axes
        a = np.sum(dd * dd, 1)
        b = 2 * dd @ oc
        cc = oc @ oc - 1
        disc = b * b - 4 * a * cc
        sq = np.sqrt(np.maximum(disc, 0))
        s = (-b - sq) / (2 * a)
        ok = (disc > 0) & (s > 1e-6) & (s < best)
        best = np.where(ok, s, best)
        hit = np.where(ok, j, hit)
    p = ow + best[:, None] * dw
    rgb = texture(p)
    depth = best.copy()                          # camera z, since d_c has unit z
    if depth_noise > 0:
        rng = np.random.default_rng(0) if rng is None else rng
        depth = depth * (1 + rng.normal(0, depth_noise, depth.shape))
    out = np.zeros((W * H, 4), np.float32)
    out[:, 0:3] = rgb
    out[:, 3] = depth
    return out, hit


def camera_path(n_frames: int, fps: float = 30.0):
    """Smooth camera trajectory inside the room looking roughly at its centre."""
    poses = []
    for k in range(n_frames):
        s = k / fps
        eye = np.array([0.6 * np.sin(0.5 * s), -0.2 + 0.05 * np.sin(0.9 * s), -1.8 + 0.3 * np.cos(0.4 * s)])
        target = np.array([0.4 * np.sin(0.3 * s), 0.3, 1.5])
        poses.append(look_at_pose(eye, target))
    return poses


def room_camera(width: int = 640, height: int = 480, f: float = 525.0) -> Camera:
    return Camera(f, f, width / 2.0, height / 2.0, width, height)


def mapping_scene(n: int = 200_000, views: int = 8, seed: int = 0, width: int = 640, height: int = 480) -> Scene:
    """Mapping step: n room Gaussians, `views` keyframes on a ring inside the
    room looking inward, targets ray-cast with 1% depth noise (depth outside
    0.5-5 m marked invalid)."""
    rec, oid, objs = room_scene(n, seed)
    cam = room_camera(width, height)
    rng = np.random.default_rng(seed + 1)
    poses, tgs = [], []
    for v in range(views):
        a = 2 * np.pi * v / views
        eye = np.array([1.6 * np.cos(a), -0.3, 1.6 * np.sin(a)])
        target = np.array([-0.5 * np.cos(a), 0.4, -0.5 * np.sin(a)])
        pose = look_at_pose(eye, target)
        tg, _ = raycast(cam, pose, objs, 0.0, 0.01, rng)
        tg[(tg[:, 3] < 0.5) | (tg[:, 3] > 5.0), 3] = 0.0
        poses.append(pose); tgs.append(tg)
    return Scene(rec, cam, np.stack(poses), np.stack(tgs), oid >= 0, dict(objects=objs, object_id=oid))


def _tracking_frame(cam: Camera, objs, path, frame: int, seed: int, fps: float, flip: float):
    """Observed RGB-D of `frame` (moving objects translated), the instance
    label map of the moving objects with `flip` pixel flip noise, and the
    previous frame's pose (the tracking starting point)."""
    rng = np.random.default_rng(seed + 7 + frame)
    tg, hit = raycast(cam, path[frame], objs, frame / fps, 0.01, rng)
    tg[(tg[:, 3] < 0.5) | (tg[:, 3] > 5.0), 3] = 0.0
    moving = [k for k, ob in enumerate(objs) if np.any(ob.velocity != 0)]
    inst = np.zeros(hit.shape, np.uint8)
    for lab, k in enumerate(moving, start=1):
        inst[hit == k] = lab
    if flip > 0:
        fl = rng.random(inst.shape) < flip
        repl = rng.integers(0, len(moving) + 1, inst.shape).astype(np.uint8)
        same = repl == inst
        repl[same] = (repl[same] + 1) % (len(moving) + 1)
        inst = np.where(fl, repl, inst).astype(np.uint8)
    prev = path[frame - 1] if frame > 0 else path[0]
    return tg, inst, prev, path[frame], moving


def tracking_scene(n: int = 300_000, frame: int = 10, seed: int = 0, width: int = 640, height: int = 480,
                   fps: float = 30.0, flip: float = 0.05) -> Scene:
    """Tracking + MP update: the map holds the objects at their frame-0
    positions; the target of `frame` is ray-cast with the two moving objects
    translated at 0.3 m/s; the pose is the previous frame's (the tracking
    starting point) and extra['gt_pose'] the frame's own. Also returns the
    instance label map of the moving objects with `flip` pixel flip noise."""
    rec, oid, objs = room_scene(n, seed)
    cam = room_camera(width, height)
    path = camera_path(frame + 1, fps)
    tg, inst, prev, gt, moving = _tracking_frame(cam, objs, path, frame, seed, fps, flip)
    return Scene(rec, cam, prev[None], tg[None], np.isin(oid, moving),
                 dict(objects=objs, object_id=oid, gt_pose=gt, instance=inst, n_instances=len(moving)))


def tracking_sequence(n: int = 300_000, frames=range(10, 60), seed: int = 0, width: int = 640, height: int = 480,
                      fps: float = 30.0, flip: float = 0.05):
    """The tracking workload over several frames of one sequence: one map
    (records, camera) and, per frame, dict(target, instance, pose (the
    previous frame's: the starting point), gt_pose). Each frame equals
    tracking_scene(n, frame, seed, ...)'s."""
    rec, oid, objs = room_scene(n, seed)
    cam = room_camera(width, height)
    frames = list(frames)
    path = camera_path(max(frames) + 1, fps)
    out = []
    moving = []
    for f in frames:
        tg, inst, prev, gt, moving = _tracking_frame(cam, objs, path, f, seed, fps, flip)
        out.append(dict(frame=f, target=tg, instance=inst, pose=prev, gt_pose=gt))
    return rec, cam, out, dict(objects=objs, object_id=oid, n_instances=len(moving))


def spline_path(n_frames: int, fps: float = 30.0, seed: int = 0):
    """Camera on a smooth closed Catmull-Rom spline through eight seeded
    viewpoints inside the room (one loop per 10 s), looking at a target that
    moves on a second spline; world-to-camera poses."""
    rng = np.random.default_rng(seed + 555)
    k = 8
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    eyes = np.stack([0.9 * np.cos(ang), -0.2 + rng.uniform(-0.15, 0.15, k), -1.2 + 0.6 * np.sin(ang)], 1)
    tgts = np.stack([0.5 * np.sin(ang + 1.0), 0.3 + rng.uniform(-0.1, 0.1, k), 1.5 + 0.2 * np.cos(ang)], 1)

    def cr(pts, u):
        i = int(np.floor(u)) % k
        t = u - np.floor(u)
        p0, p1, p2, p3 = pts[(i - 1) % k], pts[i], pts[(i + 1) % k], pts[(i + 2) % k]
        return 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t +
                      (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3)

    poses = []
    for f in range(n_frames):
        u = (f / fps) / 10.0 * k
        poses.append(look_at_pose(cr(eyes, u), cr(tgts, u)))
    return poses


def full_loop_sequence(n: int = 1_000_000, frames=range(0, 12), seed: int = 0, width: int = 1200, height: int = 680,
                       fps: float = 30.0, flip: float = 0.05):
    """The full loop at scale: n room Gaussians with three moving ellipsoids
    (0.3 m/s along x, z and the xz diagonal) and one static one, a
    width x height RGB-D camera with the 640x480 rig's horizontal field of
    view (f = 525 * width / 640), the camera on spline_path. Per frame: the
    ray-cast target (1% depth noise), the moving objects' instance map with
    `flip` pixel flips, the ground-truth pose. Returns (records, camera,
    [dict(frame, target, instance, gt_pose)], extra)."""
    cs = [np.array([-1.2, 0.6, 0.8]), np.array([1.0, 0.5, -0.6]), np.array([0.1, 0.7, 0.2]),
          np.array([0.2, 0.9, 1.6])]
    ax = [np.array([0.35, 0.5, 0.3]), np.array([0.4, 0.3, 0.45]), np.array([0.3, 0.3, 0.3]),
          np.array([0.5, 0.25, 0.2])]
    vs = [np.array([0.3, 0.0, 0.0]), np.array([0.0, 0.0, 0.3]), np.array([0.21, 0.0, -0.21]), np.zeros(3)]
    objs = [Ellipsoid(c.copy(), a.copy(), v.copy()) for c, a, v in zip(cs, ax, vs)]
    rec, oid, objs = room_scene(n, seed, objects=objs)
    f = 525.0 * width / 640.0
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height)
    frames = list(frames)
    path = spline_path(max(frames) + 1, fps, seed)
    out = []
    moving = [k for k, ob in enumerate(objs) if np.any(ob.velocity != 0)]
    for fr in frames:
        rng = np.random.default_rng(seed + 31 + fr)
        tg, hit = raycast(cam, path[fr], objs, fr / fps, 0.01, rng)
        tg[(tg[:, 3] < 0.5) | (tg[:, 3] > 5.0), 3] = 0.0
        inst = np.zeros(hit.shape, np.uint8)
        for lab, k in enumerate(moving, start=1):
            inst[hit == k] = lab
        if flip > 0:
            fl = rng.random(inst.shape) < flip
            repl = rng.integers(0, len(moving) + 1, inst.shape).astype(np.uint8)
            same = repl == inst
            repl[same] = (repl[same] + 1) % (len(moving) + 1)
            inst = np.where(fl, repl, inst).astype(np.uint8)
        out.append(dict(frame=fr, target=tg, instance=inst, gt_pose=path[fr]))
    return rec, cam, out, dict(objects=objs, object_id=oid, n_instances=len(moving),
                               dynamic=np.isin(oid, moving))


def epipolar_matches(n: int = 300_000, frames=(11, 16), seed: int = 0, width: int = 640, height: int = 480,
                     fps: float = 30.0, n_sample: int = 20_000, per_gauss: int = 4, noise_px: float = 0.3,
                     suppressed: float = 0.1):
    """Feature matches between two frames of the tracking sequence for the
    epipolar verification: n_sample Gaussians visible in both frames, each
    with per_gauss matches (the Gaussian's world position at each frame's
    time projected with that frame's ground-truth pose, plus N(0, noise_px)
    pixel noise per match; moving objects' Gaussians move between the frames).
    Labels: the moving objects' Gaussians dynamic (1) and a `suppressed`
    fraction of static ones also dynamic (static structure an MP prior
    suppressed). Returns dict(records, camera, pose_1, pose_2, p1, p2 (m x 2
    float32), gid (m int32), labels (n uint8), moving (n bool))."""
    rng = np.random.default_rng(seed + 991)
    rec, oid, objs = room_scene(n, seed)
    cam = room_camera(width, height)
    f1, f2 = frames
    path = camera_path(max(frames) + 1, fps)
    T1, T2 = path[f1], path[f2]
    vel = np.zeros((n, 3))
    for k, ob in enumerate(objs):
        vel[oid == k] = ob.velocity
    moving = np.linalg.norm(vel, axis=1) > 0

    def project(T, X):
        Y = X @ T[:, :3].T + T[:, 3]
        z = Y[:, 2]
        u = cam.fx * Y[:, 0] / np.maximum(z, 1e-9) + cam.cx
        v = cam.fy * Y[:, 1] / np.maximum(z, 1e-9) + cam.cy
        ok = (z > 0.3) & (u >= 0) & (u <= width - 1) & (v >= 0) & (v <= height - 1)
        return np.stack([u, v], 1), ok

    X1 = rec[:, 0:3].astype(np.float64) + vel * (f1 / fps)
    X2 = rec[:, 0:3].astype(np.float64) + vel * (f2 / fps)
    q1, ok1 = project(T1, X1)
    q2, ok2 = project(T2, X2)
    cand = np.nonzero(ok1 & ok2)[0]
    pick = rng.choice(cand, size=min(n_sample, len(cand)), replace=False)
    gid = np.repeat(pick, per_gauss).astype(np.int32)
    p1 = (q1[gid] + rng.normal(0, noise_px, (len(gid), 2))).astype(np.float32)
    p2 = (q2[gid] + rng.normal(0, noise_px, (len(gid), 2))).astype(np.float32)
    labels = moving.astype(np.uint8)
    labels[(~moving) & (rng.random(n) < suppressed)] = 1
    return dict(records=rec, camera=cam, pose_1=T1, pose_2=T2, p1=p1, p2=p2, gid=gid, labels=labels,
                moving=moving)


# ------------------------------------------------------------------ learned MP network

MPNET_BLOB_BYTES = 22016
MPNET_PARAMS = 10881


def mpnet_init(seed: int = 0):
    """Seeded He-style initial weights of the per-pixel MP network in the
    library's layouts: (blob uint8[22016] with BF16 weights and FP32 biases,
    master float32[10881] parameter vector). Biases start at zero."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((32, 16), np.float32)
    W1[:, :8] = rng.normal(0, np.sqrt(2.0 / 8), (32, 8))
    W2 = rng.normal(0, np.sqrt(2.0 / 288), (32, 288)).astype(np.float32)   # column (ky * 3 + kx) * 32 + in
    W3 = rng.normal(0, np.sqrt(2.0 / 32), (32, 32)).astype(np.float32)
    w4 = rng.normal(0, np.sqrt(1.0 / 32), 32).astype(np.float32)
    wb = np.concatenate([f32_to_bf16_bits(a.ravel()) for a in (W1, W2, W3, w4)])
    blob = np.zeros(MPNET_BLOB_BYTES, np.uint8)
    blob[:wb.size * 2] = wb.view(np.uint8)
    master = np.zeros(MPNET_PARAMS, np.float32)
    master[:wb.size] = bf16_bits_to_f32(wb)
    return blob, master
