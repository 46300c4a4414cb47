"""Seeded synthetic inputs for the 3DGS-Calib splatting path.

This module only draws inputs: Gaussian attributes, LiDAR-shaped point clouds,
keyframed LiDAR trajectories, camera intrinsics, frame timestamps and
extrinsics.  It contains none of the method's arithmetic (no trajectory
interpolation, projection, compositing or gradients), so both the CPU oracle
and the CUDA path can consume it without sharing any of the computation.

Conventions shared by every consumer:

* World frame: x forward along the road, y left, z up; ground plane z = 0.
* Camera frame: x right, y down, z forward (pinhole, OpenCV style).
* Quaternions are Hamilton (w, x, y, z).
* A LiDAR keyframe is (t, p[3], q[4]) giving the LiDAR-to-world pose at t.
* An extrinsic is (omega[3], t[3]): the camera-to-LiDAR transform
  L_T_i = [Exp(omega) | t] (the paper's notation table, Sec. III-A), with
  Exp the SO(3) exponential of the rotation vector omega.
* The time offset delta shifts a camera timestamp onto the LiDAR clock:
  the camera pose is T_L(t + delta) * L_T_i (Eq. 1).

The workloads mirror the paper's KITTI-360 setting (Sec. IV-A: a 64-beam
spinning LiDAR, a 1408x376 forward camera, driving trajectories, and
0.25-3.4 M accumulated points, Table 4); the dataset itself is not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Camera", "Scene", "Frame", "Problem",
    "tiny_problem", "lidar_frame_problem", "batched_problem", "uneven_problem",
    "calibration_problem", "random_splat_records", "make_problem",
]


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


@dataclass
class Scene:
    """One set of Gaussians anchored at accumulated LiDAR points (Sec. III-B)."""
    X: np.ndarray          # [N,3] float32 world positions (fixed, not optimised)
    quat: np.ndarray       # [N,4] float32 rotation quaternion r (w,x,y,z)
    log_scale: np.ndarray  # [N,3] float32 log of the axis scales s
    logit_opacity: np.ndarray  # [N] float32 logit of the opacity alpha
    rgb: np.ndarray        # [N,3] float32 view-independent colour c
    traj_t: np.ndarray     # [K] float64 keyframe times (s)
    traj_p: np.ndarray     # [K,3] float64 keyframe LiDAR positions (world)
    traj_q: np.ndarray     # [K,4] float64 keyframe LiDAR orientations (w,x,y,z)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


@dataclass
class Frame:
    camera: Camera
    timestamp: float       # t^{n_i}, seconds on the camera clock
    camera_id: int = 0     # which extrinsic / time offset
    scene_id: int = 0      # which scene (Gaussians + trajectory)
    row0: int = 0          # first image row used (height // 2: the bottom half, Sec. III-D)


@dataclass
class Problem:
    name: str
    scenes: list
    frames: list
    ext: np.ndarray        # [C,6] float64 (omega, t) used for rendering
    delta: np.ndarray      # [C] float64
    ext_target: np.ndarray | None = None    # extrinsic of the target images
    delta_target: np.ndarray | None = None
    tile: int = 16
    meta: dict = field(default_factory=dict)

    @property
    def num_cameras(self) -> int:
        return int(self.ext.shape[0])


# ----------------------------------------------------------------------------
# small helpers (input construction only)
# ----------------------------------------------------------------------------

def _axis_angle_quat(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle
    return np.concatenate([[math.cos(h)], math.sin(h) * axis])


def _unit(rng, n, d):
    v = rng.normal(size=(n, d))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _attributes(rng, n, scale_lo, scale_hi):
    log_s = rng.uniform(math.log(scale_lo), math.log(scale_hi), size=(n, 3))
    q = _unit(rng, n, 4)
    logit_o = rng.normal(size=n)
    return (q.astype(np.float32), log_s.astype(np.float32),
            logit_o.astype(np.float32))


# The nominal camera-to-LiDAR rotation of a forward-looking camera on a car:
# camera z (forward) -> LiDAR x, camera x (right) -> LiDAR -y,
# camera y (down) -> LiDAR -z.  As a rotation vector this is a 120 degree
# turn about (-1, 1, -1)/sqrt(3).
NOMINAL_CAM_TO_LIDAR_OMEGA = (2.0 * math.pi / 3.0) * np.array([-1.0, 1.0, -1.0]) / math.sqrt(3.0)
NOMINAL_CAM_TO_LIDAR_T = np.array([1.0, 0.3, -0.2])
LIDAR_HEIGHT = 1.8

CAM_KITTI = Camera(1408, 376, 552.0, 552.0, 682.0, 238.0)
CAM_HALF = Camera(704, 188, 276.0, 276.0, 341.0, 119.0)
CAM_HD = Camera(1920, 1080, 960.0, 960.0, 959.5, 539.5)


def _perturb_rotvec(rng, omega, angle_deg):
    """Rotation vector of R(omega) * R(angle about a seeded random axis)."""
    from scipy.spatial.transform import Rotation
    axis = _unit(rng, 1, 3)[0]
    r = Rotation.from_rotvec(omega) * Rotation.from_rotvec(math.radians(angle_deg) * axis)
    return r.as_rotvec()


def _true_extrinsic(rng):
    omega = _perturb_rotvec(rng, NOMINAL_CAM_TO_LIDAR_OMEGA, 2.0)
    return np.concatenate([omega, NOMINAL_CAM_TO_LIDAR_T])


# ----------------------------------------------------------------------------
# C1: tiny plain render
# ----------------------------------------------------------------------------

def tiny_problem(seed: int = 0, n: int = 64, width: int = 64, height: int = 48,
                 focal: float = 60.0) -> Problem:
    """64 Gaussians in front of one 64x48 pinhole camera.

    The trajectory has two keyframes at t = 0 s and t = 1 s, moving 1 m/s
    along x and turning 10 deg/s about the vertical (y) axis; they are placed
    symmetrically so that the LiDAR pose at the frame time t = 0.5 s is the
    identity.  The extrinsic is the identity and delta = 0, so the Gaussian
    means are drawn directly in the camera frame.  The target images are
    rendered with the extrinsic perturbed by 1 deg about a seeded axis and
    5 cm along a seeded direction.
    """
    rng = np.random.default_rng(seed)
    X = np.stack([rng.uniform(-2, 2, n), rng.uniform(-1.5, 1.5, n),
                  rng.uniform(2, 10, n)], axis=1).astype(np.float32)
    q, log_s, logit_o = _attributes(rng, n, 0.05, 0.5)
    rgb = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
    yaw = math.radians(5.0)
    traj_t = np.array([0.0, 1.0])
    traj_p = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])
    traj_q = np.stack([_axis_angle_quat([0, 1, 0], -yaw), _axis_angle_quat([0, 1, 0], yaw)])
    scene = Scene(X, q, log_s, logit_o, rgb, traj_t, traj_p, traj_q)
    cam = Camera(width, height, focal, focal, (width - 1) / 2.0, (height - 1) / 2.0)
    ext = np.zeros((1, 6))
    axis = _unit(rng, 1, 3)[0]
    direction = _unit(rng, 1, 3)[0]
    ext_t = np.concatenate([math.radians(1.0) * axis, 0.05 * direction])[None]
    return Problem("tiny", [scene], [Frame(cam, 0.5)], ext, np.zeros(1),
                   ext_target=ext_t, delta_target=np.zeros(1), tile=16)


# ----------------------------------------------------------------------------
# LiDAR-shaped worlds
# ----------------------------------------------------------------------------

@dataclass
class _World:
    lo: np.ndarray   # [B,3] box minimum corners
    hi: np.ndarray   # [B,3] box maximum corners
    base: np.ndarray  # [B+1,3] base colour per surface (last = ground)


def _make_world(rng, n_boxes, x_range):
    lo, hi = [], []
    for _ in range(n_boxes):
        side = rng.choice([-1.0, 1.0])
        length = rng.uniform(5.0, 30.0)
        depth = rng.uniform(2.0, 10.0)
        height = rng.uniform(3.0, 15.0)
        x0 = rng.uniform(x_range[0], x_range[1])
        y_near = rng.uniform(4.0, 15.0)
        y0 = side * y_near if side > 0 else -(y_near + depth)
        lo.append([x0, y0, 0.0])
        hi.append([x0 + length, y0 + depth, height])
    base = rng.uniform(0.15, 0.85, size=(n_boxes + 1, 3))
    base[-1] = [0.35, 0.35, 0.38]
    return _World(np.array(lo), np.array(hi), base)


N_ELEV, N_AZIM = 64, 2048
ELEV_LO, ELEV_HI = -25.0, 3.0


def _beam_dirs(rng, jitter):
    """Unit ray directions of one sweep as a [64, 2048, 3] grid
    (elevation-major); jittered re-casts move each ray by up to half a step."""
    elev = np.deg2rad(np.linspace(ELEV_LO, ELEV_HI, N_ELEV))
    azim = np.linspace(0.0, 2.0 * math.pi, N_AZIM, endpoint=False)
    e, a = np.meshgrid(elev, azim, indexing="ij")
    if jitter:
        e = e + rng.uniform(-0.5, 0.5, e.shape) * np.deg2rad((ELEV_HI - ELEV_LO) / (N_ELEV - 1))
        a = a + rng.uniform(-0.5, 0.5, a.shape) * (2.0 * math.pi / N_AZIM)
    return np.stack([np.cos(e) * np.cos(a), np.cos(e) * np.sin(a), np.sin(e)], axis=-1)


def _cast(world, origin, dirs, r_min=2.0, r_max=80.0):
    """Nearest hit of the rays origin + t*dirs ([64, 2048, 3] grid) with the
    ground plane and the boxes.  A box only needs the azimuth columns it
    spans; boxes lie off the road (|y| >= 4 m), so that span never wraps."""
    ne, na, _ = dirs.shape
    t_best = np.full((ne, na), np.inf)
    hit_id = np.full((ne, na), -1, dtype=np.int64)
    dz = dirs[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        t_g = np.where(dz < 0, -origin[2] / dz, np.inf)
    t_best[:] = t_g
    hit_id[np.isfinite(t_g)] = len(world.lo)
    step = 2.0 * math.pi / na
    for b in range(len(world.lo)):
        lo, hi = world.lo[b], world.hi[b]
        centre = 0.5 * (lo + hi)
        if np.linalg.norm(centre[:2] - origin[:2]) > r_max + 0.5 * np.linalg.norm(hi - lo):
            continue
        cx = np.array([lo[0], hi[0], lo[0], hi[0]]) - origin[0]
        cy = np.array([lo[1], lo[1], hi[1], hi[1]]) - origin[1]
        az = np.mod(np.arctan2(cy, cx), 2.0 * math.pi)
        c0 = max(int(math.floor(az.min() / step)) - 2, 0)
        c1 = min(int(math.ceil(az.max() / step)) + 2, na - 1)
        d = dirs[:, c0:c1 + 1]
        inv = 1.0 / np.where(np.abs(d) < 1e-12, 1e-12, d)
        t1 = (lo - origin) * inv
        t2 = (hi - origin) * inv
        tn = np.minimum(t1, t2).max(axis=-1)
        tf = np.maximum(t1, t2).min(axis=-1)
        tb = t_best[:, c0:c1 + 1]
        ok = (tf >= tn) & (tn > 0) & (tn < tb)
        tb[ok] = tn[ok]
        hit_id[:, c0:c1 + 1][ok] = b
    keep = (t_best >= r_min) & (t_best <= r_max)
    pts = origin + dirs[keep] * t_best[keep][:, None]
    return pts, hit_id[keep]


def _smooth_colour(rng, world, pts, ids):
    base = world.base[ids]
    k = rng.uniform(0.2, 0.9, size=(3, 3))
    ph = rng.uniform(0, 2 * math.pi, size=(3, 3))
    wave = np.zeros_like(pts)
    for c in range(3):
        wave[:, c] = 0.12 * (np.sin(k[c, 0] * pts[:, 0] + ph[c, 0])
                             + np.sin(k[c, 1] * pts[:, 1] + ph[c, 1])
                             + np.sin(k[c, 2] * pts[:, 2] + ph[c, 2]))
    col = base + wave + rng.normal(0, 0.05, size=pts.shape)
    return np.clip(col, 0.0, 1.0)


def _identity_quats(k):
    q = np.zeros((k, 4))
    q[:, 0] = 1.0
    return q


def lidar_frame_problem(seed: int = 1, n: int = 200_000) -> Problem:
    """One LiDAR sweep at the origin re-cast with jitter to exactly n hits,
    seen by one 1408x376 camera with the true extrinsic."""
    rng = np.random.default_rng(seed)
    world = _make_world(rng, 20, (-40.0, 40.0))
    origin = np.array([0.0, 0.0, LIDAR_HEIGHT])
    pts, ids, total = [], [], 0
    jitter = False
    while total < n:
        p, i = _cast(world, origin, _beam_dirs(rng, jitter))
        pts.append(p)
        ids.append(i)
        total += len(p)
        jitter = True
    pts = np.concatenate(pts)[:n]
    ids = np.concatenate(ids)[:n]
    q, log_s, logit_o = _attributes(rng, n, 0.02, 0.3)
    rgb = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
    traj_t = np.array([-1.0, 1.0])
    traj_p = np.array([[-10.0, 0.0, LIDAR_HEIGHT], [10.0, 0.0, LIDAR_HEIGHT]])
    scene = Scene(pts.astype(np.float32), q, log_s, logit_o, rgb, traj_t, traj_p,
                  _identity_quats(2))
    ext = _true_extrinsic(rng)[None]
    return Problem("lidar_frame", [scene], [Frame(CAM_KITTI, 0.0)], ext, np.zeros(1),
                   tile=16, meta={"hit_ids": ids})


def _yaw_rotate(dirs, yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    out = dirs.copy()
    out[..., 0] = c * dirs[..., 0] - s * dirs[..., 1]
    out[..., 1] = s * dirs[..., 0] + c * dirs[..., 1]
    return out


def _surface_attributes(rng, world, pts, ids):
    """Attributes that vary smoothly along each surface: discs flattened
    along the surface normal (the ground's z; for a box, the axis of the face
    the point lies on), about 6 cm across and 1 cm thick with a low-frequency
    modulation, opacity between ~0.8 and ~0.95, no rotation.  Real surfaces
    are continuous over large areas (walls, roads), which a spatially
    regularised attribute model can represent."""
    n = len(pts)
    normal = np.full(n, 2)
    on_box = ids < len(world.lo)
    if on_box.any():
        lo, hi = world.lo[ids[on_box]], world.hi[ids[on_box]]
        p = pts[on_box]
        d = np.minimum(np.abs(p - lo), np.abs(p - hi))
        normal[on_box] = np.argmin(d, axis=1)
    k = rng.uniform(0.3, 0.8, size=3)
    ph = rng.uniform(0, 2 * math.pi, size=3)
    wave = np.sin(k[0] * pts[:, 0] + ph[0]) + np.sin(k[1] * pts[:, 1] + ph[1]) + np.sin(k[2] * pts[:, 2] + ph[2])
    s = np.full((n, 3), 0.06) * np.exp(0.15 * wave)[:, None]
    s[np.arange(n), normal] = 0.01
    logit_o = 2.0 + 0.4 * np.sin(0.5 * pts[:, 0] + ph[0]) * np.cos(0.5 * pts[:, 1] + ph[1])
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return q.astype(np.float32), np.log(s).astype(np.float32), logit_o.astype(np.float32)


def _drive_scene(rng, n, sweeps=50, speed=10.0, rate=10.0, smooth=True, trajectory="straight",
                 attributes="random"):
    """Points from LiDAR sweeps along a drive.  'straight': 10 m/s along x
    with a constant heading.  'zigzag': the same forward speed with a lateral
    swing y = 3 sin(2 pi t / 2.5) m and the heading following the path (so
    velocity and orientation change over time)."""
    world = _make_world(rng, 60, (-30.0, 120.0))
    traj_t = np.arange(sweeps) / rate
    if trajectory == "straight":
        y = np.zeros(sweeps)
        yaw = np.zeros(sweeps)
    elif trajectory == "zigzag":
        w = 2.0 * math.pi / 2.5
        y = 3.0 * np.sin(w * traj_t)
        yaw = np.arctan2(3.0 * w * np.cos(w * traj_t), speed)
    else:
        raise ValueError(trajectory)
    traj_p = np.stack([speed * traj_t, y, np.full(sweeps, LIDAR_HEIGHT)], axis=1)
    traj_q = np.stack([np.cos(yaw / 2), np.zeros(sweeps), np.zeros(sweeps), np.sin(yaw / 2)], axis=1)
    pts, ids = [], []
    for k in range(sweeps):
        p, i = _cast(world, traj_p[k], _yaw_rotate(_beam_dirs(rng, k > 0), yaw[k]))
        pts.append(p)
        ids.append(i)
    pts = np.concatenate(pts)
    ids = np.concatenate(ids)
    while len(pts) < n:  # extra jittered sweeps if the quota is not reached
        k = int(rng.integers(sweeps))
        p, i = _cast(world, traj_p[k], _yaw_rotate(_beam_dirs(rng, True), yaw[k]))
        pts = np.concatenate([pts, p])
        ids = np.concatenate([ids, i])
    sel = rng.choice(len(pts), size=n, replace=False)
    sel.sort()
    pts, ids = pts[sel], ids[sel]
    q, log_s, logit_o = _attributes(rng, n, 0.02, 0.3)
    if attributes == "surface":
        q, log_s, logit_o = _surface_attributes(rng, world, pts, ids)
    elif attributes != "random":
        raise ValueError(attributes)
    if smooth:
        rgb = _smooth_colour(rng, world, pts, ids)
    else:
        rgb = rng.uniform(0, 1, size=(n, 3))
    return Scene(pts.astype(np.float32), q, log_s, logit_o, rgb.astype(np.float32),
                 traj_t, traj_p, traj_q)


def batched_problem(seed: int = 2, n: int = 1_000_000, frames: int = 8, trajectory: str = "straight",
                    attributes: str = "random") -> Problem:
    """1M Gaussians from 50 sweeps along a 10 m/s drive sampled at 10 Hz
    (straight by default); eight 1408x376 frames at t = 0.5, 1.0, ..., 4.0 s;
    true delta 40 ms."""
    rng = np.random.default_rng(seed)
    scene = _drive_scene(rng, n, trajectory=trajectory, attributes=attributes)
    ext = _true_extrinsic(rng)[None]
    fr = [Frame(CAM_KITTI, 0.5 * (i + 1)) for i in range(frames)]
    return Problem("batched", [scene], fr, ext, np.array([0.04]), tile=16)


def uneven_problem(seed: int = 3, sizes=(300_000, 1_000_000, 3_000_000),
                   cams=(CAM_HALF, CAM_KITTI, CAM_HD), frames_per_scene: int = 4) -> Problem:
    """Three independent scenes of uneven size, each with its own camera
    resolution, trajectory and extrinsic; all frames go through one launch
    per stage."""
    scenes, frames, exts = [], [], []
    for s, (n, cam) in enumerate(zip(sizes, cams)):
        rng = np.random.default_rng(seed + s)
        scenes.append(_drive_scene(rng, n))
        exts.append(_true_extrinsic(rng))
        for i in range(frames_per_scene):
            frames.append(Frame(cam, 0.5 + 0.9 * i, camera_id=s, scene_id=s))
    return Problem("uneven", scenes, frames, np.array(exts), np.full(len(sizes), 0.04), tile=16)


STEREO_BASELINE = 0.6  # metres between the two front cameras of a rig (KITTI-360 scale)


def rig_extrinsics(rng, cameras: int):
    """True extrinsics of `cameras` forward cameras on one car: the nominal
    mounting, each with its own seeded 2 deg tilt, spaced STEREO_BASELINE to
    the left (LiDAR +y) of one another; and true time offsets 0, 20, 40 ms..."""
    exts = []
    for c in range(cameras):
        e = _true_extrinsic(rng)
        e[4] += c * STEREO_BASELINE
        exts.append(e)
    return np.array(exts), 0.02 * np.arange(cameras)


def calibration_problem(seed: int = 0, n: int = 1_000_000, frames: int = 8,
                        rot_deg: float = 5.0, trans_m: float = 0.5,
                        delta0: float = 0.05, scene_seed: int = 2, trajectory: str = "straight",
                        cameras: int = 1, attributes: str = "random") -> Problem:
    """The batched scene; targets at the true extrinsic and delta = 0, start
    from the extrinsic perturbed by rot_deg about a seeded axis and trans_m
    along a seeded direction, and delta = delta0.  On the straight drive a
    time offset and a translation along the motion are interchangeable; the
    zigzag drive makes both observable.

    cameras > 1: a rig of forward cameras on one scene (rig_extrinsics),
    `frames` frames per camera at the same timestamps, each camera with its
    own true extrinsic and time offset and its own seeded start (the same
    rot_deg / trans_m distance, delta0 above its true offset).

    attributes="surface": Gaussian shapes and opacities that vary smoothly
    along each surface (_surface_attributes) instead of i.i.d. random ones."""
    base = batched_problem(scene_seed, n, frames, trajectory=trajectory, attributes=attributes)
    rng = np.random.default_rng(1000 + seed)
    if cameras == 1:
        true, true_delta = base.ext.copy(), np.zeros(1)
    else:
        true, true_delta = rig_extrinsics(np.random.default_rng(2000 + scene_seed), cameras)
        base.frames = [Frame(f.camera, f.timestamp, camera_id=c) for c in range(cameras) for f in base.frames]
    start = []
    for c in range(cameras):
        omega0 = _perturb_rotvec(rng, true[c, :3], rot_deg)
        t0 = true[c, 3:] + trans_m * _unit(rng, 1, 3)[0]
        start.append(np.concatenate([omega0, t0]))
    base.name = "calibration" if cameras == 1 else "rig calibration"
    base.ext_target = true
    base.delta_target = true_delta
    base.ext = np.array(start)
    base.delta = true_delta + delta0
    return base


def random_splat_records(seed: int, frames_tiles, n_per_frame, tie_fraction=0.3,
                         max_extent_tiles=6):
    """Seeded synthetic per-(frame, Gaussian) tile rectangles and depths for
    testing the tile binning and depth sort on their own.

    frames_tiles: list of (tiles_x, tiles_y).  Returns (rect [R,4] int32 with
    x0,y0,x1,y1 inclusive tile coordinates, an empty rect encoded x0 > x1;
    depth [R] float32).  A fraction of depths repeat exactly so that the
    stability of the sort is exercised.
    """
    rng = np.random.default_rng(seed)
    rects, depths = [], []
    for (tx, ty), n in zip(frames_tiles, n_per_frame):
        x0 = rng.integers(-2, tx + 1, n)
        y0 = rng.integers(-2, ty + 1, n)
        w = rng.integers(0, max_extent_tiles, n)
        h = rng.integers(0, max_extent_tiles, n)
        x1 = np.minimum(x0 + w, tx - 1)
        y1 = np.minimum(y0 + h, ty - 1)
        x0 = np.maximum(x0, 0)
        y0 = np.maximum(y0, 0)
        empty = (rng.uniform(size=n) < 0.1) | (x0 > x1) | (y0 > y1)
        x0 = np.where(empty, 1, x0)
        x1 = np.where(empty, 0, x1)
        y0 = np.where(empty, 1, y0)
        y1 = np.where(empty, 0, y1)
        rects.append(np.stack([x0, y0, x1, y1], axis=1))
        d = rng.uniform(0.2, 90.0, n).astype(np.float32)
        ties = rng.uniform(size=n) < tie_fraction
        d[ties] = rng.choice(d[:max(1, n // 20)], size=int(ties.sum()))
        depths.append(d)
    return np.concatenate(rects).astype(np.int32), np.concatenate(depths).astype(np.float32)


def make_problem(name: str, **kw) -> Problem:
    return {
        "tiny": tiny_problem,
        "lidar_frame": lidar_frame_problem,
        "batched": batched_problem,
        "uneven": uneven_problem,
        "calibration": calibration_problem,
    }[name](**kw)
