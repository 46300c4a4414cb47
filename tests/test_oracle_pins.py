"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand
closed forms (tests/golden), library routines (scipy rotations, numpy,
Python's stable sort), invariances that follow from Eq. 1-3, and central
finite differences of the oracle's own forward for every gradient.
"""
import copy
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2403_11577_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _single_scene(Xs, scales, logit_o, rgb, quats=None):
    n = len(Xs)
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.asarray(quats, float)
    return scenes.Scene(np.asarray(Xs, np.float64), q, np.log(np.asarray(scales, float)),
                        np.asarray(logit_o, float), np.asarray(rgb, float),
                        np.array([0.0]), np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]))


CAM = scenes.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)
FRAME = scenes.Frame(CAM, 0.0)
BG = (0.1, 0.2, 0.3)


def test_single_gaussian_closed_form():
    """Isotropic Gaussian on the optical axis: EWA covariance, conic, peak
    alpha = min(0.99, opacity), C = alpha c + (1 - alpha) bg (Eq. 2-3, Eq. 5)."""
    g = json.load(open(GOLDEN))["single_isotropic_on_axis"]
    sc = _single_scene([[0, 0, 2]], [[0.1] * 3], [0.0], [[0.8, 0.4, 0.2]])
    opts = oracle.Opts(bg=BG)
    pr = oracle.project(sc, CAM, np.eye(3), np.zeros(3), opts)
    assert pr["cov"][0, 0] == pytest.approx(g["cov_xx"], rel=1e-12)
    assert pr["conic"][0, 0] == pytest.approx(g["conic_a"], rel=1e-12)
    assert abs(pr["conic"][0, 1]) < 1e-15
    np.testing.assert_allclose(pr["mean"][0], g["mean"], atol=1e-12)
    rgb, T, last, flags = oracle.render(sc, FRAME, np.zeros(6), 0.0, opts, pixels=[[32, 24], [33, 24]])
    np.testing.assert_allclose(rgb[0], g["rgb_at_mean"], atol=1e-12)
    assert T[0] == pytest.approx(g["T_at_mean"], abs=1e-12)
    assert T[1] == pytest.approx(1 - g["alpha_at_33_24"], abs=1e-12)
    np.testing.assert_allclose(rgb[1], g["rgb_at_33_24"], atol=1e-12)
    assert list(last) == [0, 0] and list(flags) == [0, 0]


def test_peak_alpha_clamp():
    """A nearly opaque Gaussian is clamped to alpha_max = 0.99 at its peak."""
    sc = _single_scene([[0, 0, 2]], [[0.1] * 3], [8.0], [[1.0, 1.0, 1.0]])
    rgb, T, _, _ = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(), pixels=[[32, 24]])
    assert T[0] == pytest.approx(0.01, abs=1e-12)
    np.testing.assert_allclose(rgb[0], [0.99] * 3, atol=1e-12)


def test_two_gaussians_depth_order():
    """Front-to-back compositing of two depth-ordered splats (Eq. 5); the
    farther Gaussian is first in memory."""
    g = json.load(open(GOLDEN))["two_gaussians_on_axis"]
    sc = _single_scene([[0, 0, 3], [0, 0, 2]], [[0.1] * 3] * 2, [0.0, math.log(3.0)],
                       [[1, 0, 0], [0, 0, 1]])
    rgb, T, last, _ = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(bg=BG), pixels=[[32, 24]])
    np.testing.assert_allclose(rgb[0], g["rgb_at_mean"], atol=1e-12)
    assert T[0] == pytest.approx(g["T_at_mean"], abs=1e-12)
    assert last[0] == 0  # the farther one is composited last


def test_early_termination_closed_form():
    """Compositing stops before a Gaussian would bring T below t_min."""
    g = json.load(open(GOLDEN))["stacked_opaque_on_axis"]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]]
    sc = _single_scene([[0, 0, z] for z in (2, 3, 4, 5, 6)], [[0.1] * 3] * 5,
                       [math.log(19.0)] * 5, cols)
    rgb, T, last, flags = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(bg=BG), pixels=[[32, 24]])
    np.testing.assert_allclose(rgb[0], g["rgb_at_mean"], atol=1e-12)
    assert T[0] == pytest.approx(g["T_at_mean"], rel=1e-12)
    assert last[0] == g["last"] and flags[0] == 0


def test_opacity_zero_gives_background():
    p = scenes.tiny_problem()
    sc = copy.deepcopy(p.scenes[0])
    sc.logit_opacity = np.full(sc.n, -60.0)
    rgb, T, last, _ = oracle.render(sc, p.frames[0], p.ext[0], 0.0, oracle.Opts(bg=BG))
    assert np.all(T == 1.0) and np.all(last == -1)
    assert np.all(rgb == np.array(BG))


def test_transmittance_monotone_and_colour_linear():
    p = scenes.tiny_problem()
    sc, fr = p.scenes[0], p.frames[0]
    opts = oracle.Opts(t_min=0.0)
    R, t = oracle.frame_pose(sc, p.ext[0], 0.0, fr.timestamp)
    depth = oracle.project(sc, fr.camera, R, t, opts)["depth"]
    order = np.argsort(depth, kind="stable")
    prev = np.ones(fr.camera.width * fr.camera.height)
    for k in range(8, sc.n + 1, 8):
        sub = copy.deepcopy(sc)
        sub.logit_opacity = sc.logit_opacity.astype(np.float64).copy()
        sub.logit_opacity[order[k:]] = -60.0
        T = oracle.render(sub, fr, p.ext[0], 0.0, opts)[1]
        assert np.all(T <= prev + 1e-15) and np.all(T > 0) and np.all(T <= 1)
        prev = T
    # colour linearity with bg = 0: C(a c1 + b c2) = a C(c1) + b C(c2)
    rng = np.random.default_rng(3)
    c1, c2 = rng.uniform(size=(sc.n, 3)), rng.uniform(size=(sc.n, 3))
    s1, s2, s3 = (copy.deepcopy(sc) for _ in range(3))
    s1.rgb, s2.rgb, s3.rgb = c1, c2, 0.3 * c1 + 1.7 * c2
    r1 = oracle.render(s1, fr, p.ext[0], 0.0)[0]
    r2 = oracle.render(s2, fr, p.ext[0], 0.0)[0]
    r3 = oracle.render(s3, fr, p.ext[0], 0.0)[0]
    np.testing.assert_allclose(r3, 0.3 * r1 + 1.7 * r2, atol=1e-12)


def test_trajectory_closed_form():
    """Lerp + SLERP between keyframes (Sec. III-A): constant velocity and
    constant yaw rate give p(tau), R(tau) and dR/dtau in closed form."""
    yaw = math.radians(60.0)
    sc = _single_scene([[0, 0, 5]], [[0.1] * 3], [0.0], [[1, 1, 1]])
    sc.traj_t = np.array([0.0, 1.0, 3.0])
    sc.traj_p = np.array([[0, 0, 0], [1, 2, 3], [1, 2, 3]], float)
    sc.traj_q = np.array([[1, 0, 0, 0], [math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)],
                          [math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)]])
    for tau in [0.0, 0.25, 0.5, 0.999]:
        R, p, dR, dp = oracle.lidar_pose(sc, tau)
        Rz = Rotation.from_rotvec([0, 0, yaw * tau]).as_matrix()
        np.testing.assert_allclose(p, np.array([1, 2, 3]) * tau, atol=1e-12)
        np.testing.assert_allclose(R, Rz, atol=1e-12)
        np.testing.assert_allclose(dp, [1, 2, 3], atol=1e-12)
        W = np.array([[0, -yaw, 0], [yaw, 0, 0], [0, 0, 0]])
        np.testing.assert_allclose(dR, Rz @ W, atol=1e-10)
    # keyframes are reproduced exactly and the next segment starts at t_1
    R, p, dR, dp = oracle.lidar_pose(sc, 1.0)
    np.testing.assert_allclose(p, [1, 2, 3], atol=1e-12)
    np.testing.assert_allclose(R, Rotation.from_rotvec([0, 0, yaw]).as_matrix(), atol=1e-12)
    np.testing.assert_allclose(dp, 0, atol=1e-12)
    np.testing.assert_allclose(dR, 0, atol=1e-12)
    # outside the keyframes the end segment is extended linearly
    R, p, _, _ = oracle.lidar_pose(sc, -0.5)
    np.testing.assert_allclose(p, np.array([1, 2, 3]) * -0.5, atol=1e-12)
    np.testing.assert_allclose(R, Rotation.from_rotvec([0, 0, -yaw / 2]).as_matrix(), atol=1e-12)


def test_slerp_shortest_arc():
    """q and -q are the same rotation; SLERP takes the shorter arc."""
    sc = _single_scene([[0, 0, 5]], [[0.1] * 3], [0.0], [[1, 1, 1]])
    a = math.radians(40.0)
    sc.traj_t = np.array([0.0, 1.0])
    sc.traj_p = np.zeros((2, 3))
    sc.traj_q = np.array([[1, 0, 0, 0], [-math.cos(a / 2), 0, -math.sin(a / 2), 0]])
    R, _, _, _ = oracle.lidar_pose(sc, 0.5)
    np.testing.assert_allclose(R, Rotation.from_rotvec([0, a / 2, 0]).as_matrix(), atol=1e-12)


def test_frame_pose_matches_library_composition():
    """Eq. 1: T^n = T_L(t + delta) * L_T_i; X^n = (T^n)^-1 X (Eq. 2) --
    against scipy's rotation-vector exponential and numpy's inverse."""
    p = scenes.tiny_problem()
    sc = p.scenes[0]
    ext = np.array([0.3, -0.2, 0.5, 0.4, -0.1, 0.2])
    for delta in [0.0, 0.07, -0.13]:
        R_wL, p_wL, _, _ = oracle.lidar_pose(sc, 0.4 + delta)
        Re = Rotation.from_rotvec(ext[:3]).as_matrix()
        T = np.eye(4)
        T[:3, :3] = R_wL @ Re
        T[:3, 3] = R_wL @ ext[3:] + p_wL
        Tinv = np.linalg.inv(T)
        R_cw, t_cw = oracle.frame_pose(sc, ext, delta, 0.4)
        np.testing.assert_allclose(R_cw, Tinv[:3, :3], atol=1e-12)
        np.testing.assert_allclose(t_cw, Tinv[:3, 3], atol=1e-12)


def test_rotated_anisotropic_projection():
    """Eq. 3 and EWA: the oracle's 2D covariance equals J Sigma_c J^T + lp I
    with Sigma_c built from the quaternion product q_c = q_cw * q (scipy) and
    J the finite-difference Jacobian of the pinhole map."""
    rng = np.random.default_rng(11)
    n = 16
    X = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(3, 8, n)], 1)
    q = rng.normal(size=(n, 4))
    ls = np.log(rng.uniform(0.05, 0.5, (n, 3)))
    sc = scenes.Scene(X, q, ls, np.zeros(n), np.ones((n, 3)), np.array([0.0]), np.zeros((1, 3)),
                      np.array([[1.0, 0, 0, 0]]))
    Rcw = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    tcw = np.array([0.2, -0.1, 0.3])
    cam = scenes.Camera(640, 480, 500.0, 480.0, 320.0, 240.0)
    pr = oracle.project(sc, cam, Rcw, tcw, oracle.Opts())
    rcw = Rotation.from_matrix(Rcw)
    for g in range(n):
        qg = Rotation.from_quat(np.r_[q[g, 1:], q[g, 0]])  # scipy is (x, y, z, w)
        Rc = (rcw * qg).as_matrix()
        Sc = Rc @ np.diag(np.exp(2 * ls[g])) @ Rc.T
        pc = Rcw @ X[g] + tcw

        def pin(v):
            return np.array([cam.fx * v[0] / v[2] + cam.cx, cam.fy * v[1] / v[2] + cam.cy])
        Jfd = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            Jfd[:, k] = (pin(pc + e) - pin(pc - e)) / 2e-6
        cov = Jfd @ Sc @ Jfd.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov"][g], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6)
        np.testing.assert_allclose(pr["conic"][g], np.linalg.inv(cov)[[0, 0, 1], [0, 1, 1]], rtol=1e-6)
        np.testing.assert_allclose(pr["mean"][g], pin(pc), rtol=1e-12)
        assert pr["depth"][g] == pytest.approx(pc[2], rel=1e-12)


def test_jacobian_frustum_clamp():
    """Centres outside the field of view widened by 15% of the image per
    side (3DGS's EWA) use the Jacobian of the pinhole map at the clamped
    ray (x/z, y/z limited), computed here by finite differences at that ray;
    inside it the plain Jacobian is used."""
    cam = scenes.Camera(200, 100, 100.0, 90.0, 90.0, 45.0)
    lim = [(-(cam.cx + 0.15 * cam.width) / cam.fx, (cam.width - cam.cx + 0.15 * cam.width) / cam.fx),
           (-(cam.cy + 0.15 * cam.height) / cam.fy, (cam.height - cam.cy + 0.15 * cam.height) / cam.fy)]
    X = np.array([[5.0, 0.3, 2.0], [-4.0, -3.0, 1.5], [0.2, 0.1, 3.0], [1.0, 2.5, 1.0]])
    rng = np.random.default_rng(2)
    q = rng.normal(size=(4, 4))
    ls = np.log(rng.uniform(0.2, 0.6, (4, 3)))
    sc = scenes.Scene(X, q, ls, np.full(4, 3.0), np.ones((4, 3)), np.array([0.0]), np.zeros((1, 3)),
                      np.array([[1.0, 0, 0, 0]]))
    pr = oracle.project(sc, cam, np.eye(3), np.zeros(3), oracle.Opts())
    pr_free = oracle.project(sc, cam, np.eye(3), np.zeros(3), oracle.Opts(frustum_margin=-1.0))
    clamped = 0
    for g in range(4):
        x, y, z = X[g]
        jx = min(max(x / z, lim[0][0]), lim[0][1])
        jy = min(max(y / z, lim[1][0]), lim[1][1])
        clamped += (jx != x / z) or (jy != y / z)
        pc = np.array([jx * z, jy * z, z])

        def pin(v):
            return np.array([cam.fx * v[0] / v[2] + cam.cx, cam.fy * v[1] / v[2] + cam.cy])
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            J[:, k] = (pin(pc + e) - pin(pc - e)) / 2e-6
        Rg = Rotation.from_quat(np.r_[q[g, 1:], q[g, 0]]).as_matrix()
        S = Rg @ np.diag(np.exp(2 * ls[g])) @ Rg.T
        cov = J @ S @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov"][g], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6)
        np.testing.assert_allclose(pr["mean"][g], pin(X[g]), rtol=1e-12)  # the mean is not clamped
        if (jx == x / z) and (jy == y / z):
            np.testing.assert_allclose(pr["cov"][g], pr_free["cov"][g], rtol=1e-12)
    assert clamped == 3


def test_rigid_motion_invariance():
    """Moving the points, the Gaussian orientations and the LiDAR trajectory
    by one rigid motion leaves every image unchanged (Eq. 1-3)."""
    p = scenes.tiny_problem()
    sc, fr = p.scenes[0], p.frames[0]
    ext = np.array([0.05, 0.02, -0.03, 0.1, 0.0, -0.05])
    M = Rotation.from_rotvec([0.4, -0.7, 0.2])
    t0 = np.array([3.0, -2.0, 1.5])
    sc2 = copy.deepcopy(sc)
    sc2.X = M.apply(sc.X.astype(np.float64)) + t0
    qg = Rotation.from_quat(np.c_[sc.quat[:, 1:], sc.quat[:, 0]].astype(np.float64))
    qq = (M * qg).as_quat()
    sc2.quat = np.c_[qq[:, 3], qq[:, :3]]
    sc2.traj_p = M.apply(sc.traj_p) + t0
    tq = (M * Rotation.from_quat(np.c_[sc.traj_q[:, 1:], sc.traj_q[:, 0]])).as_quat()
    sc2.traj_q = np.c_[tq[:, 3], tq[:, :3]]
    a = oracle.render(sc, fr, ext, 0.01)
    b = oracle.render(sc2, fr, ext, 0.01)
    np.testing.assert_allclose(a[0], b[0], atol=1e-10)
    np.testing.assert_array_equal(a[2], b[2])


def test_stationary_trajectory_has_zero_time_gradient():
    p = scenes.tiny_problem()
    sc = copy.deepcopy(p.scenes[0])
    sc.traj_p = np.zeros((2, 3))
    sc.traj_q = np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]])
    W = np.random.default_rng(0).normal(size=(64 * 48, 3))
    g = oracle.backward(sc, p.frames[0], p.ext[0], 0.0, W)
    assert g["delta"][0] == 0.0
    assert np.any(g["ext"] != 0)


def _clamped_scene():
    """Large Gaussians centred beyond the Jacobian clamp on every side of a
    64x48 image (|x/z| > 0.685 or |y/z| > 0.52), plus a few inside."""
    p = scenes.tiny_problem()
    sc = p.scenes[0]
    rng = np.random.default_rng(21)
    X = np.array([[1.7, 0.2, 2.0], [-1.8, -0.3, 2.4], [0.3, 1.3, 2.2], [-0.2, -1.25, 2.1],
                  [1.6, 1.2, 2.0], [0.1, 0.05, 4.0], [-0.4, 0.3, 3.0], [0.5, -0.2, 5.0]])
    n = len(X)
    sc2 = scenes.Scene(X, rng.normal(size=(n, 4)), np.log(rng.uniform(0.3, 0.6, (n, 3))),
                       rng.normal(size=n), rng.uniform(size=(n, 3)), sc.traj_t, sc.traj_p, sc.traj_q)
    return p, sc2


def _fd_check(opts, seed, opacity_shift=0.0, clamped=False):
    p = scenes.tiny_problem()
    sc, fr = p.scenes[0], p.frames[0]
    if clamped:
        p, sc = _clamped_scene()
    sc.logit_opacity = sc.logit_opacity.astype(np.float64) + opacity_shift
    ext = p.ext_target[0]  # a non-identity extrinsic
    delta = 0.013
    W = np.random.default_rng(seed).normal(size=(fr.camera.width * fr.camera.height, 3))
    # pixels on a discontinuity (alpha skip/clamp, T stop) get no weight
    W[oracle.render(sc, fr, ext, delta, opts)[3] != 0] = 0.0

    def L(scene, e, d):
        rgb, _, _, flags = oracle.render(scene, fr, e, d, opts)
        return float((rgb * W).sum()), flags

    L0, flags = L(sc, ext, delta)
    G = oracle.backward(sc, fr, ext, delta, W, opts)
    errs = {}
    for k in range(6):
        h = 1e-6
        e1, e2 = ext.copy(), ext.copy()
        e1[k] += h
        e2[k] -= h
        fd = (L(sc, e1, delta)[0] - L(sc, e2, delta)[0]) / (2 * h)
        errs["ext%d" % k] = abs(fd - G["ext"][k]) / max(abs(G["ext"][k]), 1e-3)
    fd = (L(sc, ext, delta + 1e-6)[0] - L(sc, ext, delta - 1e-6)[0]) / 2e-6
    errs["delta"] = abs(fd - G["delta"][0]) / max(abs(G["delta"][0]), 1e-3)
    for name in ["quat", "log_scale", "logit_opacity", "rgb"]:
        ga = G[name].ravel()
        scale = np.abs(ga).max()
        for i in np.argsort(-np.abs(ga))[:12]:
            s1, s2 = copy.deepcopy(sc), copy.deepcopy(sc)
            a1 = getattr(s1, name).astype(np.float64)
            a2 = getattr(s2, name).astype(np.float64)
            h = 1e-6 * max(1.0, abs(a1.ravel()[i]))
            a1.ravel()[i] += h
            a2.ravel()[i] -= h
            setattr(s1, name, a1)
            setattr(s2, name, a2)
            fd = (L(s1, ext, delta)[0] - L(s2, ext, delta)[0]) / (2 * h)
            errs["%s%d" % (name, i)] = abs(fd - ga[i]) / scale
    return errs, flags[W[:, 0] != 0]


@pytest.mark.parametrize("mode", ["smooth", "default", "opaque_bg", "clamped"])
def test_gradients_match_finite_differences(mode):
    """Every oracle gradient (Gaussian parameters, extrinsic, time offset)
    against FP64 central differences of the oracle's forward.  'opaque_bg'
    raises the opacities so that compositing terminates early at many pixels
    and uses a non-zero background."""
    if mode == "smooth":
        errs, flags = _fd_check(oracle.SMOOTH, 7)
    elif mode == "default":
        errs, flags = _fd_check(oracle.Opts(), 7)
    elif mode == "opaque_bg":
        errs, flags = _fd_check(oracle.Opts(bg=(0.2, 0.5, 0.8)), 8, opacity_shift=5.0)
    else:
        errs, flags = _fd_check(oracle.Opts(), 9, clamped=True)
    assert np.all(flags == 0)
    worst = max(errs, key=errs.get)
    assert errs[worst] < 1e-6, (worst, errs[worst])


def test_bin_sort_matches_python_stable_sort():
    """Tile binning + depth order against Python's stable sort of the
    emitted (key, value) pairs."""
    tiles = [(5, 3), (2, 4), (7, 1)]
    npf = [40, 25, 30]
    rect, depth = scenes.random_splat_records(9, tiles, npf, tie_fraction=0.5, max_extent_tiles=4)
    keys, vals, ranges = oracle.bin_sort(tiles, npf, rect, depth)
    pairs = []
    rec = 0
    tile_off = 0
    for (tx, ty), n in zip(tiles, npf):
        for g in range(n):
            x0, y0, x1, y1 = rect[rec + g]
            bits = int(np.frombuffer(depth[rec + g].tobytes(), np.uint32)[0])
            for yy in range(y0, y1 + 1):
                for xx in range(x0, x1 + 1):
                    pairs.append(((tile_off + yy * tx + xx) << 32 | bits, g))
        rec += n
        tile_off += tx * ty
    pairs.sort(key=lambda kv: kv[0])  # stable: equal keys keep emission order
    assert len(pairs) == len(keys)
    assert [k for k, _ in pairs] == [int(k) for k in keys]
    assert [v for _, v in pairs] == [int(v) for v in vals]
    for t in range(tile_off):
        idx = [i for i, (k, _) in enumerate(pairs) if k >> 32 == t]
        if idx:
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(ranges[t]) == (0, 0)
    assert sum(1 for i in range(1, len(pairs)) if pairs[i][0] == pairs[i - 1][0]) > 0


def test_l1_matches_numpy():
    rng = np.random.default_rng(1)
    a, b = rng.uniform(size=(7, 5, 3)), rng.uniform(size=(7, 5, 3))
    b[0, 0, 0] = a[0, 0, 0]
    loss, grad = oracle.l1(a, b)
    assert loss == pytest.approx(np.abs(a - b).mean(), rel=1e-14)
    np.testing.assert_array_equal(grad, np.sign(a - b) / a.size)


def _outcomes(sc, cam, pixels, opts=oracle.Opts(bg=BG)):
    """Every outcome (rgb, T, last) per pixel, the FP64 one first, and the flags."""
    rgb, T, last, flags, (nalt, alt) = oracle.render(sc, scenes.Frame(cam, 0.0), np.zeros(6), 0.0, opts,
                                                       pixels=pixels, alternatives=True)
    out = []
    for p in range(len(flags)):
        o = [(rgb[p], T[p], int(last[p]))]
        o += [(alt[p, k, :3], alt[p, k, 3], int(alt[p, k, 4])) for k in range(nalt[p])]
        out.append(o)
    return out, flags


def _same_outcomes(got, want):
    """The outcome sets agree (any order), colours and T to 1e-12."""
    assert len(got) == len(want), (got, want)
    for w in want:
        assert any(abs(g[1] - w[1]) < 1e-12 and g[2] == w[2] and np.abs(np.asarray(g[0]) - w[0]).max() < 1e-12
                   for g in got), (w, got)


# The renderer decides skip, stop, clamp and order on float32 values; where
# the exact value lies within the float32 evaluation's error bound of a
# threshold, either outcome is a correct result.  Each pin below places a
# pixel on such an edge (both outcomes, in closed form) and one just off it
# (the one FP64 outcome, no flag).  For these well-conditioned Gaussians the
# bound is a few 1e-5 in log2 units, so 1e-3 is clearly off the edge.

def test_alpha_min_edge_has_both_outcomes():
    """alpha = opacity exp(power) = alpha_min exactly: the Gaussian is
    composited (C = alpha c + (1 - alpha) bg) or skipped (C = bg)."""
    sc = _single_scene([[0, 0, 2]], [[0.1] * 3], [0.0], [[1.0, 0.5, 0.25]])
    cov = (60.0 * 0.1 / 2) ** 2 + 0.3  # EWA covariance of the on-axis Gaussian, px^2
    amin = 1.0 / 255.0
    for shift, on_edge in ((0.0, True), (1e-3, False), (-1e-3, False)):
        # log2 alpha = log2 alpha_min + shift at a distance dx from the mean
        power = math.log(amin / 0.5) + shift * math.log(2.0)
        dx = math.sqrt(-2.0 * power * cov)
        cam = scenes.Camera(64, 48, 60.0, 60.0, 42.0 - dx, 24.0)
        (got,), flags = _outcomes(sc, cam, [[42, 24]])
        a = 0.5 * math.exp(power)
        composited = (a * np.array([1.0, 0.5, 0.25]) + (1 - a) * np.array(BG), 1 - a, 0)
        skipped = (np.array(BG), 1.0, -1)
        if on_edge:
            assert flags[0] == oracle.FLAG_BRANCH
            _same_outcomes(got, [composited, skipped])
        else:
            assert flags[0] == 0
            _same_outcomes(got, [composited if shift > 0 else skipped])


def test_stop_edge_has_both_outcomes():
    """T (1 - alpha) = t_min exactly at the second of two stacked Gaussians
    (alpha 0.98 then 0.9, t_min = 0.002): compositing stops before it, or
    composites it; just off the edge it stops."""
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    for a2, on_edge in ((0.9, True), (0.9 * (1 + 1e-3), False)):
        sc = _single_scene([[0, 0, 2], [0, 0, 3]], [[0.1] * 3] * 2, [math.log(49.0), math.log(a2 / (1 - a2))],
                           [c1, c2])
        opts = oracle.Opts(bg=BG, t_min=0.02 * 0.1)
        (got,), flags = _outcomes(sc, CAM, [[32, 24]], opts)
        stopped = (0.98 * c1 + 0.02 * np.array(BG), 0.02, 0)
        T2 = 0.02 * (1 - a2)
        through = (0.98 * c1 + 0.02 * a2 * c2 + T2 * np.array(BG), T2, 1)
        if on_edge:
            assert flags[0] == oracle.FLAG_BRANCH
            _same_outcomes(got, [stopped, through])
        else:
            assert flags[0] == 0
            _same_outcomes(got, [stopped])


def test_exponent_sign_edge_of_a_needle():
    """Along the long axis of a needle (scales 50 m x 1 mm x 1 mm, at 45
    degrees in the image, 2 m away) the exponent is -d^2 / (2 sigma_long^2),
    a few 1e-6, while its terms are of order 10: its float32 sign is not
    decided, so the Gaussian is composited or skipped (C = bg).  Across a
    moderate Gaussian the same offset is decided."""
    c = np.array([0.2, 0.9, 0.4])
    q45 = [math.cos(math.pi / 8), 0, 0, math.sin(math.pi / 8)]
    needle = _single_scene([[0, 0, 2]], [[50.0, 1e-3, 1e-3]], [0.0], [c], quats=[q45])
    (got,), flags = _outcomes(needle, CAM, [[36, 28]])
    assert flags[0] == oracle.FLAG_BRANCH
    rgb, T, last = got[0]
    a = 1 - T
    assert 0.49 < a <= 0.5 and last == 0  # alpha ~ opacity along the axis
    _same_outcomes(got, [(a * c + (1 - a) * np.array(BG), T, 0), (np.array(BG), 1.0, -1)])
    plain = _single_scene([[0, 0, 2]], [[0.3, 0.1, 0.1]], [0.0], [c], quats=[q45])
    (got,), flags = _outcomes(plain, CAM, [[36, 28]])
    assert flags[0] == 0 and len(got) == 1


def test_alpha_max_clamp_edge_flag():
    """opacity 0.995 with alpha_raw = alpha_max = 0.99 exactly at the pixel:
    the colour is continuous (one outcome) but the gradient is not, so the
    pixel is flagged CLAMP_EDGE; at the peak (0.995, clearly clamped) and
    1.5 px away (0.88) it is not."""
    sc = _single_scene([[0, 0, 2]], [[0.1] * 3], [math.log(199.0)], [[1.0, 1.0, 1.0]])
    cov = (60.0 * 0.1 / 2) ** 2 + 0.3
    dx = math.sqrt(-2.0 * math.log(0.99 / 0.995) * cov)
    cam = scenes.Camera(64, 48, 60.0, 60.0, 33.0 - dx, 24.0)
    (got,), flags = _outcomes(sc, cam, [[33, 24]])
    assert flags[0] == oracle.FLAG_CLAMP_EDGE and len(got) == 1
    assert got[0][1] == pytest.approx(0.01, abs=1e-12)
    cam2 = scenes.Camera(64, 48, 60.0, 60.0, 33.0, 24.0)
    outs, flags = _outcomes(sc, cam2, [[33, 24], [34, 24], [35, 24]])
    assert flags[0] == 0 and flags[2] == 0  # peak (clamped) and 2 px away (0.80)
    assert outs[0][0][1] == pytest.approx(0.01, abs=1e-12)


def _f32_neighbours(z):
    f = np.float32(z)
    return float(f), float(np.nextafter(f, np.float32(np.inf)))


def test_depth_order_by_float32_key_and_index():
    """The depth order is the float32 depth key, equal keys by Gaussian index
    (Eq. 5's depth order decided in float32): a Gaussian slightly farther in
    FP64 but with the same key, and a lower index, is composited first."""
    lo, hi = _f32_neighbours(4.0)
    c0, c1 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    z_far = lo + 0.25 * (hi - lo)  # rounds to lo, as does z = lo
    sc = _single_scene([[0, 0, z_far], [0, 0, lo]], [[0.1] * 3] * 2, [0.0, 0.0], [c0, c1])
    rgb, T, last, flags = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(bg=BG), pixels=[[32, 24]])
    assert flags[0] == 0 and last[0] == 1
    pr = oracle.project(sc, CAM, np.eye(3), np.zeros(3), oracle.Opts())
    assert pr["zkey"][0] == pr["zkey"][1] == np.float32(lo)
    a0 = 1 - math.sqrt(T[0])  # both alphas are equal at the shared centre
    np.testing.assert_allclose(rgb[0], a0 * c0 + (1 - a0) * a0 * c1 + (1 - a0) ** 2 * np.array(BG), atol=1e-12)


def test_depth_tie_flag_on_an_undecided_rounding():
    """Two contributors, one at depth lo (a float) and one at the exact
    midpoint between lo and the next float (its key is not decided: either
    rounding is within the float32 evaluation's error).  With the midpoint
    Gaussian first in index order, one rounding puts it before the other and
    one after: DEPTH_TIE.  With it second in index order, both roundings give
    the same order (equal keys go by index): no flag.  Moved 1e-9 m off the
    midpoint, the key is decided: no flag."""
    lo, hi = _f32_neighbours(4.0)
    mid = 0.5 * (lo + hi)
    for z, mid_first, flagged in ((mid, True, True), (mid, False, False), (mid + 1e-9, True, False)):
        Xs = [[0, 0, z], [0, 0, lo]] if mid_first else [[0, 0, lo], [0, 0, z]]
        sc = _single_scene(Xs, [[0.1] * 3] * 2, [0.0, 0.0], [[1, 0, 0], [0, 1, 0]])
        pr = oracle.project(sc, CAM, np.eye(3), np.zeros(3), oracle.Opts())
        k = 0 if mid_first else 1
        assert bool(pr["zamb"][k]) == (z == mid) and not pr["zamb"][1 - k]
        flags = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(bg=BG), pixels=[[32, 24]])[3]
        assert flags[0] == (oracle.FLAG_DEPTH_TIE if flagged else 0), (z, mid_first)


def test_near_plane_culling_decided_in_float32():
    """Culling at the near plane compares the float32 depth key with float32
    near_z: a centre at the midpoint above float32(0.2) may be kept or
    culled (NEAR_EDGE where it would contribute); at 0.3 m it is decided."""
    lo, hi = _f32_neighbours(0.2)
    for z, flagged in ((0.5 * (lo + hi), True), (0.3, False)):
        sc = _single_scene([[0, 0, z]], [[0.01] * 3], [0.0], [[1, 1, 1]])
        pr = oracle.project(sc, CAM, np.eye(3), np.zeros(3), oracle.Opts())
        assert bool(pr["near_undecided"][0]) == flagged
        flags = oracle.render(sc, FRAME, np.zeros(6), 0.0, oracle.Opts(bg=BG), pixels=[[32, 24]])[3]
        assert flags[0] == (oracle.FLAG_NEAR_EDGE if flagged else 0)
    # exactly on float32(near_z) the key is not in front: culled, decided
    sc = _single_scene([[0, 0, lo]], [[0.01] * 3], [0.0], [[1, 1, 1]])
    pr = oracle.project(sc, CAM, np.eye(3), np.zeros(3), oracle.Opts())
    assert pr["valid"][0] == 0 and not pr["near_undecided"][0]


def test_branch_limit_flag():
    """More ambiguous decisions than OR_MAX_BRANCHES outcomes: twenty
    stacked Gaussians, each with alpha exactly alpha_min at the pixel, give
    2^20 outcomes: the pixel is flagged BRANCH_LIMIT (undecided)."""
    n = 20
    cov = (60.0 * 0.1 / 2) ** 2 + 0.3
    dx = math.sqrt(-2.0 * math.log((1 / 255.0) / 0.5) * cov)
    cam = scenes.Camera(64, 48, 60.0, 60.0, 42.0 - dx, 24.0)
    zs = [2.0 * (1 + 0.01 * k) for k in range(n)]
    # the same pixel offset at each depth: scale the Gaussians with depth
    sc = _single_scene([[0, 0, z] for z in zs], [[0.1 * z / 2.0] * 3 for z in zs], [0.0] * n, [[1, 1, 1]] * n)
    _, flags = _outcomes(sc, cam, [[42, 24]])
    assert flags[0] & oracle.FLAG_BRANCH_LIMIT and flags[0] & oracle.FLAG_BRANCH


def test_scale_clamp():
    """scale_max clamps the axis scales (voxel-size bound, Sec. III-D1)."""
    p = scenes.tiny_problem()
    sc = p.scenes[0]
    sc2 = copy.deepcopy(sc)
    sc2.log_scale = np.minimum(sc.log_scale.astype(np.float64), math.log(0.2))
    a = oracle.render(sc, p.frames[0], p.ext[0], 0.0, oracle.Opts(scale_max=0.2))
    b = oracle.render(sc2, p.frames[0], p.ext[0], 0.0, oracle.Opts())
    np.testing.assert_allclose(a[0], b[0], atol=1e-12)


# ------------------------------------------------------------ D-SSIM (Eq. 4)


def _ssim_scipy(a, b):
    """SSIM map from scipy's Gaussian filter: sigma 1.5, 11 taps (truncate at
    5 px), zero padding, per channel; constants of Wang et al."""
    from scipy.ndimage import gaussian_filter

    def f(x):
        return gaussian_filter(x, sigma=(1.5, 1.5, 0.0), mode="constant", cval=0.0, truncate=5.0 / 1.5)

    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ma, mb = f(a), f(b)
    saa, sbb, sab = f(a * a) - ma * ma, f(b * b) - mb * mb, f(a * b) - ma * mb
    return ((2 * ma * mb + C1) * (2 * sab + C2)) / ((ma * ma + mb * mb + C1) * (saa + sbb + C2))


def test_dssim_map_matches_scipy_gaussian_filter():
    """The oracle's SSIM map is the textbook SSIM computed with a library
    Gaussian filter (independent code path), on ragged sizes."""
    rng = np.random.default_rng(3)
    imgs = [rng.uniform(size=(19, 23, 3)), rng.uniform(size=(7, 40, 3))]
    tgts = [np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1) for x in imgs]
    loss, _, maps = oracle.dssim(imgs, tgts, with_map=True)
    ref = [_ssim_scipy(a, b) for a, b in zip(imgs, tgts)]
    for m, r in zip(maps, ref):
        np.testing.assert_allclose(m, r, rtol=0, atol=1e-12)
    n = sum(x.size for x in imgs)
    assert loss == pytest.approx(1 - sum(r.sum() for r in ref) / n, rel=1e-12)


def test_dssim_identical_images_and_constant_closed_form():
    rng = np.random.default_rng(4)
    a = rng.uniform(size=(15, 18, 3))
    loss, (g,) = oracle.dssim([a], [a])
    assert abs(loss) < 1e-14 and np.abs(g).max() < 1e-13  # SSIM = 1 is the maximum
    # constant images: away from the border the window sees only the constants,
    # so SSIM = (2 a b + C1) / (a^2 + b^2 + C1) (the variance factor is 1)
    ca, cb = 0.3, 0.7
    _, _, (m,) = oracle.dssim([np.full((31, 33, 3), ca)], [np.full((31, 33, 3), cb)], with_map=True)
    C1 = 0.01 ** 2
    assert m[15, 16, 1] == pytest.approx((2 * ca * cb + C1) / (ca * ca + cb * cb + C1), rel=1e-13)


@pytest.mark.parametrize("lambda1", [1.0, 0.2])
def test_photo_loss_gradient_matches_central_differences(lambda1):
    """d L_photo / d image against FP64 central differences (D-SSIM alone for
    lambda1 = 1, the paper's mix for 0.2), at pixels near the border, in the
    interior and in a second image."""
    rng = np.random.default_rng(5)
    imgs = [rng.uniform(0.1, 0.9, size=(12, 15, 3)), rng.uniform(0.1, 0.9, size=(9, 8, 3))]
    tgts = [rng.uniform(0.1, 0.9, size=x.shape) for x in imgs]
    loss, grads = oracle.photo_loss(imgs, tgts, lambda1)
    for (k, y, x, c) in [(0, 0, 0, 0), (0, 6, 7, 1), (0, 11, 14, 2), (0, 3, 12, 0), (1, 4, 4, 1), (1, 8, 0, 2)]:
        h = 1e-6
        up = [v.copy() for v in imgs]
        dn = [v.copy() for v in imgs]
        up[k][y, x, c] += h
        dn[k][y, x, c] -= h
        fd = (oracle.photo_loss(up, tgts, lambda1)[0] - oracle.photo_loss(dn, tgts, lambda1)[0]) / (2 * h)
        assert grads[k][y, x, c] == pytest.approx(fd, rel=1e-6, abs=1e-12), (k, y, x, c)


# ----------------------------------------------- voxel downsampling (Sec. III-D)


def _voxel_brute(X, v):
    """Definition, point by point: the first point (by index) of every
    voxel, coordinates from float32 quotients."""
    seen, kept = set(), []
    v32 = np.float32(v)
    for i, p in enumerate(np.asarray(X, np.float32)):
        q = tuple(int(np.floor(c / v32)) if np.isfinite(np.floor(c / v32)) else None for c in p)
        if None in q or any(abs(c) >= oracle.VOXEL_LIMIT for c in q):
            continue
        if q not in seen:
            seen.add(q)
            kept.append(i)
    return np.array(kept, np.int64)


@pytest.mark.parametrize("v", [0.1, 0.05, 0.02, 0.5])
def test_voxel_downsample_matches_point_by_point_definition(v):
    rng = np.random.default_rng(int(v * 1000))
    # clustered points: many share voxels; negative coordinates; exact multiples of v
    c = rng.uniform(-3, 3, (40, 3))
    X = (c[rng.integers(0, 40, 3000)] + rng.normal(0, 2 * v, (3000, 3))).astype(np.float32)
    X[:50] = (np.round(X[:50] / v) * v).astype(np.float32)
    kept = oracle.voxel_downsample(X, v)
    np.testing.assert_array_equal(kept, _voxel_brute(X, v))
    # properties: kept voxels are distinct, every occupied voxel is kept once,
    # and the kept point is the voxel's smallest index
    q = np.floor(X / np.float32(v)).astype(np.int64)
    keys = {tuple(r) for r in q}
    assert len(kept) == len(keys) == len({tuple(q[i]) for i in kept})
    first = {}
    for i, r in enumerate(map(tuple, q)):
        first.setdefault(r, i)
    assert sorted(first.values()) == list(kept)


def test_voxel_downsample_drops_non_finite_and_far_points():
    X = np.array([[0.01, 0.02, 0.03], [np.nan, 0, 0], [0.04, 0.01, 0.02], [np.inf, 1, 1],
                  [3e6, 0, 0], [-0.05, 0.0, 0.0]], np.float32)
    np.testing.assert_array_equal(oracle.voxel_downsample(X, 0.1), [0, 5])
    assert len(oracle.voxel_downsample(X[[1, 3]], 0.1)) == 0


def _rect_cases(seed=21, n=80):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-0.9, 0.9, n), rng.uniform(2.0, 5.0, n)], 1)
    q = rng.normal(size=(n, 4))
    ls = np.log(rng.uniform(0.08, 0.4, (n, 3)))
    op = np.exp(-rng.uniform(np.log(1.2), np.log(40.0), n))  # opacity 0.025..0.83, log-uniform
    lo = np.log(op / (1 - op))
    sc = scenes.Scene(X, q, ls, lo, np.ones((n, 3)), np.array([0.0]), np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]))
    cam = scenes.Camera(320, 240, 200.0, 200.0, 159.5, 119.5)
    return sc, cam


def test_tile_rect_holds_every_pixel_that_reaches_alpha_min():
    """Reading 8 by brute force: for anisotropic Gaussians of every
    orientation and opacities from 0.025 to 0.83, every pixel centre where
    opacity * exp(-1/2 d^T conic d) >= alpha_min lies in a tile of the
    Gaussian's rectangle, and the rectangle reaches at most one tile beyond
    the tiles of those pixels on each side.  Its extent is therefore the
    alpha = alpha_min ellipse: a fixed number of sigmas, or an extent that
    ignores the opacity, fails one of the two bounds."""
    sc, cam = _rect_cases()
    T = 16
    pr = oracle.project(sc, cam, np.eye(3), np.zeros(3), oracle.Opts(), T)
    u, v = np.meshgrid(np.arange(cam.width, dtype=np.float64), np.arange(cam.height, dtype=np.float64))
    tight = 0
    for g in np.nonzero(pr["valid"])[0]:
        a, b, c = pr["conic"][g]
        dx, dy = u - pr["mean"][g][0], v - pr["mean"][g][1]
        alpha = pr["opacity"][g] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        hit = alpha >= 1.0 / 255.0
        x0, y0, x1, y1 = pr["rect"][g]
        tx, ty = (u[hit] // T).astype(int), (v[hit] // T).astype(int)
        assert np.all((tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)), g
        if hit.any():
            assert x0 >= tx.min() - 1 and x1 <= tx.max() + 1 and y0 >= ty.min() - 1 and y1 <= ty.max() + 1, g
            tight += 1
    assert tight >= 60
