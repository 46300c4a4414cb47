"""The hash-grid MLP F(X | Theta) (Sec. III-C) on the GPU, through the
C-ABI, against the FP64 oracle (oracle/ngp.py)."""
import numpy as np
import pytest
import torch

from oracle import ngp as ongp
from paper_2403_11577_gb300 import capi, ngp, scenes

from _util import ensure_built, rel_l2

pytestmark = pytest.mark.gpu

LO, HI = [-10.0, -8.0, -1.0], [30.0, 12.0, 9.0]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _random_theta(cfg, seed):
    """Parameters of the sizes the oracle expects, scaled so that every part
    of the model matters (tables +-0.5, weights ~ 1/sqrt(fan_in))."""
    rng = np.random.default_rng(seed)
    o = ongp.NgpConfig(cfg.aabb_min, cfg.aabb_max, levels=cfg.levels, log2_table=cfg.log2_table)
    theta = np.zeros(o.count())
    P = o.unpack(theta)
    P["tables"][...] = rng.uniform(-0.5, 0.5, P["tables"].shape)
    for k, fan in (("W1", o.D), ("W2", o.H), ("W3", o.H)):
        P[k][...] = rng.normal(0, 1.0 / np.sqrt(fan), P[k].shape)
    for k in ("b1", "b2", "b3"):
        P[k][...] = rng.normal(0, 0.1, P[k].shape)
    return o, theta.astype(np.float32)


def _attrs(n):
    return {"rgb": torch.empty((n, 3), device="cuda"), "logit_opacity": torch.empty(n, device="cuda"),
            "log_scale": torch.empty((n, 3), device="cuda"), "quat": torch.empty((n, 4), device="cuda")}


def _points(rng, n):
    X = rng.uniform(LO, HI, (n, 3))
    X[:4] = [LO, HI, [HI[0], LO[1], HI[2]], [LO[0] - 3.0, HI[1] + 2.0, 0.5]]  # corners and outside the box
    return X.astype(np.float32)


# A point whose hidden pre-activation lies within this fraction of the size
# of its terms can take the other ReLU branch on the GPU: the layers' split
# bf16 products carry a relative error of about 2^-16 (1.5e-5) of those terms.
RELU_FLAG = 1e-4


@pytest.mark.parametrize("log2_table,levels", [(19, 16), (12, 16), (12, 6)])
def test_ngp_forward_matches_oracle(log2_table, levels):
    """400 points: three full tiles of 128 and a ragged tail; six levels
    leave the encoding columns beyond 2L as zero padding."""
    cfg = ngp.HashGridConfig(LO, HI, log2_table=log2_table, levels=levels)
    o, theta = _random_theta(cfg, 1)
    assert cfg.res == o.res and cfg.param_count() == o.count()
    mlp = ngp.HashGridMLP(cfg)
    mlp.theta.copy_(torch.from_numpy(theta))
    X = _points(np.random.default_rng(2), 400)
    out = _attrs(len(X))
    mlp.forward(torch.from_numpy(X).cuda(), out)
    ref = ongp.forward(o, theta.astype(np.float64), X)
    for k in ref:
        np.testing.assert_allclose(out[k].cpu().numpy(), ref[k], rtol=0, atol=5e-5, err_msg=k)


@pytest.mark.parametrize("log2_table,levels", [(19, 16), (10, 16), (12, 6)])
def test_ngp_backward_matches_oracle(log2_table, levels):
    """Every parameter block of the gradient, with dense, hashed and (small
    tables) colliding levels, and with fewer levels than the 16 column pairs
    of the tensor-core layout.  Points with a ReLU decision within RELU_FLAG
    of zero carry no upstream gradient (on both sides)."""
    cfg = ngp.HashGridConfig(LO, HI, log2_table=log2_table, levels=levels)
    o, theta = _random_theta(cfg, 3)
    mlp = ngp.HashGridMLP(cfg)
    mlp.theta.copy_(torch.from_numpy(theta))
    rng = np.random.default_rng(4)
    X = _points(rng, 300)
    d = {"rgb": rng.normal(size=(300, 3)), "logit_opacity": rng.normal(size=300),
         "log_scale": rng.normal(size=(300, 3)), "quat": rng.normal(size=(300, 4))}
    flagged = ongp.relu_margins(o, theta.astype(np.float64), X) < RELU_FLAG
    assert flagged.sum() <= 30
    for v in d.values():
        v[flagged] = 0.0
    mlp.backward(torch.from_numpy(X).cuda(), {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in d.items()})
    got = mlp.grad.cpu().numpy()
    ref = ongp.backward(o, theta.astype(np.float64), X, d["rgb"], d["logit_opacity"], d["log_scale"], d["quat"])
    off = 0
    for name, numel in cfg.blocks():
        assert rel_l2(got[off:off + numel], ref[off:off + numel]) <= 1e-4, name
        off += numel


def test_ngp_on_the_accumulated_cloud():
    """The 1M-point cloud of the batched scene with the default configuration
    (2^19 entries, initial parameters): attributes of sampled points, and the
    full gradient for attribute gradients on those points only (the oracle's
    backward over them is then exact)."""
    X = scenes.batched_problem(n=1_000_000).scenes[0].X
    Xd = torch.from_numpy(X).cuda()
    cfg = ngp.HashGridConfig.for_points(Xd)
    mlp = ngp.HashGridMLP(cfg, seed=5)
    o = ongp.NgpConfig(cfg.aabb_min, cfg.aabb_max)
    assert o.res == cfg.res
    theta = mlp.theta.cpu().numpy().astype(np.float64)
    out = _attrs(len(X))
    mlp.forward(Xd, out)
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(len(X), 120, replace=False))
    idx = idx[ongp.relu_margins(o, theta, X[idx]) >= RELU_FLAG]
    assert len(idx) >= 100
    ref = ongp.forward(o, theta, X[idx])
    for k in ref:
        np.testing.assert_allclose(out[k].cpu().numpy()[idx], ref[k], rtol=0, atol=2e-5, err_msg=k)
    m = len(idx)
    dd = {"rgb": rng.normal(size=(m, 3)), "logit_opacity": rng.normal(size=m),
          "log_scale": rng.normal(size=(m, 3)), "quat": rng.normal(size=(m, 4))}
    full = {k: torch.zeros_like(v) for k, v in out.items()}
    for k, v in dd.items():
        full[k][torch.from_numpy(idx).cuda()] = torch.from_numpy(v.astype(np.float32)).cuda().view(-1, *full[k].shape[1:])
    mlp.backward(Xd, full)
    ref_g = ongp.backward(o, theta, X[idx], dd["rgb"], dd["logit_opacity"], dd["log_scale"], dd["quat"])
    got = mlp.grad.cpu().numpy()
    off = 0
    for name, numel in cfg.blocks():
        assert rel_l2(got[off:off + numel], ref_g[off:off + numel]) <= 1e-4, name
        off += numel
    assert capi.gs_ngp_fault() == 0  # no tensor-core wait ran out


def test_joint_calibration_through_the_hash_grid_mlp():
    """Joint calibration (Sec. III-C, III-D): the Gaussians' attributes are
    learned through F(X | Theta) from its initialisation while the extrinsic
    and the time offset are recovered from 1 deg / 10 cm / 10 ms, with
    L_photo on the bottom half of every frame of a small surface scene."""
    from paper_2403_11577_gb300 import calib
    p = scenes.calibration_problem(seed=3, n=150_000, frames=4, rot_deg=1.0, trans_m=0.1, delta0=0.01,
                                   trajectory="zigzag", attributes="surface")
    for f in p.frames:
        f.camera = scenes.Camera(704, 188, 276.0, 276.0, 341.0, 119.0)
        f.row0 = f.camera.height // 2
    res = calib.run_calibration(p, iters=1500, warmup=300, model="mlp", loss="photo", log_every=0)
    st, fin = res["start"], res["final"]
    assert st["rot_deg"] > 0.9 and st["trans_cm"] > 9.0 and st["delta_ms"] > 9.0
    assert fin["rot_deg"] < 0.2 and fin["trans_cm"] < 3.0 and fin["delta_ms"] < 3.0, fin


def test_ngp_backward_on_coherent_points():
    """Points in scan order along a smooth curve (like a LiDAR ring): runs of
    consecutive points share cells at the coarse levels, so the backward
    sums them in the warp before adding to the table.  Every point has an
    upstream gradient; the full gradient against the oracle."""
    cfg = ngp.HashGridConfig(LO, HI, log2_table=14)
    o, theta = _random_theta(cfg, 7)
    mlp = ngp.HashGridMLP(cfg)
    mlp.theta.copy_(torch.from_numpy(theta))
    n = 2000
    s = np.linspace(0.0, 1.0, n)
    X = np.stack([LO[0] + 38.0 * s, LO[1] + 10.0 + 6.0 * np.sin(9.0 * s), LO[2] + 4.0 + np.cos(5.0 * s)], axis=1)
    X = X.astype(np.float32)
    rng = np.random.default_rng(8)
    d = {"rgb": rng.normal(size=(n, 3)), "logit_opacity": rng.normal(size=n),
         "log_scale": rng.normal(size=(n, 3)), "quat": rng.normal(size=(n, 4))}
    flagged = ongp.relu_margins(o, theta.astype(np.float64), X) < RELU_FLAG
    assert flagged.sum() <= n // 10
    for v in d.values():
        v[flagged] = 0.0
    mlp.backward(torch.from_numpy(X).cuda(), {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in d.items()})
    got = mlp.grad.cpu().numpy()
    ref = ongp.backward(o, theta.astype(np.float64), X, d["rgb"], d["logit_opacity"], d["log_scale"], d["quat"])
    off = 0
    for name, numel in cfg.blocks():
        assert rel_l2(got[off:off + numel], ref[off:off + numel]) <= 1e-4, name
        off += numel


def test_ngp_wait_limit_runs_out_and_the_context_stays_usable():
    """The waits for the tensor cores' MMAs are bounded.  With the bound set
    to 0, the first wait that finds its MMAs unfinished gives up: the
    backward reports bit 0 of gs_ngp_fault and poisons d_theta[0] with NaN
    (its gradient is incomplete), after a bounded drain of the MMAs in flight.
    With the default bound restored, the next call is clean and gives the
    gradient of a call made before (to the rounding of the table atomics)."""
    cfg = ngp.HashGridConfig(LO, HI, log2_table=12, levels=16)
    o, theta = _random_theta(cfg, 5)
    mlp = ngp.HashGridMLP(cfg)
    mlp.theta.copy_(torch.from_numpy(theta))
    rng = np.random.default_rng(6)
    X = torch.from_numpy(_points(rng, 1000)).cuda()
    d = {k: torch.from_numpy(rng.normal(size=s).astype(np.float32)).cuda()
         for k, s in (("rgb", (1000, 3)), ("logit_opacity", (1000,)), ("log_scale", (1000, 3)),
                      ("quat", (1000, 4)))}
    assert capi.gs_ngp_fault() == 0
    mlp.backward(X, d)
    torch.cuda.synchronize()
    before = mlp.grad.clone()
    assert capi.gs_ngp_fault() == 0 and bool(torch.isfinite(before).all())
    capi.gs_ngp_set_wait_limit(0)
    try:
        mlp.backward(X, d)
        torch.cuda.synchronize()
        assert capi.gs_ngp_fault() & 1
        assert bool(torch.isnan(mlp.grad[0]))
    finally:
        capi.gs_ngp_set_wait_limit(10 ** 9)
    mlp.backward(X, d)
    torch.cuda.synchronize()
    assert capi.gs_ngp_fault() == 0
    assert rel_l2(mlp.grad.cpu().numpy(), before.cpu().numpy()) < 1e-5
