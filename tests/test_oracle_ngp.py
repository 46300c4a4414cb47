"""Pins of the FP64 hash-grid MLP oracle (oracle/ngp.py), checked against
closed forms, an independent uint32 hash, torch's float64 linear layers and
central finite differences."""
import numpy as np
import pytest
import torch

from oracle import ngp


def _cfg(log2_table=19):
    return ngp.NgpConfig([-10.0, -8.0, -1.0], [30.0, 12.0, 9.0], log2_table=log2_table)


def test_levels_and_resolutions():
    cfg = _cfg()
    assert cfg.res[0] == 16 and cfg.res[-1] == 2048 and len(cfg.res) == 16
    assert all(b > a for a, b in zip(cfg.res, cfg.res[1:]))
    dense = [l for l in range(cfg.L) if (cfg.res[l] + 1) ** 3 <= cfg.T]
    assert dense == [0, 1, 2, 3, 4]


def test_dense_levels_interpolate_affine_fields_exactly():
    """Trilinear interpolation reproduces an affine function of the level
    coordinates exactly: a table holding a.v + c at every dense vertex v
    yields a.q + c at any point (q = p * N_l)."""
    cfg = _cfg()
    rng = np.random.default_rng(0)
    theta = np.zeros(cfg.count())
    P = cfg.unpack(theta)
    coef = rng.normal(size=(cfg.L, cfg.F, 4))
    for l in range(5):
        n1 = cfg.res[l] + 1
        z, y, x = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
        slots = (x + y * n1 + z * n1 * n1).ravel()
        for f in range(cfg.F):
            P["tables"][l, slots, f] = (coef[l, f, 0] * x + coef[l, f, 1] * y + coef[l, f, 2] * z).ravel() + coef[l, f, 3]
    for x in rng.uniform(cfg.aabb_min, cfg.aabb_max, (20, 3)):
        enc, _ = ngp.encode_point(cfg, P["tables"], x)
        p = ngp.unit_point(cfg, x)
        for l in range(5):
            q = p * cfg.res[l]
            want = coef[l, :, :3] @ q + coef[l, :, 3]
            np.testing.assert_allclose(enc[l * 2:(l + 1) * 2], want, rtol=1e-12, atol=1e-10)


def test_unit_point_is_the_float32_box_map():
    cfg = _cfg()
    x = np.array([1.2345678, -3.3, 8.99999])
    lo = cfg.aabb_min.astype(np.float32)
    inv = (np.float32(1) / (cfg.aabb_max.astype(np.float32) - lo)).astype(np.float32)
    want = ((x.astype(np.float32) - lo) * inv).astype(np.float32)
    np.testing.assert_array_equal(ngp.unit_point(cfg, x), want.astype(np.float64))
    assert abs(ngp.unit_point(cfg, x)[0] - (x[0] - cfg.aabb_min[0]) / 40.0) < 1e-7


def test_points_on_and_beyond_the_box_faces():
    """p is clamped to [0, 1]; a point on the far face uses the last cell
    (weight 1 on its far vertices), so the encoding is continuous there."""
    cfg = _cfg()
    rng = np.random.default_rng(6)
    tables = rng.normal(size=(cfg.L, cfg.T, cfg.F))
    top = cfg.aabb_max.copy()
    e_face, taps = ngp.encode_point(cfg, tables, top)
    e_near, _ = ngp.encode_point(cfg, tables, top - 1e-6 * (cfg.aabb_max - cfg.aabb_min))
    np.testing.assert_allclose(e_face, e_near, atol=2e-2)  # within a few float32 steps of the face
    assert all(0 <= s < cfg.T for (_, s, _) in taps)
    e_out, _ = ngp.encode_point(cfg, tables, top + 5.0)
    np.testing.assert_array_equal(e_out, e_face)


def test_hash_matches_uint32_arithmetic():
    """Hashed levels: (x * 1 ^ y * 2654435761 ^ z * 805459861) mod 2^32 mod T,
    against numpy's wrapping uint32 products."""
    cfg = _cfg()
    rng = np.random.default_rng(1)
    v = rng.integers(0, 2049, (200, 3)).astype(np.uint32)
    with np.errstate(over="ignore"):
        h = (v[:, 0] * np.uint32(1)) ^ (v[:, 1] * np.uint32(2654435761)) ^ (v[:, 2] * np.uint32(805459861))
    want = (h % np.uint32(cfg.T)).astype(np.int64)
    got = np.array([ngp.vertex_index(cfg, 10, row) for row in v])
    np.testing.assert_array_equal(got, want)


def _random_theta(cfg, rng):
    theta = np.zeros(cfg.count())
    P = cfg.unpack(theta)
    P["tables"][...] = rng.uniform(-0.5, 0.5, P["tables"].shape)
    for k, fan in (("W1", cfg.D), ("W2", cfg.H), ("W3", cfg.H)):
        P[k][...] = rng.normal(0, 1.0 / np.sqrt(fan), P[k].shape)
    for k in ("b1", "b2", "b3"):
        P[k][...] = rng.normal(0, 0.1, P[k].shape)
    return theta


def test_mlp_matches_torch_float64_layers():
    cfg = _cfg(log2_table=12)
    rng = np.random.default_rng(2)
    theta = _random_theta(cfg, rng)
    P = cfg.unpack(theta)
    X = rng.uniform(cfg.aabb_min, cfg.aabb_max, (16, 3))
    out = ngp.forward(cfg, theta, X)
    enc = torch.tensor(np.stack([ngp.encode_point(cfg, P["tables"], x)[0] for x in X]))
    t = {k: torch.tensor(v) for k, v in P.items() if k != "tables"}
    h = torch.relu(torch.nn.functional.linear(enc, t["W1"], t["b1"]))
    h = torch.relu(torch.nn.functional.linear(h, t["W2"], t["b2"]))
    o = torch.nn.functional.linear(h, t["W3"], t["b3"]).numpy()
    np.testing.assert_allclose(out["rgb"], 1 / (1 + np.exp(-o[:, :3])), rtol=1e-13)
    np.testing.assert_allclose(out["logit_opacity"], o[:, 3], rtol=1e-13)
    np.testing.assert_allclose(out["log_scale"], o[:, 4:7], rtol=1e-13)
    np.testing.assert_allclose(out["quat"], o[:, 7:11], rtol=1e-13)


def test_relu_margins_against_torch_layers_and_an_exact_zero():
    """The margin is the smallest |pre-activation| / (sum of |terms| + |bias|)
    over both hidden layers (torch float64 layers on |W| and |x| give the
    scales); a bias set to cancel one pre-activation exactly gives 0."""
    cfg = _cfg(log2_table=12)
    rng = np.random.default_rng(5)
    theta = _random_theta(cfg, rng)
    P = cfg.unpack(theta)
    X = rng.uniform(cfg.aabb_min, cfg.aabb_max, (12, 3))
    enc = torch.tensor(np.stack([ngp.encode_point(cfg, P["tables"], x)[0] for x in X]))
    t = {k: torch.tensor(v) for k, v in P.items() if k != "tables"}
    lin = torch.nn.functional.linear
    a1 = lin(enc, t["W1"], t["b1"])
    s1 = lin(enc.abs(), t["W1"].abs(), t["b1"].abs())
    h1 = torch.relu(a1)
    a2 = lin(h1, t["W2"], t["b2"])
    s2 = lin(h1, t["W2"].abs(), t["b2"].abs())
    want = torch.cat([a1.abs() / s1, a2.abs() / s2], dim=1).min(dim=1).values.numpy()
    np.testing.assert_allclose(ngp.relu_margins(cfg, theta, X), want, rtol=1e-12)
    P["b1"][5] = -float(P["W1"][5] @ enc[3].numpy())
    assert ngp.relu_margins(cfg, theta, X[3:4])[0] < 1e-14


@pytest.mark.parametrize("log2_table", [19, 8])
def test_backward_matches_central_differences(log2_table):
    """Gradient of sum(d . F(X | theta)) against FP64 central differences, on
    entries of every parameter block (table entries the points read, dense
    and hashed; small tables force collisions)."""
    cfg = _cfg(log2_table)
    rng = np.random.default_rng(3)
    theta = _random_theta(cfg, rng)
    X = rng.uniform(cfg.aabb_min, cfg.aabb_max, (5, 3))
    d = {"rgb": rng.normal(size=(5, 3)), "logit_opacity": rng.normal(size=5), "log_scale": rng.normal(size=(5, 3)),
         "quat": rng.normal(size=(5, 4))}

    def S(th):
        out = ngp.forward(cfg, th, X)
        return sum(float((out[k] * d[k]).sum()) for k in d)

    g = ngp.backward(cfg, theta, X, d["rgb"], d["logit_opacity"], d["log_scale"], d["quat"])
    P = cfg.unpack(np.arange(cfg.count(), dtype=np.float64))
    # table entries actually read by the points, at a dense and a hashed level
    picks = []
    for l in (0, 3, 9, 15):
        _, taps = ngp.encode_point(cfg, cfg.unpack(theta)["tables"], X[0])
        slot = [s for (ll, s, w) in taps if ll == l][0]
        picks.append(int(P["tables"][l, slot, 1]))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P[k].ravel()
        picks += [int(flat[0]), int(flat[len(flat) // 2]), int(flat[-1])]
    for j in picks:
        h = 1e-6
        up, dn = theta.copy(), theta.copy()
        up[j] += h
        dn[j] -= h
        fd = (S(up) - S(dn)) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9), j
