"""FP64 oracle of the paper's attribute model F(X | Theta) (Sec. III-C):
Instant-NGP's multiresolution hash encoding of the Gaussian centre followed
by an MLP whose four heads give the Gaussian's colour, opacity, scale and
rotation.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes only the model family ("the model from Instant-NGP", input
the 3D position, four heads).  The readings, stated once here and in the
design notes:
  - encoding: L = 16 levels of F = 2 features, 2^19 table entries per level,
    resolutions N_l = floor(N_min * b^l) with N_min = 16 and b chosen so that
    N_{L-1} = 2048, over the scene's bounding box;
  - a level whose (N_l + 1)^3 vertices fit in the table is indexed densely,
    x + y (N_l + 1) + z (N_l + 1)^2, otherwise by the spatial hash
    (x * 1 XOR y * 2654435761 XOR z * 805459861) mod 2^32 mod T;
  - a point is mapped to p in [0, 1]^3 (clamped) by the bounding box, in
    float32 like the points themselves: p = clamp((x - lo) * inv), with lo
    the box minimum and inv = 1 / (hi - lo) rounded to float32 (a rough
    hash field is sensitive to the last bit of p, so the oracle takes the
    input coordinate in the same precision as the kernel and works in FP64
    from there); its
    level coordinates are q = p * N_l, its cell c = min(floor(q), N_l - 1)
    (so that p = 1 stays in the last cell), and its feature is the trilinear
    interpolation of the cell's 8 vertices with weights from q - c;
  - MLP: 32 -> 64 -> 64 -> 11, ReLU after the two hidden layers;
  - heads (the renderer's raw inputs): rgb = sigmoid(o[0:3]),
    logit_opacity = o[3], log_scale = o[4:7], quat = o[7:11].

Parameters are one flat vector: the L tables [L, T, F], then W1 [64, 32],
b1 [64], W2 [64, 64], b2 [64], W3 [11, 64], b3 [11].
"""
import math

import numpy as np

PRIMES = (1, 2654435761, 805459861)


class NgpConfig:
    def __init__(self, aabb_min, aabb_max, levels=16, features=2, log2_table=19, base_res=16, max_res=2048,
                 hidden=64, outputs=11):
        self.aabb_min = np.asarray(aabb_min, np.float64)
        self.aabb_max = np.asarray(aabb_max, np.float64)
        self.L, self.F, self.T = levels, features, 1 << log2_table
        self.b = math.exp((math.log(max_res) - math.log(base_res)) / (levels - 1))
        self.res = [int(math.floor(base_res * self.b ** l)) for l in range(levels)]
        self.H, self.O = hidden, outputs
        self.D = levels * features  # encoding width

    def sizes(self):
        """(name, shape) of the parameter blocks in order."""
        return [("tables", (self.L, self.T, self.F)), ("W1", (self.H, self.D)), ("b1", (self.H,)),
                ("W2", (self.H, self.H)), ("b2", (self.H,)), ("W3", (self.O, self.H)), ("b3", (self.O,))]

    def count(self):
        return sum(int(np.prod(s)) for _, s in self.sizes())

    def unpack(self, theta):
        out, o = {}, 0
        for name, shape in self.sizes():
            n = int(np.prod(shape))
            out[name] = theta[o:o + n].reshape(shape)
            o += n
        return out


def vertex_index(cfg, level, v):
    """Table slot of integer vertex v = (x, y, z) at `level` (dense or hashed)."""
    n1 = cfg.res[level] + 1
    x, y, z = (int(c) for c in v)
    if n1 ** 3 <= cfg.T:
        return x + y * n1 + z * n1 * n1
    h = ((x * PRIMES[0]) & 0xFFFFFFFF) ^ ((y * PRIMES[1]) & 0xFFFFFFFF) ^ ((z * PRIMES[2]) & 0xFFFFFFFF)
    return h % cfg.T


def unit_point(cfg, x):
    """p = clamp((x - lo) * inv, 0, 1) in float32 (see the module notes)."""
    lo = np.float32(cfg.aabb_min)
    inv = np.float32(1.0) / (np.float32(cfg.aabb_max) - lo)
    p = (np.asarray(x, np.float32) - lo) * inv
    return np.clip(p, np.float32(0), np.float32(1)).astype(np.float64)


def encode_point(cfg, tables, x):
    """Encoding of one point and the (level, slot, weight) list it reads."""
    p = unit_point(cfg, x)
    enc = np.zeros(cfg.D)
    taps = []
    for l in range(cfg.L):
        q = p * cfg.res[l]
        c = np.minimum(np.floor(q), cfg.res[l] - 1)
        f = q - c
        for corner in range(8):
            d = np.array([(corner >> a) & 1 for a in range(3)])
            w = float(np.prod(np.where(d == 1, f, 1.0 - f)))
            slot = vertex_index(cfg, l, c + d)
            enc[l * cfg.F:(l + 1) * cfg.F] += w * tables[l, slot]
            taps.append((l, slot, w))
    return enc, taps


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def forward(cfg, theta, X):
    """Attributes of every point: dict with rgb [n,3], logit_opacity [n],
    log_scale [n,3], quat [n,4]."""
    P = cfg.unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64).reshape(-1, 3)
    out = np.zeros((len(X), cfg.O))
    for i, x in enumerate(X):
        enc, _ = encode_point(cfg, P["tables"], x)
        h1 = np.maximum(P["W1"] @ enc + P["b1"], 0.0)
        h2 = np.maximum(P["W2"] @ h1 + P["b2"], 0.0)
        out[i] = P["W3"] @ h2 + P["b3"]
    return {"rgb": sigmoid(out[:, 0:3]), "logit_opacity": out[:, 3].copy(), "log_scale": out[:, 4:7].copy(),
            "quat": out[:, 7:11].copy()}


def relu_margins(cfg, theta, X):
    """Per point, the smallest |a| / (sum_k |W_jk x_k| + |b_j|) over the
    pre-activations a_j of both hidden layers: how close a ReLU decision is
    to zero relative to the size of the terms that form it.  A kernel whose
    products carry a relative error e can take a different decision only
    where this margin is below about e; tests exclude such points instead of
    comparing a gradient that depends on which side of zero a rounding fell."""
    P = cfg.unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64).reshape(-1, 3)
    out = np.zeros(len(X))
    for i, x in enumerate(X):
        enc, _ = encode_point(cfg, P["tables"], x)
        a1 = P["W1"] @ enc + P["b1"]
        s1 = np.abs(P["W1"]) @ np.abs(enc) + np.abs(P["b1"])
        h1 = np.maximum(a1, 0.0)
        a2 = P["W2"] @ h1 + P["b2"]
        s2 = np.abs(P["W2"]) @ h1 + np.abs(P["b2"])
        with np.errstate(divide="ignore", invalid="ignore"):
            m = np.concatenate([np.abs(a1) / s1, np.abs(a2) / s2])
        out[i] = np.nanmin(np.where(np.isfinite(m), m, np.inf))
    return out


def backward(cfg, theta, X, d_rgb, d_logit_opacity, d_log_scale, d_quat):
    """Gradient of sum(d_attr . attr) with respect to theta (flat)."""
    theta = np.asarray(theta, np.float64)
    P = cfg.unpack(theta)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    X = np.asarray(X, np.float64).reshape(-1, 3)
    d_rgb, d_lo = np.asarray(d_rgb, np.float64).reshape(-1, 3), np.asarray(d_logit_opacity, np.float64).ravel()
    d_ls, d_q = np.asarray(d_log_scale, np.float64).reshape(-1, 3), np.asarray(d_quat, np.float64).reshape(-1, 4)
    for i, x in enumerate(X):
        enc, taps = encode_point(cfg, P["tables"], x)
        a1 = P["W1"] @ enc + P["b1"]
        h1 = np.maximum(a1, 0.0)
        a2 = P["W2"] @ h1 + P["b2"]
        h2 = np.maximum(a2, 0.0)
        o = P["W3"] @ h2 + P["b3"]
        s = sigmoid(o[0:3])
        do = np.concatenate([d_rgb[i] * s * (1 - s), [d_lo[i]], d_ls[i], d_q[i]])
        G["W3"] += np.outer(do, h2)
        G["b3"] += do
        da2 = (P["W3"].T @ do) * (a2 > 0)
        G["W2"] += np.outer(da2, h1)
        G["b2"] += da2
        da1 = (P["W2"].T @ da2) * (a1 > 0)
        G["W1"] += np.outer(da1, enc)
        G["b1"] += da1
        denc = P["W1"].T @ da1
        for (l, slot, w) in taps:
            G["tables"][l, slot] += w * denc[l * cfg.F:(l + 1) * cfg.F]
    return np.concatenate([G[name].ravel() for name, _ in cfg.sizes()])
