"""The paper's attribute model F(X | Theta) (Sec. III-C) on the GPU: the
Instant-NGP hash-grid encoding of each Gaussian's centre and an MLP whose
four heads give its colour, opacity, scale and rotation (gs_ngp_forward /
gs_ngp_backward).  The configuration follows Instant-NGP's defaults: 16
levels of 2 features, 2^19 entries per level, resolutions from 16 to 2048
growing geometrically, over the bounding box of the points.
"""
from __future__ import annotations

import math

import torch

from . import capi

HIDDEN, OUTPUTS = 64, 11


class HashGridConfig:
    def __init__(self, aabb_min, aabb_max, levels=16, log2_table=19, base_res=16, max_res=2048):
        self.aabb_min = [float(v) for v in aabb_min]
        self.aabb_max = [float(v) for v in aabb_max]
        self.levels, self.log2_table = levels, log2_table
        growth = math.exp((math.log(max_res) - math.log(base_res)) / max(levels - 1, 1))
        self.res = [int(math.floor(base_res * growth ** l)) for l in range(levels)]
        self.T = 1 << log2_table

    @staticmethod
    def for_points(X: torch.Tensor, margin=1e-3, **kw) -> "HashGridConfig":
        lo = X.min(dim=0).values.double()
        hi = X.max(dim=0).values.double()
        pad = margin * (hi - lo).clamp_min(1e-6)
        return HashGridConfig((lo - pad).tolist(), (hi + pad).tolist(), **kw)

    def c(self) -> capi.GsNgp:
        g = capi.GsNgp()
        f3 = capi.C.c_float * 3
        g.aabb_min = f3(*self.aabb_min)
        g.aabb_max = f3(*self.aabb_max)
        g.levels, g.log2_table = self.levels, self.log2_table
        g.res = (capi.C.c_int32 * 16)(*(self.res + [1] * (16 - self.levels)))
        return g

    def param_count(self) -> int:
        return capi.gs_ngp_param_count(self.c())

    def blocks(self):
        """(name, numel) of the parameter blocks of theta, in order."""
        D = 2 * self.levels
        return [("tables", self.levels * self.T * 2), ("W1", HIDDEN * D), ("b1", HIDDEN), ("W2", HIDDEN * HIDDEN),
                ("b2", HIDDEN), ("W3", OUTPUTS * HIDDEN), ("b3", OUTPUTS)]


class HashGridMLP:
    """Parameters theta (one float32 tensor) and the forward/backward calls.

    Initialisation: tables uniform in +-1e-4 (Instant-NGP), weights uniform
    in +-sqrt(6 / fan_in), biases zero except the heads, whose biases start
    the Gaussians as in 3DGS: opacity 0.1, the given log scale, identity
    rotation; colours start near 0.5."""

    def __init__(self, cfg: HashGridConfig, device="cuda", seed=0, init_log_scale=math.log(0.05)):
        self.cfg, self.device = cfg, torch.device(device)
        self.cfg_c = cfg.c()
        n = cfg.param_count()
        gen = torch.Generator(device="cpu").manual_seed(seed)
        theta = torch.zeros(n, dtype=torch.float32)
        o = 0
        D = 2 * cfg.levels
        for name, numel in cfg.blocks():
            blk = theta[o:o + numel]
            if name == "tables":
                blk.uniform_(-1e-4, 1e-4, generator=gen)
            elif name.startswith("W"):
                fan = {"W1": D, "W2": HIDDEN, "W3": HIDDEN}[name]
                b = math.sqrt(6.0 / fan) * (0.1 if name == "W3" else 1.0)
                blk.uniform_(-b, b, generator=gen)
            elif name == "b3":
                blk.copy_(torch.tensor([0, 0, 0, math.log(0.1 / 0.9)] + [init_log_scale] * 3 + [1, 0, 0, 0],
                                       dtype=torch.float32))
            o += numel
        assert o == n
        self.theta = theta.to(self.device)
        self.grad = torch.zeros_like(self.theta)

    def forward(self, X: torch.Tensor, out: dict):
        """Writes out['rgb'], ['logit_opacity'], ['log_scale'], ['quat'] for the points X."""
        capi.gs_ngp_forward(self.cfg_c, self.theta, X, out["rgb"], out["logit_opacity"], out["log_scale"],
                            out["quat"])

    def backward(self, X: torch.Tensor, grads: dict, accumulate=False):
        """Gradient of sum(grads[k] . attr_k) into self.grad."""
        if not accumulate:
            self.grad.zero_()
        capi.gs_ngp_backward(self.cfg_c, self.theta, X, grads["rgb"], grads["logit_opacity"], grads["log_scale"],
                             grads["quat"], self.grad)


def _main():
    """Times forward and backward on a synthetic cloud: points uniform in a
    120 x 40 x 15 m box, random upstream gradients on every point (CUDA
    events; one JSON line with the median times)."""
    import argparse
    import json
    import statistics

    ap = argparse.ArgumentParser(description=_main.__doc__)
    ap.add_argument("--points", type=int, default=831_000)
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args()
    n = a.points
    g = torch.Generator(device="cpu").manual_seed(0)
    X = (torch.rand((n, 3), generator=g) * torch.tensor([120.0, 40.0, 15.0]) - torch.tensor([10.0, 20.0, 2.0]))
    X = X.cuda()
    mlp = HashGridMLP(HashGridConfig.for_points(X), device="cuda")
    out = {"rgb": torch.empty((n, 3), device="cuda"), "logit_opacity": torch.empty(n, device="cuda"),
           "log_scale": torch.empty((n, 3), device="cuda"), "quat": torch.empty((n, 4), device="cuda")}
    grads = {k: torch.randn(v.shape, generator=g).cuda() * 1e-3 for k, v in out.items()}
    res = {"points": n}
    for name, fn in (("forward", lambda: mlp.forward(X, out)), ("backward", lambda: mlp.backward(X, grads))):
        for _ in range(min(3, a.reps)):
            fn()
        ts = []
        for _ in range(a.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[name + "_ms"] = statistics.median(ts)
    res["fault"] = capi.gs_ngp_fault()
    print(json.dumps(res))


if __name__ == "__main__":
    _main()
