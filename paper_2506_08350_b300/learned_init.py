"""Learned initialisation of each Gaussian's amplitude and phase.

Not in the paper.  A 4-layer ReLU MLP (16 -> 128 -> 128 -> 128 -> 16, BF16
operands, FP32 accumulation on the tensor cores) maps a Gaussian's geometry
and colour (mean, log-scale, rotation, opacity logit, RGB) to w = a e^{j phi}
per wavelength.  It is trained, with the library's own kernels (forward,
reverse mode, MSE loss, Adam on FP32 master weights, BF16 cast), on scenes
that the plain optimiser produced; the plain initialisation (amplitude = RGB,
phase uniform in [0, 2 pi)) stays as the fallback and as the baseline it is
compared with.

Python here only sequences library calls and keeps tensors; every
arithmetic step runs in libhcgs kernels (``hcgs_init_*``, ``hcgs_mlp_*``,
``hcgs_adam_step_multi``, ``hcgs_cast_bf16`` and the render path).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import PARAM_NAMES, Context
from .train import HologramTrainer

DIMS = ((128, 16), (128, 128), (128, 128), (16, 128))


class InitNet:
    """The network's FP32 master weights, BF16 copies and Adam state."""

    def __init__(self, ctx: Context, seed: int = 0, device: str = "cuda"):
        self.ctx = ctx
        rng = np.random.default_rng(seed)
        self.W32, self.b32 = [], []
        for k, (o, i) in enumerate(DIMS):
            scale = math.sqrt(2.0 / i) * (0.1 if k == len(DIMS) - 1 else 1.0)
            self.W32.append(torch.from_numpy((rng.normal(size=(o, i)) * scale).astype(np.float32)).to(device))
            self.b32.append(torch.zeros(o, dtype=torch.float32, device=device))
        self.W16 = [torch.empty(w.shape, dtype=torch.int16, device=device) for w in self.W32]
        self.gW = [torch.empty_like(w) for w in self.W32]
        self.gb = [torch.empty_like(b) for b in self.b32]
        self.mW = [torch.zeros_like(w) for w in self.W32]
        self.vW = [torch.zeros_like(w) for w in self.W32]
        self.mb = [torch.zeros_like(b) for b in self.b32]
        self.vb = [torch.zeros_like(b) for b in self.b32]
        self.t = 0
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self._sync()

    def _sync(self):
        for w32, w16 in zip(self.W32, self.W16):
            self.ctx.cast_bf16(w32, w16)

    def forward(self, x, y):
        self.ctx.mlp_forward(x, self.W16, self.b32, y)

    def train_step(self, x, target, K: int, lr: float, y=None, gy=None):
        N = x.shape[0]
        y = torch.empty((N, 16), dtype=torch.float32, device=x.device) if y is None else y
        gy = torch.empty_like(y) if gy is None else gy
        self.forward(x, y)
        self.ctx.mlp_mse_loss(y, target, K, self.loss, gy)
        self.ctx.mlp_backward(x, self.W16, self.b32, gy, self.gW, self.gb)
        self.t += 1
        # the eight weight and bias arrays in one launch
        self.ctx.adam_step_multi(self.W32 + self.b32, self.gW + self.gb, self.mW + self.mb, self.vW + self.vb,
                                 self.t, [lr] * (2 * len(DIMS)))
        self._sync()
        return self.loss

    def fit(self, x, target, K: int, steps: int, lr: float = 1e-3, batch: int | None = None, seed: int = 0):
        """Adam steps on (x, target); with ``batch`` each step takes a random
        window of that many consecutive rows (the rows of a scene are already
        in random order, so a window is a random sample of it)."""
        N = x.shape[0]
        B = N if batch is None or batch >= N else int(batch)
        y = torch.empty((B, 16), dtype=torch.float32, device=x.device)
        gy = torch.empty_like(y)
        rng = np.random.default_rng(seed)
        hist = []
        for s in range(steps):
            off = 0 if B == N else int(rng.integers(0, N - B + 1))
            l = self.train_step(x[off:off + B], target[off:off + B], K, lr, y, gy)
            if s % max(1, steps // 20) == 0 or s == steps - 1:
                hist.append((s, float(l.item())))
        return hist

    def apply(self, g: dict, rgb):
        """Sets g['amplitude'] and g['phase'] (in place) from the network."""
        N = g["means"].shape[0]
        x = torch.empty((N, 16), dtype=torch.int16, device=g["means"].device)
        self.ctx.init_features(g, rgb, x)
        y = torch.empty((N, 16), dtype=torch.float32, device=x.device)
        self.forward(x, y)
        self.ctx.init_apply(y, g["amplitude"], g["phase"])


# ---------------------------------------------------------------------------
# experiment: scenes optimised by the plain method -> network -> held-out scenes
# ---------------------------------------------------------------------------
def make_scene(seed: int, N: int, optics, device="cuda"):
    """Synthetic scene (hcgs_synth recipe) with an RGB colour per Gaussian."""
    import hcgs_synth as S
    g = S.make_gaussians(N, optics.L, optics.C, optics.H, optics.W, seed=seed, log_scale_mean=-3.5)
    rgb = S.random_real((N, 3), seed=10_000 + seed)
    gd = {k: torch.from_numpy(g[k]).to(device) for k in PARAM_NAMES}
    return gd, torch.from_numpy(rgb).to(device)


def colour_targets(ctx: Context, g: dict, rgb, vms, it, optics, opts=None):
    """Per-plane intensity targets: the colour blend of each plane's own
    Gaussians (Eq. gaussian_blending restricted to plane l: amplitude = RGB,
    phase 0, so the plane field is real), one focal stack per view."""
    o = optics
    gc = dict(g)
    gc["amplitude"] = rgb[:, :o.C].contiguous()
    gc["phase"] = torch.zeros_like(g["phase"])
    holo = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device=rgb.device)
    U = torch.empty((1, o.L, o.C, o.H, o.W), dtype=torch.complex64, device=rgb.device)
    out = []
    for vm in vms:
        ctx.render_view(gc, vm, it, o, opts, holo, U)
        out.append(torch.view_as_real(U)[..., 0].contiguous())
    return out


def plain_init(g: dict, rgb, seed: int, zero_phase=False):
    """Plain initialisation (Algorithm 1): amplitude = RGB, phase uniform in
    [0, 2 pi) (or 0)."""
    C = g["amplitude"].shape[1]
    g["amplitude"].copy_(rgb[:, :C])
    if zero_phase:
        g["phase"].zero_()
    else:
        gen = torch.Generator(device="cpu").manual_seed(seed)
        g["phase"].copy_((torch.rand(g["phase"].shape, generator=gen) * 2 * math.pi).to(g["phase"].device))


def optimise(ctx, g, vms, it, targets, optics, steps, lrs, opts=None, record_every=5):
    """Plain optimiser on amplitude and phase; returns [(step, PSNR)] of the
    mean focal-stack loss over the views."""
    tr = HologramTrainer(ctx, g, optics, opts, lrs=lrs)
    V = len(vms)
    curve = []
    for s in range(steps + 1):
        if s % record_every == 0 or s == steps:
            torch.cuda.synchronize()
            l = np.mean([float(tr.loss_only(vms[k], it, targets[k]).item()) for k in range(V)])
            curve.append((s, -10.0 * math.log10(max(l, 1e-30))))
        if s < steps:
            tr.step(vms[s % V], it, targets[s % V])
    tr.saved.release()
    return curve


def steps_to(curve, psnr):
    for s, p in curve:
        if p >= psnr:
            return s
    return None


def run_experiment(ctx: Context, optics, n_train=16, n_test=4, N=3000, n_views=4, opt_steps=150,
                   mlp_steps=1500, lr_app=(0.01, 0.02), seed=0, opts=None, train_init="zero", mlp_lr=1e-3,
                   mlp_batch=None, log=print):
    """Trains the network on n_train scenes optimised by the plain method
    (started from zero phase, or from random phase with train_init="random")
    and compares, on n_test held-out scenes, the plain initialisation, zero
    phase and the network's initialisation under the same optimiser budget."""
    import hcgs_synth as S
    lrs = dict(amplitude=lr_app[0], phase=lr_app[1])
    o = optics
    dev = "cuda"
    t0 = time.time()
    xs, ts = [], []
    train_final = []
    for i in range(n_train):
        g, rgb = make_scene(seed * 1000 + i, N, o)
        vm_np, it_np = S.view_batch(n_views, o.H, o.W, seed=seed * 1000 + i)
        vms = [torch.from_numpy(vm_np[k:k + 1].astype(np.float32)).to(dev) for k in range(n_views)]
        it = torch.from_numpy(it_np[:1].astype(np.float32)).to(dev)
        targets = colour_targets(ctx, g, rgb, vms, it, o, opts)
        plain_init(g, rgb, seed=i, zero_phase=(train_init == "zero"))
        curve = optimise(ctx, g, vms, it, targets, o, opt_steps, lrs, opts)
        train_final.append(curve[-1][1])
        x = torch.empty((N, 16), dtype=torch.int16, device=dev)
        ctx.init_features(g, rgb, x)
        t = torch.empty((N, 16), dtype=torch.float32, device=dev)
        ctx.init_targets(g["amplitude"], g["phase"], t)
        xs.append(x)
        ts.append(t)
    t_data = time.time() - t0
    X = torch.cat(xs).contiguous()
    T = torch.cat(ts).contiguous()
    net = InitNet(ctx, seed=seed)
    t1 = time.time()
    hist = net.fit(X, T, K=2 * o.C, steps=mlp_steps, lr=mlp_lr, batch=mlp_batch, seed=seed)
    torch.cuda.synchronize()
    t_fit = time.time() - t1
    log("network fit on %d Gaussians: loss %.4e -> %.4e (%.1f s)" % (X.shape[0], hist[0][1], hist[-1][1], t_fit))
    results = {"plain": [], "zero_phase": [], "network": []}
    times = {"plain": 0.0, "zero_phase": 0.0, "network": 0.0}
    for j in range(n_test):
        sid = seed * 1000 + 500 + j
        g0, rgb = make_scene(sid, N, o)
        vm_np, it_np = S.view_batch(n_views, o.H, o.W, seed=sid)
        vms = [torch.from_numpy(vm_np[k:k + 1].astype(np.float32)).to(dev) for k in range(n_views)]
        it = torch.from_numpy(it_np[:1].astype(np.float32)).to(dev)
        targets = colour_targets(ctx, g0, rgb, vms, it, o, opts)
        for name in results:
            g = {k: v.clone() for k, v in g0.items()}
            if name == "network":
                net.apply(g, rgb)
            else:
                plain_init(g, rgb, seed=sid, zero_phase=(name == "zero_phase"))
            torch.cuda.synchronize()
            ts0 = time.time()
            results[name].append(optimise(ctx, g, vms, it, targets, o, opt_steps, lrs, opts))
            torch.cuda.synchronize()
            times[name] += time.time() - ts0
    summary = {}
    target_psnr = float(np.mean([c[-1][1] for c in results["plain"]]))
    for name, curves in results.items():
        steps_arr = np.array([c[0] for c in curves[0]])
        mean_curve = np.mean([[p for _, p in c] for c in curves], axis=0)
        hit = [steps_to(c, target_psnr) for c in curves]
        summary[name] = {
            "psnr_step0": float(mean_curve[0]),
            "psnr_final": float(mean_curve[-1]),
            "psnr_curve": [(int(s), float(p)) for s, p in zip(steps_arr, mean_curve)],
            "steps_to_plain_final": hit,
            "seconds_optimising": times[name] / max(1, n_test),
        }
    summary["target_psnr"] = target_psnr
    summary["train_scenes_final_psnr"] = float(np.mean(train_final))
    summary["network_fit"] = {"first": hist[0][1], "last": hist[-1][1], "seconds": t_fit, "rows": int(X.shape[0]),
                              "steps": mlp_steps, "batch": mlp_batch}
    summary["data_seconds"] = t_data
    return summary


def main(argv=None):
    """Runs the experiment and prints its summary as one JSON line, e.g.
    ``python -m paper_2506_08350_b300.learned_init`` for 200 training scenes of
    100k Gaussians (256 x 256 RGB, 4 planes over 0-6 mm, 4 views per scene,
    100 optimiser steps) and 8 held-out scenes."""
    import argparse
    import json

    import hcgs_synth as S
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train-scenes", type=int, default=200)
    ap.add_argument("--test-scenes", type=int, default=8)
    ap.add_argument("--gaussians", type=int, default=100_000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--planes", type=int, default=4)
    ap.add_argument("--views", type=int, default=4)
    ap.add_argument("--opt-steps", type=int, default=100)
    ap.add_argument("--mlp-steps", type=int, default=1500)
    ap.add_argument("--mlp-batch", type=int, default=65536)
    ap.add_argument("--train-init", default="zero", choices=["zero", "random"])
    a = ap.parse_args(argv)
    z = tuple(float(v) for v in np.linspace(0.0, 6e-3, a.planes))
    o = S.Optics(a.size, a.size, S.WAVELENGTHS_RGB, z)
    ctx = Context(0)
    t = time.time()
    r = run_experiment(ctx, o, n_train=a.train_scenes, n_test=a.test_scenes, N=a.gaussians, n_views=a.views,
                       opt_steps=a.opt_steps, mlp_steps=a.mlp_steps, train_init=a.train_init,
                       mlp_batch=a.mlp_batch, log=lambda *x: None)
    r["wall_seconds"] = time.time() - t
    r["config"] = vars(a)
    for k in ("plain", "zero_phase", "network"):
        r[k].pop("psnr_curve", None)
    print(json.dumps(r))
    ctx.close()


if __name__ == "__main__":
    main()
