"""Optimisation step of the complex-valued holographic Gaussians on the GPU.

One step (Algorithm 1 without densification): render the hologram of one view
(hcgs_render_view), inverse-propagate it to every depth plane and compare the
intensities with the focal-stack targets, run the adjoint
(hcgs_render_view_backward) and update every parameter array.  Two objectives:
"mse", the plain focal-stack loss (hcgs_focal_stack_loss: Eq. plane2layer_asm
and Eq. recon_loss as a mean), and "paper", L_recon + L_SSIM with the plane
masks (hcgs_paper_loss, Sec. 4.1); two optimisers: Adam (hcgs_adam_step) and
Adan (hcgs_adan_step, the optimiser of Sec. 5), optionally with cosine
annealing of the means' and plane logits' learning rates (minimum 1e-5).
All arithmetic runs in the library's kernels; this module only sequences the
calls.

Learning rates follow Sec. 5 (means and plane logits 0.01, scales 0.005,
amplitude and phase 0.0025, opacity 0.025, rotation 0.001); a learning rate of
0 freezes an array.
"""
from __future__ import annotations

import torch

from . import DEFAULT_DENSIFY, DENSIFY_PERIOD, PARAM_NAMES, SSIM_LAMBDA, Context, Saved

PAPER_LR = dict(means=0.01, log_scales=0.005, quats=0.001, opacity_logits=0.025, amplitude=0.0025,
                phase=0.0025, plane_logits=0.01)
ANNEALED = ("means", "plane_logits")  # arrays whose learning rate follows the cosine schedule
LR_MIN = 1e-5
ADAN_BETAS = (0.9, 0.92, 0.99)  # decay factors of the first moment, the gradient difference, the second moment


def cosine_lr(step: int, total: int, lr0: float, lr_min: float = LR_MIN) -> float:
    """Cosine annealing from lr0 at step 0 to lr_min at step ``total`` (held after)."""
    import math
    t = min(max(step, 0), total)
    return lr_min + (lr0 - lr_min) * (1.0 + math.cos(math.pi * t / total)) / 2.0


class HologramTrainer:
    """Optimisation of the Gaussian parameters against focal stacks.

    objective: "mse" (plain focal-stack loss) or "paper" (L_recon + L_SSIM;
    step() then takes the view's plane masks); optimizer: "adam" or "adan";
    total_steps: if given, the learning rates of the means and plane logits
    follow cosine annealing over that many steps."""

    def __init__(self, ctx: Context, params: dict, optics, opts=None, lrs=None, betas=None, eps=1e-8,
                 data_parallel: bool = False, objective: str = "mse", optimizer: str = "adam",
                 total_steps: int | None = None, lambda_ssim: float = SSIM_LAMBDA, weight_decay: float = 0.0,
                 densify: dict | None = None, densify_every: int = DENSIFY_PERIOD, densify_until: int | None = None,
                 seed: int = 0):
        if objective not in ("mse", "paper"):
            raise ValueError("objective must be 'mse' or 'paper'")
        if optimizer not in ("adam", "adan"):
            raise ValueError("optimizer must be 'adam' or 'adan'")
        self.ctx = ctx
        self.p = params
        self.optics = optics
        self.opts = opts
        self.lrs = dict(PAPER_LR if lrs is None else lrs)
        self.objective = objective
        self.optimizer = optimizer
        self.betas = betas if betas is not None else ((0.9, 0.999) if optimizer == "adam" else ADAN_BETAS)
        self.eps = eps
        self.weight_decay = weight_decay
        self.total_steps = total_steps
        self.lambda_ssim = lambda_ssim
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.g = {k: torch.empty_like(v) for k, v in params.items()}
        if optimizer == "adan":
            self.n = {k: torch.zeros_like(v) for k, v in params.items()}
            self.g_prev = {k: torch.zeros_like(v) for k, v in params.items()}
        self.t = 0
        # densification (Algorithm 1): statistics gathered every step, applied
        # every `densify_every` steps up to `densify_until` (None: always)
        self.densify_opts = None if densify is None else {**DEFAULT_DENSIFY, **densify}
        self.densify_every = densify_every
        self.densify_until = densify_until
        self.seed = seed
        self.densify_log = []
        dev0 = params["means"].device
        N0 = params["means"].shape[0]
        self.accum = torch.zeros(N0, dtype=torch.float32, device=dev0)
        self.denom = torch.zeros(N0, dtype=torch.float32, device=dev0)
        self.data_parallel = data_parallel  # sum gradients over the ranks of the process group
        self.saved = Saved(ctx)
        dev = params["means"].device
        o = optics
        self.holo = torch.empty((1, len(o.wavelengths), o.H, o.W), dtype=torch.complex64, device=dev)
        self.gholo = torch.empty_like(self.holo)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def loss_only(self, viewmat, intr, I_gt):
        """Plain focal-stack loss of the current parameters for one view (no update)."""
        self.ctx.render_view(self.p, viewmat, intr, self.optics, self.opts, self.holo, None, self.saved)
        self.ctx.focal_stack_loss(self.holo, I_gt, 1, self.optics, self.loss, None, None)
        return self.loss

    def lr(self, k: str) -> float:
        lr0 = self.lrs.get(k, 0.0)
        if self.total_steps and k in ANNEALED and lr0 > 0:
            return cosine_lr(self.t - 1, self.total_steps, lr0)
        return lr0

    def step(self, viewmat, intr, I_gt, mask=None):
        """One optimisation step on one view; returns the loss before the update
        (a device tensor).  mask: the view's plane masks [1, L, H, W] (objective
        "paper"; None = all zero).  With data_parallel the gradients are summed
        over the ranks of the process group before the update."""
        self.gradients(viewmat, intr, I_gt, mask)
        if self.data_parallel:
            from .parallel import allreduce_gradients
            allreduce_gradients(self.g)
        self.apply_gradients()
        return self.loss

    def gradients(self, viewmat, intr, I_gt, mask=None):
        """The loss of one view and its gradients w.r.t. every parameter array
        (into ``self.g``, overwritten), and the densification statistics."""
        self.ctx.render_view(self.p, viewmat, intr, self.optics, self.opts, self.holo, None, self.saved)
        if self.objective == "paper":
            self.ctx.paper_loss(self.holo, I_gt, mask, 1, self.optics, self.loss, self.gholo, None,
                                lambda_ssim=self.lambda_ssim)
        else:
            self.ctx.focal_stack_loss(self.holo, I_gt, 1, self.optics, self.loss, self.gholo, None)
        self.ctx.render_view_backward(self.saved, self.p, self.gholo, self.g)
        if self.densify_opts is not None:
            self.ctx.densify_accumulate(self.saved, self.accum, self.denom)
        return self.loss

    def apply_gradients(self):
        """The optimiser step with the gradients in ``self.g`` (and the
        densification, when its period comes round)."""
        self.t += 1
        # every parameter array with a positive learning rate, in one launch
        ks = [k for k in PARAM_NAMES if self.lr(k) > 0]

        def sel(d):
            return [d[k] for k in ks]

        if ks and self.optimizer == "adan":
            b1, b2, b3 = self.betas
            self.ctx.adan_step_multi(sel(self.p), sel(self.g), sel(self.g_prev), sel(self.m), sel(self.v),
                                     sel(self.n), self.t, [self.lr(k) for k in ks], b1, b2, b3, self.eps,
                                     self.weight_decay)
        elif ks:
            self.ctx.adam_step_multi(sel(self.p), sel(self.g), sel(self.m), sel(self.v), self.t,
                                     [self.lr(k) for k in ks], self.betas[0], self.betas[1], self.eps)
        if (self.densify_opts is not None and self.t % self.densify_every == 0
                and (self.densify_until is None or self.t <= self.densify_until)):
            self.densify()

    # ---- checkpoint / resume ----
    STATE_KEYS = ("m", "v", "n", "g_prev")

    def state_dict(self) -> dict:
        """Everything a resumed run needs, on the host: parameters, optimiser
        state, step count, densification statistics and log, and the settings
        that shape the next steps (learning rates, schedule, recipe, seed)."""
        def host(d):
            return {k: t.detach().cpu().clone() for k, t in d.items()}
        st = {"params": host(self.p), "t": self.t, "accum": self.accum.cpu().clone(),
              "denom": self.denom.cpu().clone(), "densify_log": list(self.densify_log),
              "lrs": dict(self.lrs), "betas": tuple(self.betas), "eps": self.eps,
              "weight_decay": self.weight_decay, "objective": self.objective, "optimizer": self.optimizer,
              "total_steps": self.total_steps, "lambda_ssim": self.lambda_ssim, "seed": self.seed,
              "densify_opts": self.densify_opts, "densify_every": self.densify_every,
              "densify_until": self.densify_until}
        for k in self.STATE_KEYS:
            if hasattr(self, k):
                st[k] = host(getattr(self, k))
        return st

    def load_state_dict(self, st: dict):
        """Restore a state_dict (parameters and optimiser state are copied to
        this trainer's device; array sizes may differ after densification)."""
        dev = self.p["means"].device
        for k, t in st["params"].items():
            self.p[k] = t.to(dev).contiguous()
        for k in self.STATE_KEYS:
            if k in st:
                setattr(self, k, {a: t.to(dev).contiguous() for a, t in st[k].items()})
        self.g = {k: torch.empty_like(v) for k, v in self.p.items()}
        self.accum = st["accum"].to(dev)
        self.denom = st["denom"].to(dev)
        self.t = int(st["t"])
        self.densify_log = list(st["densify_log"])
        for k in ("lrs", "eps", "weight_decay", "objective", "optimizer", "total_steps", "lambda_ssim", "seed",
                  "densify_opts", "densify_every", "densify_until"):
            setattr(self, k, st[k])
        self.betas = tuple(st["betas"])

    def save(self, path: str):
        torch.save(self.state_dict(), path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, map_location="cpu", weights_only=False))

    def densify(self):
        """Prune, clone and split (Algorithm 1) with the gathered statistics;
        the optimiser state follows kept Gaussians and starts at zero for new
        ones; the statistics restart.  Returns (old N, new N, action counts)."""
        ctx = self.ctx
        N = self.p["means"].shape[0]
        C, L = self.p["amplitude"].shape[1], self.p["plane_logits"].shape[1]
        # quantiles of the mean statistic over the Gaussians seen (host copy, for the log)
        import numpy as np
        a_h, d_h = self.accum.cpu().numpy(), self.denom.cpu().numpy()
        seen = d_h > 0
        q = np.quantile(a_h[seen] / d_h[seen], [0.5, 0.9, 0.99]).tolist() if seen.any() else [0.0, 0.0, 0.0]
        act, off, n_new = ctx.densify_plan(self.p, self.accum, self.denom, self.densify_opts)
        dev = self.p["means"].device
        noise = torch.empty((N, 2, 3 + C), dtype=torch.float32, device=dev)
        ctx.philox(self.seed, noise.numel(), noise, kind=1, stream_id=self.t)
        newp = {k: torch.empty((n_new,) + tuple(v.shape[1:]), dtype=v.dtype, device=dev) for k, v in self.p.items()}
        states = [self.m, self.v] + ([self.n, self.g_prev] if self.optimizer == "adan" else [])
        news = [{k: torch.empty_like(newp[k]) for k in PARAM_NAMES} for _ in states]
        extras = [(st[k], ns[k]) for st, ns in zip(states, news) for k in PARAM_NAMES]
        ctx.densify_apply(self.p, C, L, act, off, noise, newp, self.densify_opts, extras)
        counts = np.bincount(act.cpu().numpy(), minlength=4).tolist() if N else [0, 0, 0, 0]
        self.p.update(newp)
        self.m, self.v = news[0], news[1]
        if self.optimizer == "adan":
            self.n, self.g_prev = news[2], news[3]
        self.g = {k: torch.empty_like(v) for k, v in self.p.items()}
        self.accum = torch.zeros(n_new, dtype=torch.float32, device=dev)
        self.denom = torch.zeros(n_new, dtype=torch.float32, device=dev)
        self.densify_log.append(dict(step=self.t, n_before=N, n_after=n_new, keep=counts[0], prune=counts[1],
                                     clone=counts[2], split=counts[3], seen=int(seen.sum()),
                                     stat_median=q[0], stat_p90=q[1], stat_p99=q[2]))
        return self.densify_log[-1]


def focal_stack(ctx: Context, params: dict, viewmat, intr, optics, opts=None):
    """Intensities I_l = |IDFT(H_{-Z_l} DFT(P))|^2 of the hologram of one view,
    shape [1, L, C, H, W] (used to make targets from a teacher scene); computed
    by the loss kernel against a zero target."""
    o = optics
    dev = params["means"].device
    holo = torch.empty((1, len(o.wavelengths), o.H, o.W), dtype=torch.complex64, device=dev)
    ctx.render_view(params, viewmat, intr, o, opts, holo)
    shape = (1, len(o.plane_z), len(o.wavelengths), o.H, o.W)
    I = torch.empty(shape, dtype=torch.float32, device=dev)
    zero = torch.zeros(shape, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ctx.focal_stack_loss(holo, zero, 1, o, loss, None, I)
    return I


def plane_masks(ctx: Context, params: dict, viewmat, intr, optics, opts=None):
    """Binary plane masks [1, L, H, W] of one view of a scene, the synthetic
    counterpart of masks cut from a target's quantised depth: a pixel belongs
    to the plane whose Gaussians cover it most (1 - T_l largest), if that
    coverage exceeds one half; otherwise to no plane.  The per-plane
    transmittances come from the library's rasterizer; the arg-max is data
    preparation on the host."""
    import numpy as np

    o = optics
    dev = params["means"].device
    saved = Saved(ctx)
    ctx.project(params, viewmat, intr, o, opts, saved)
    U = torch.empty((1, len(o.plane_z), len(o.wavelengths), o.H, o.W), dtype=torch.complex64, device=dev)
    T = torch.empty((1, len(o.plane_z), o.H, o.W), dtype=torch.float32, device=dev)
    ctx.rasterize_planes(saved, U, T)
    cov = 1.0 - T.cpu().numpy()[0]
    saved.release()
    best = np.argmax(cov, axis=0)
    keep = np.take_along_axis(cov, best[None], axis=0)[0] > 0.5
    M = np.zeros((1,) + cov.shape, dtype=np.float32)
    for l in range(cov.shape[0]):
        M[0, l] = (best == l) & keep
    return torch.from_numpy(M).to(dev)


def ring_run(ctx: Context, optics, N: int, steps: int, n_views: int = 50, footprint: int = 0, teacher_seed: int = 3,
             student_seed: int = 0, lrs=None, device: str = "cuda", objective: str = "mse",
             optimizer: str = "adam", anneal: bool = False, densify: dict | None = None):
    """A full optimisation run on synthetic data: the focal stacks of a teacher
    scene seen from ``n_views`` cameras on a ring are the targets; the student
    has the teacher's geometry and a fresh draw of amplitude and phase
    (amplitude U[0, 1], phase U[0, 2 pi), the plain initialisation) and is
    optimised one view per step (render, inverse propagation + loss, adjoint,
    optimiser step on every parameter array).  ``footprint`` selects the FP32
    (0), FP16x2 (1) or BF16x2 (2) footprint tier; ``objective``, ``optimizer`` and
    ``anneal`` (cosine schedule over ``steps``) as in HologramTrainer; with the
    "paper" objective the plane masks come from the teacher (plane_masks).

    Returns steps/s over the timed steps (CUDA events) and the PSNR over all
    views before and after, PSNR = 10 log10(peak^2 / MSE) with the view's
    largest target intensity as the peak and the focal-stack MSE of Eq.
    recon_loss (mean over planes, channels and pixels)."""
    import numpy as np

    import hcgs_synth as S
    from . import DEFAULT_OPTS, PARAM_NAMES

    o = optics
    vms_np = S.ring_cameras(n_views).astype(np.float32)
    it_np = S.intrinsics(o.H, o.W).astype(np.float32)[None]
    vms = [torch.from_numpy(vms_np[k:k + 1].copy()).to(device) for k in range(n_views)]
    it = torch.from_numpy(it_np).to(device)
    teacher = S.make_gaussians(N, o.L, o.C, o.H, o.W, seed=teacher_seed)
    tdev = {k: torch.from_numpy(teacher[k]).to(device) for k in PARAM_NAMES}
    targets = [focal_stack(ctx, tdev, vm, it, o) for vm in vms]
    masks = [plane_masks(ctx, tdev, vm, it, o, DEFAULT_OPTS) for vm in vms] if objective == "paper" else None
    peaks = [float(t.max().item()) for t in targets]
    del tdev
    student = dict(teacher)
    rng = np.random.default_rng(student_seed)
    student["amplitude"] = rng.random(teacher["amplitude"].shape).astype(np.float32)
    student["phase"] = (rng.random(teacher["phase"].shape) * 2.0 * np.pi).astype(np.float32)
    p = {k: torch.from_numpy(np.ascontiguousarray(student[k])).to(device) for k in PARAM_NAMES}
    opts = dict(DEFAULT_OPTS, footprint=int(footprint))
    tr = HologramTrainer(ctx, p, o, opts, lrs=lrs, objective=objective, optimizer=optimizer,
                         total_steps=steps if anneal else None, densify=densify)

    def psnr():
        vals = []
        for k in range(n_views):
            mse = float(tr.loss_only(vms[k], it, targets[k]).item())
            vals.append(10.0 * np.log10(peaks[k] ** 2 / max(mse, 1e-300)))
        return float(np.mean(vals))

    p0 = psnr()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for s in range(steps):
        k = s % n_views
        tr.step(vms[k], it, targets[k], masks[k] if masks else None)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(steps, 1)
    p1 = psnr()
    tr.saved.release()
    out = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "psnr_start": p0, "psnr_end": p1, "steps": steps,
           "views": n_views, "footprint": ("fp32", "fp16x2", "bf16x2")[int(footprint)], "objective": objective,
           "optimizer": optimizer, "anneal": bool(anneal)}
    if densify is not None:
        out["densify"] = tr.densify_log
        out["N_end"] = int(tr.p["means"].shape[0])
    return out
