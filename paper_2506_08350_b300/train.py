"""Optimisation step of the complex-valued holographic Gaussians on the GPU.

One step (Algorithm 1 without densification; the optimiser is Adam as in the
training configurations): render the hologram of one view (hcgs_render_view),
inverse-propagate it to every depth plane and compare the intensities with the
focal-stack targets (hcgs_focal_stack_loss: Eq. plane2layer_asm and
Eq. recon_loss as a mean), run the adjoint (hcgs_render_view_backward) and
update every parameter array with Adam (hcgs_adam_step).  All arithmetic runs
in the library's kernels; this module only sequences the calls.

Learning rates follow Sec. 5 (means and plane logits 0.01, scales 0.005,
amplitude and phase 0.0025, opacity 0.025, rotation 0.001); a learning rate of
0 freezes an array.
"""
from __future__ import annotations

import torch

from . import PARAM_NAMES, Context, Saved

PAPER_LR = dict(means=0.01, log_scales=0.005, quats=0.001, opacity_logits=0.025, amplitude=0.0025,
                phase=0.0025, plane_logits=0.01)


class HologramTrainer:
    """Adam optimisation of the Gaussian parameters against focal stacks."""

    def __init__(self, ctx: Context, params: dict, optics, opts=None, lrs=None, betas=(0.9, 0.999), eps=1e-8,
                 data_parallel: bool = False):
        self.ctx = ctx
        self.p = params
        self.optics = optics
        self.opts = opts
        self.lrs = dict(PAPER_LR if lrs is None else lrs)
        self.betas = betas
        self.eps = eps
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.g = {k: torch.empty_like(v) for k, v in params.items()}
        self.t = 0
        self.data_parallel = data_parallel  # sum gradients over the ranks of the process group
        self.saved = Saved(ctx)
        dev = params["means"].device
        o = optics
        self.holo = torch.empty((1, len(o.wavelengths), o.H, o.W), dtype=torch.complex64, device=dev)
        self.gholo = torch.empty_like(self.holo)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def loss_only(self, viewmat, intr, I_gt):
        """Focal-stack loss of the current parameters for one view (no update)."""
        self.ctx.render_view(self.p, viewmat, intr, self.optics, self.opts, self.holo, None, self.saved)
        self.ctx.focal_stack_loss(self.holo, I_gt, 1, self.optics, self.loss, None, None)
        return self.loss

    def step(self, viewmat, intr, I_gt):
        """One optimisation step on one view; returns the loss before the update
        (a device tensor)."""
        self.ctx.render_view(self.p, viewmat, intr, self.optics, self.opts, self.holo, None, self.saved)
        self.ctx.focal_stack_loss(self.holo, I_gt, 1, self.optics, self.loss, self.gholo, None)
        self.ctx.render_view_backward(self.saved, self.p, self.gholo, self.g)
        if self.data_parallel:
            from .parallel import allreduce_gradients
            allreduce_gradients(self.g)
        self.t += 1
        for k in PARAM_NAMES:
            lr = self.lrs.get(k, 0.0)
            if lr > 0:
                self.ctx.adam_step(self.p[k], self.g[k], self.m[k], self.v[k], self.t, lr, self.betas[0],
                                   self.betas[1], self.eps)
        return self.loss


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


def ring_run(ctx: Context, optics, N: int, steps: int, n_views: int = 50, footprint: int = 0, teacher_seed: int = 3,
             student_seed: int = 0, lrs=None, device: str = "cuda"):
    """A full optimisation run on synthetic data: the focal stacks of a teacher
    scene seen from ``n_views`` cameras on a ring are the targets; the student
    has the teacher's geometry and a fresh draw of amplitude and phase
    (amplitude U[0, 1], phase U[0, 2 pi), the plain initialisation) and is
    optimised one view per step (render, inverse propagation + focal-stack
    loss, adjoint, Adam on every parameter array).  ``footprint`` selects the
    FP32 (0) or FP16x2 (1) footprint tier.

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
    peaks = [float(t.max().item()) for t in targets]
    del tdev
    student = dict(teacher)
    rng = np.random.default_rng(student_seed)
    student["amplitude"] = rng.random(teacher["amplitude"].shape).astype(np.float32)
    student["phase"] = (rng.random(teacher["phase"].shape) * 2.0 * np.pi).astype(np.float32)
    p = {k: torch.from_numpy(np.ascontiguousarray(student[k])).to(device) for k in PARAM_NAMES}
    opts = dict(DEFAULT_OPTS, footprint=int(footprint))
    tr = HologramTrainer(ctx, p, o, opts, lrs=lrs)

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
        tr.step(vms[s % n_views], it, targets[s % n_views])
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(steps, 1)
    p1 = psnr()
    tr.saved.release()
    return {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "psnr_start": p0, "psnr_end": p1, "steps": steps,
            "views": n_views, "footprint": "fp16x2" if footprint else "fp32"}
