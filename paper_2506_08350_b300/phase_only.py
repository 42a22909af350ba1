"""Phase-only hologram conversion (Sec. 6, phase-only hologram conversion
paragraph): a complex hologram P = A e^{j phi} is turned into a phase-only
one e^{j phi_opt} for a phase-only SLM by matching their propagated fields on
every depth plane (hcgs_phase_only_loss: field error over the real and
imaginary parts plus SSIM), optimised with Adam on the phase and started from
the complex hologram's own phase.  All arithmetic runs in the library's
kernels; this module only sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import SSIM_LAMBDA, Context


def convert(ctx: Context, hologram, optics, steps: int = 300, lr: float = 0.02, lambda_ssim: float = SSIM_LAMBDA,
            betas=(0.9, 0.999), init: str = "hologram", seed: int = 0):
    """hologram: device complex64 [B][C][H][W], scaled to RMS amplitude 1
    before the conversion; init "hologram" starts from its phase, "random"
    from uniform phases.  Returns (phase [B][C][H][W] float32, report) with
    the objective before and after, the focal-stack
    intensity PSNR of the phase-only hologram against the complex one (peak =
    the largest target intensity) before and after, and the time per step."""
    B = hologram.shape[0]
    o = optics
    L, C = len(o.plane_z), len(o.wavelengths)
    dev = hologram.device
    # a phase-only hologram has unit amplitude: scale the complex hologram to
    # RMS amplitude 1 first (the scale factor is read on the host)
    h = hologram.detach().cpu().numpy()
    rms = float(np.sqrt(np.mean(np.abs(h.astype(np.complex128)) ** 2)))
    hologram_s = torch.empty_like(hologram)
    ctx.scale(hologram, 1.0 / max(rms, 1e-30), hologram_s)
    hologram = hologram_s
    U = torch.empty((B, L, C, o.H, o.W), dtype=torch.complex64, device=dev)
    ctx.asm_propagate(hologram, B, o, -1, 0, U)
    phase = torch.empty((B, C, o.H, o.W), dtype=torch.float32, device=dev)
    if init == "hologram":
        ctx.hologram_phase(hologram, phase)
    else:  # uniform phases in (0, 2 pi) from the counter-based generator
        ctx.philox(seed, phase.numel(), phase, kind=2)
        ctx.scale(phase, 2.0 * math.pi, phase)
    g = torch.empty_like(phase)
    m, v = torch.zeros_like(phase), torch.zeros_like(phase)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)

    # focal-stack intensities of the complex hologram, the PSNR reference
    I_ref = torch.empty((B, L, C, o.H, o.W), dtype=torch.float32, device=dev)
    zero = torch.zeros_like(I_ref)
    ctx.focal_stack_loss(hologram, zero, B, o, loss, None, I_ref)
    peak = float(I_ref.max().item())
    ph_holo = torch.empty_like(hologram)

    def psnr():
        # e^{j phase} through the same inverse propagation, MSE against I_ref
        ctx.phase_hologram(phase, ph_holo)
        ctx.focal_stack_loss(ph_holo, I_ref, B, o, loss, None, None)
        return 10.0 * math.log10(peak ** 2 / max(float(loss.item()), 1e-300))

    def objective():
        ctx.phase_only_loss(U, phase, B, o, loss, None, lambda_ssim)
        return float(loss.item())

    l0, p0 = objective(), psnr()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for t in range(1, steps + 1):
        ctx.phase_only_loss(U, phase, B, o, loss, g, lambda_ssim)
        ctx.adam_step(phase, g, m, v, t, lr, betas[0], betas[1], 1e-8)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(steps, 1)
    l1, p1 = objective(), psnr()
    return phase, {"loss_start": l0, "loss_end": l1, "psnr_start": p0, "psnr_end": p1, "steps": steps,
                   "ms_per_step": ms}

