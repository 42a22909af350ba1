"""FP64 CPU oracle for the complex-valued holographic Gaussian renderer.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2506_08350_b300``) and never imports it.

What each function follows (arXiv 2506.08350):

* ``project``            Sec. 3 (Eq. gaussian_density, gaussian_decompose,
                         gaussian_projection, gaussian_projection_2d) and the
                         plane argmax of Eq. hard_assignment;
* ``composite``          the per-plane complex field of Sec. 4.1 and
                         Algorithm 2 (per-pixel walk in depth order);
* ``transfer_function``  Eq. band_limited_asm_transfer_function;
* ``propagate_planes``   Eq. layer2plane_asm and Eq. sum_planes (the plane sum
                         is taken literally, after each inverse transform);
* ``inverse_propagate``  Eq. plane2layer_asm, intensity I_l = |U|^2;
* ``focal_stack_loss``   Eq. recon_loss (mean over planes, channels, pixels);
* ``render_backward``    Supp. D.4, re-derived in reverse mode (C code);
* ``adam_step``          Adam (the optimiser of the plain training step);
* ``paper_loss``         the paper's training loss L_recon + L_SSIM (masked
                         reconstruction loss and structural similarity);
* ``adan_step``, ``cosine_lr``  the paper's optimiser and learning-rate schedule;
* ``phase_only_loss``    the phase-only hologram conversion objective (Sec. 6,
                         phase-only hologram conversion paragraph);
* ``philox4x32_10``, ``philox_normals``  the counter-based generator that
                         draws the densification noise (Salmon et al. 2011)
                         and standard normals from it by Box-Muller;
                         ``philox_uniforms``' half-word offset (w + 1/2) 2^-32
                         is a convention: parity unpinned;
* ``densify_accumulate``, ``densify``  Algorithm 1's pruning and phase-aware
                         clone / split (the 3DGS densification rules);
* ``mlp_*``              the learned-initialisation network (no counterpart in
                         the paper): plain float64 matrix products.

The FFT is numpy's (a library primitive); everything else is plain loops in
``hcgs_oracle.c`` or direct numpy expressions of the equations.

Pins (closed forms, invariants, brute force) live in ``tests/test_oracle_*.py``.
The paper prints no numeric worked example, so agreement with numbers the paper
prints is "parity unpinned"; every pin comes from mathematics instead.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hcgs_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_OPTS = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, T_eps=1e-4, dilation=0.3,
                    near_z=0.2, clip=1.3, order=0, tau=1e-3)
# "exact" preset: no thresholds, no dilation, no clamp; support = whole grid.
EXACT_OPTS = dict(alpha_min=0.0, alpha_max=1.0, T_eps=0.0, dilation=0.0,
                  near_z=0.2, clip=0.0, order=0, tau=1e-3)


def build() -> str:
    """Compile the C part of the oracle (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.POINTER(ctypes.c_int)
            I = ctypes.c_int
            lib.oracle_project.argtypes = [I, I, I, I, I] + [d] * 7 + [d, d, d] + [d, d, d, d, d, i, d, d, i]
            lib.oracle_project.restype = None
            lib.oracle_composite.argtypes = [I] * 5 + [d, d, d, d, i, d, d, i, d, I, I, d, d, i]
            lib.oracle_composite.restype = None
            lib.oracle_composite_backward.argtypes = [I] * 5 + [d, d, d, d, i, d, d, i, d, I, I, d, d, d, d, d]
            lib.oracle_composite_backward.restype = None
            lib.oracle_project_backward.argtypes = [I] * 5 + [d] * 7 + [d, d, d] + [d, d, d, d] + [d] * 7
            lib.oracle_project_backward.restype = None
            lib.oracle_sort.argtypes = [I, d, i, I, i]
            lib.oracle_sort.restype = I
            lib.oracle_composite_soft.argtypes = [I] * 5 + [d, d, d, d, d, d, d, i, d, d, d]
            lib.oracle_composite_soft.restype = None
            lib.oracle_composite_rho_dense.argtypes = [I] * 5 + [d, d, d, d, i, d, d, i, d, d, d]
            lib.oracle_composite_rho_dense.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _opt_vec(opts):
    o = dict(DEFAULT_OPTS)
    o.update(opts or {})
    return np.array([o["alpha_min"], o["alpha_max"], o["T_eps"], o["dilation"], o["near_z"],
                     o["clip"], float(o["order"]), o["tau"]], dtype=np.float64)


PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "amplitude", "phase", "plane_logits")


def _params64(g):
    return {k: _f64(g[k]) for k in PARAM_NAMES}


# ----------------------------------------------------------------------------
# projection and compositing (C, FP64)
# ----------------------------------------------------------------------------
def project(gauss: dict, viewmat, intr, H: int, W: int, opts=None) -> dict:
    """Per-Gaussian screen-space quantities for one view (Sec. 3, Eq.
    gaussian_projection / gaussian_projection_2d; Eq. hard_assignment)."""
    p = _params64(gauss)
    N = p["means"].shape[0]
    L = p["plane_logits"].shape[1]
    C = p["amplitude"].shape[1]
    out = dict(mu=np.zeros((N, 2)), conic=np.zeros((N, 3)), cov=np.zeros((N, 3)), opac=np.zeros(N),
               depth=np.zeros(N), plane=np.zeros(N, dtype=np.int32), w=np.zeros((N, C, 2)),
               bbox=np.zeros((N, 4)), valid=np.zeros(N, dtype=np.int32))
    vm, it, ov = _f64(viewmat).reshape(16), _f64(intr).reshape(4), _opt_vec(opts)
    _L().oracle_project(N, L, C, H, W, *[_dp(p[k]) for k in PARAM_NAMES], _dp(vm), _dp(it), _dp(ov),
                        _dp(out["mu"]), _dp(out["conic"]), _dp(out["cov"]), _dp(out["opac"]),
                        _dp(out["depth"]), _ip(out["plane"]), _dp(out["w"]), _dp(out["bbox"]),
                        _ip(out["valid"]))
    out.update(N=N, L=L, C=C, H=H, W=W)
    return out


def visiting_order(proj: dict, order: int = 0) -> np.ndarray:
    N = proj["N"]
    out = np.zeros(N, dtype=np.int32)
    m = _L().oracle_sort(N, _dp(proj["depth"]), _ip(proj["valid"]), int(order), _ip(out))
    return out[:m]


def composite(proj: dict, opts=None, rows=None):
    """Complex per-plane fields U[L][C][H][W] (complex128), final
    transmittance T[L][H][W] and contributor counts for one view."""
    N, L, C, H, W = (proj[k] for k in ("N", "L", "C", "H", "W"))
    r0, r1 = (0, H) if rows is None else rows
    U = np.zeros((L, C, H, W, 2))
    T = np.ones((L, H, W))
    nc = np.zeros((L, H, W), dtype=np.int32)
    ov = _opt_vec(opts)
    _L().oracle_composite(N, L, C, H, W, _dp(proj["mu"]), _dp(proj["conic"]), _dp(proj["opac"]),
                          _dp(proj["depth"]), _ip(proj["plane"]), _dp(proj["w"]), _dp(proj["bbox"]),
                          _ip(proj["valid"]), _dp(ov), int(r0), int(r1), _dp(U), _dp(T), _ip(nc))
    return U[..., 0] + 1j * U[..., 1], T, nc


def composite_backward(proj: dict, gU, opts=None, rows=None):
    """Adjoint of ``composite``: per-Gaussian gradients w.r.t. mu, conic
    (A, B, C), the activated opacity and w (= c e^{j phi}, as Re/Im).
    ``rows`` = (row0, row1) restricts the sum to a band of image rows."""
    N, L, C, H, W = (proj[k] for k in ("N", "L", "C", "H", "W"))
    r0, r1 = (0, H) if rows is None else rows
    g = np.ascontiguousarray(np.stack([np.real(gU), np.imag(gU)], axis=-1), dtype=np.float64)
    out = dict(mu=np.zeros((N, 2)), conic=np.zeros((N, 3)), opac=np.zeros(N), w=np.zeros((N, C, 2)))
    ov = _opt_vec(opts)
    _L().oracle_composite_backward(N, L, C, H, W, _dp(proj["mu"]), _dp(proj["conic"]), _dp(proj["opac"]),
                                   _dp(proj["depth"]), _ip(proj["plane"]), _dp(proj["w"]), _dp(proj["bbox"]),
                                   _ip(proj["valid"]), _dp(ov), int(r0), int(r1), _dp(g),
                                   _dp(out["mu"]), _dp(out["conic"]), _dp(out["opac"]), _dp(out["w"]))
    return out


def composite_soft(proj: dict, rho, opts=None):
    """Compositing with continuous plane weights rho[N][L] (alpha_eff = alpha
    rho_l, every Gaussian visited on every plane): the smooth extension of
    ``composite`` that defines the dense plane-weight gradient; equal to
    ``composite`` at the one-hot rho of the argmax planes."""
    N, L, C, H, W = (proj[k] for k in ("N", "L", "C", "H", "W"))
    U = np.zeros((L, C, H, W, 2))
    T = np.ones((L, H, W))
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(N, L)
    _L().oracle_composite_soft(N, L, C, H, W, _dp(proj["mu"]), _dp(proj["conic"]), _dp(proj["opac"]),
                               _dp(proj["depth"]), _dp(r), _dp(proj["w"]), _dp(proj["bbox"]), _ip(proj["valid"]),
                               _dp(_opt_vec(opts)), _dp(U), _dp(T))
    return U[..., 0] + 1j * U[..., 1], T


def composite_rho_dense(proj: dict, gU, opts=None) -> np.ndarray:
    """dL/drho_{n,l} [N][L] of ``composite_soft`` at the one-hot rho, for the
    planes each Gaussian is not assigned to (zero at the assigned plane, whose
    value is o dL/do of ``composite_backward``)."""
    N, L, C, H, W = (proj[k] for k in ("N", "L", "C", "H", "W"))
    g = np.ascontiguousarray(np.stack([np.real(gU), np.imag(gU)], axis=-1), dtype=np.float64)
    out = np.zeros((N, L))
    _L().oracle_composite_rho_dense(N, L, C, H, W, _dp(proj["mu"]), _dp(proj["conic"]), _dp(proj["opac"]),
                                    _dp(proj["depth"]), _ip(proj["plane"]), _dp(proj["w"]), _dp(proj["bbox"]),
                                    _ip(proj["valid"]), _dp(_opt_vec(opts)), _dp(g), _dp(out))
    return out


def ste_softmax(plane_logits, tau: float) -> np.ndarray:
    """softmax(rho'/tau) per Gaussian, max-subtracted (Eq. ste's backward weights)."""
    r = np.asarray(plane_logits, dtype=np.float64)
    e = np.exp((r - r.max(axis=1, keepdims=True)) / tau)
    return e / e.sum(axis=1, keepdims=True)


def project_backward(gauss: dict, viewmat, intr, H, W, g2d: dict, opts=None, acc=None) -> dict:
    """Adjoint of ``project`` (plus the straight-through plane-logit rule of
    Eq. ste), accumulated into ``acc`` (float64 arrays keyed like the params)."""
    p = _params64(gauss)
    N = p["means"].shape[0]
    L = p["plane_logits"].shape[1]
    C = p["amplitude"].shape[1]
    if acc is None:
        acc = {k: np.zeros_like(p[k]) for k in PARAM_NAMES}
    vm, it, ov = _f64(viewmat).reshape(16), _f64(intr).reshape(4), _opt_vec(opts)
    _L().oracle_project_backward(N, L, C, H, W, *[_dp(p[k]) for k in PARAM_NAMES], _dp(vm), _dp(it), _dp(ov),
                                 _dp(g2d["mu"]), _dp(g2d["conic"]), _dp(g2d["opac"]), _dp(g2d["w"]),
                                 *[_dp(acc[k]) for k in PARAM_NAMES])
    return acc


# ----------------------------------------------------------------------------
# band-limited angular spectrum method (numpy FFT, FP64)
# ----------------------------------------------------------------------------
def frequencies(n: int, pitch: float) -> np.ndarray:
    """Spatial frequencies of DFT bins in FFT order: k/(n pitch) for
    k = 0..ceil(n/2)-1, then -floor(n/2)..-1."""
    k = np.arange(n)
    k = np.where(k < (n + 1) // 2, k, k - n)
    return k / (n * pitch)


def transfer_function(H: int, W: int, pitch: float, wavelength: float, z: float, band_limit: int = 0) -> np.ndarray:
    """H_z(f_x, f_y) of Eq. band_limited_asm_transfer_function on the H x W
    grid in FFT order: exp(j 2 pi z sqrt(1/lambda^2 - f^2)) inside
    f^2 <= 1/lambda^2, zero outside.  With band_limit = 1 the band limit of
    Matsushima and Shimobaba (the reference the paper gives for the
    band-limited method) is applied as well: on a grid of n samples the
    frequency spacing is du = 1/(n pitch), and H is kept only where
    |f_x| <= 1/(lambda sqrt((2 du_x z)^2 + 1)) and likewise for f_y."""
    fx = frequencies(W, pitch)[None, :]
    fy = frequencies(H, pitch)[:, None]
    arg = 1.0 / wavelength ** 2 - (fx ** 2 + fy ** 2)
    inside = arg >= 0
    if band_limit:
        dux, duy = 1.0 / (W * pitch), 1.0 / (H * pitch)
        lim_x = 1.0 / (wavelength * np.sqrt((2.0 * dux * z) ** 2 + 1.0))
        lim_y = 1.0 / (wavelength * np.sqrt((2.0 * duy * z) ** 2 + 1.0))
        inside = inside & (np.abs(fx) <= lim_x) & (np.abs(fy) <= lim_y)
    phase = 2.0 * np.pi * z * np.sqrt(np.where(inside, arg, 0.0))
    return np.where(inside, np.exp(1j * phase), 0.0)


def zero_pad(u: np.ndarray) -> np.ndarray:
    """Embed the last two axes (H, W) in a 2H x 2W grid of zeros, the field
    at rows H//2 .. H//2 + H - 1 and columns W//2 .. W//2 + W - 1."""
    H, W = u.shape[-2], u.shape[-1]
    out = np.zeros(u.shape[:-2] + (2 * H, 2 * W), dtype=np.complex128)
    out[..., H // 2:H // 2 + H, W // 2:W // 2 + W] = u
    return out


def crop(u: np.ndarray, H: int, W: int) -> np.ndarray:
    """The H x W window of a 2H x 2W grid that ``zero_pad`` filled."""
    return u[..., H // 2:H // 2 + H, W // 2:W // 2 + W]


def propagate(u: np.ndarray, pitch: float, wavelength: float, z: float, band_limit: int = 0,
              padding: int = 0) -> np.ndarray:
    """One field through Eq. layer2plane_asm: IDFT(H_z DFT(u)).  padding = 1:
    on the 2x zero-padded grid (a linear instead of a circular convolution;
    H_z and its band limit then use that grid's frequencies), cropped back."""
    if padding:
        H, W = u.shape[-2], u.shape[-1]
        return crop(propagate(zero_pad(u), pitch, wavelength, z, band_limit), H, W)
    Hz = transfer_function(u.shape[-2], u.shape[-1], pitch, wavelength, z, band_limit)
    return np.fft.ifft2(Hz * np.fft.fft2(u))


def propagate_planes(U: np.ndarray, pitch: float, wavelengths, plane_z, band_limit: int = 0,
                     padding: int = 0) -> np.ndarray:
    """Eq. layer2plane_asm for every plane, then Eq. sum_planes.
    U[L][C][H][W] -> P[C][H][W]."""
    L, C = U.shape[0], U.shape[1]
    P = np.zeros(U.shape[1:], dtype=np.complex128)
    for c in range(C):
        for l in range(L):
            P[c] += propagate(U[l, c], pitch, wavelengths[c], plane_z[l], band_limit, padding)
    return P


def propagate_planes_adjoint(gP: np.ndarray, pitch: float, wavelengths, plane_z, band_limit: int = 0,
                             padding: int = 0) -> np.ndarray:
    """Adjoint of ``propagate_planes`` for g = dL/dRe + j dL/dIm:
    gU_l = IDFT(conj(H_{Z_l}) DFT(gP)).  (With F the unnormalised DFT,
    (F^-1 D F)^H = F^-1 conj(D) F; with padding the adjoint of the zero
    embedding is the crop and vice versa.)"""
    C, H, W = gP.shape
    L = len(plane_z)
    gU = np.zeros((L, C, H, W), dtype=np.complex128)
    for c in range(C):
        g = zero_pad(gP[c]) if padding else gP[c]
        G = np.fft.fft2(g)
        for l in range(L):
            Hz = transfer_function(g.shape[0], g.shape[1], pitch, wavelengths[c], plane_z[l], band_limit)
            r = np.fft.ifft2(np.conj(Hz) * G)
            gU[l, c] = crop(r, H, W) if padding else r
    return gU


def inverse_propagate(P: np.ndarray, pitch: float, wavelengths, plane_z, band_limit: int = 0,
                      padding: int = 0) -> np.ndarray:
    """Eq. plane2layer_asm: V_l = IDFT(H_{-Z_l} DFT(P)), P[C][H][W] -> V[L][C][H][W]."""
    C, H, W = P.shape
    L = len(plane_z)
    V = np.zeros((L, C, H, W), dtype=np.complex128)
    for c in range(C):
        for l in range(L):
            V[l, c] = propagate(P[c], pitch, wavelengths[c], -plane_z[l], band_limit, padding)
    return V


def inverse_propagate_adjoint(gV: np.ndarray, pitch: float, wavelengths, plane_z, band_limit: int = 0,
                              padding: int = 0) -> np.ndarray:
    """Adjoint of ``inverse_propagate``: gP = sum_l IDFT(conj(H_{-Z_l}) DFT(gV_l))
    (through the zero embedding and crop when padding = 1)."""
    L, C, H, W = gV.shape
    gP = np.zeros((C, H, W), dtype=np.complex128)
    for c in range(C):
        for l in range(L):
            g = zero_pad(gV[l, c]) if padding else gV[l, c]
            Hm = transfer_function(g.shape[0], g.shape[1], pitch, wavelengths[c], -plane_z[l], band_limit)
            r = np.fft.ifft2(np.conj(Hm) * np.fft.fft2(g))
            gP[c] += crop(r, H, W) if padding else r
    return gP


def focal_stack_loss(P: np.ndarray, I_gt: np.ndarray, pitch: float, wavelengths, plane_z, band_limit: int = 0,
                     padding: int = 0):
    """Eq. recon_loss with the mean taken over planes, channels and pixels:
    returns (loss, dL/dP as g = dL/dRe + j dL/dIm, intensities I[L][C][H][W])."""
    V = inverse_propagate(P, pitch, wavelengths, plane_z, band_limit, padding)
    I = np.abs(V) ** 2
    n = I.size
    loss = float(np.mean((I - I_gt) ** 2))
    gV = (4.0 / n) * (I - I_gt) * V
    return loss, inverse_propagate_adjoint(gV, pitch, wavelengths, plane_z, band_limit, padding), I


# ----------------------------------------------------------------------------
# the paper's training objective (Sec. 4.1 loss paragraph): L = L_recon + L_SSIM
# ----------------------------------------------------------------------------
SSIM_SIZE = 11          # Gaussian window, standard deviation 1.5 (structural similarity of Wang et al.)
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2     # stabilising constants for a data range of 1
SSIM_C2 = 0.03 ** 2
SSIM_LAMBDA = 0.005     # lambda_1 of L_SSIM


def ssim_window(size: int = SSIM_SIZE, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """The 1D factor of the separable, normalised Gaussian window."""
    x = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-(x * x) / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(a: np.ndarray) -> np.ndarray:
    """Local mean under the window at every pixel of the last two axes, the
    image continued by zeros (a 'same'-size correlation; the window is
    symmetric, so this operator is its own adjoint)."""
    from scipy.ndimage import correlate1d
    g = ssim_window()
    a = correlate1d(np.asarray(a, dtype=np.float64), g, axis=-1, mode="constant", cval=0.0)
    return correlate1d(a, g, axis=-2, mode="constant", cval=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of images x, y (last two axes):
    ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sxx + syy + C2)) with
    local means m, variances s and covariance under the window."""
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def ssim(x: np.ndarray, y: np.ndarray) -> float:
    """Mean SSIM over the pixels of one image pair."""
    return float(np.mean(ssim_map(x, y)))


def ssim_grad(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d mean(SSIM(x, y)) / dx.  With a = 2 mx my + C1, b = 2 sxy + C2,
    c = mx^2 + my^2 + C1, d = sxx + syy + C2 and S = ab/(cd) at every pixel:
    dS/dmx = 2 my (b - a)/(cd) - 2 mx S/c + 2 mx S/d (through mx, sxx and sxy),
    dS/d<x^2> = -S/d, dS/d<xy> = 2a/(cd); the gradient is the adjoint of the
    local means applied to these, G(dS/dmx) + 2x G(dS/d<x^2>) + y G(dS/d<xy>),
    divided by the pixel count."""
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    a = 2 * mx * my + SSIM_C1
    b = 2 * sxy + SSIM_C2
    c = mx * mx + my * my + SSIM_C1
    d = sxx + syy + SSIM_C2
    S = a * b / (c * d)
    d_m = 2 * my * (b - a) / (c * d) - 2 * mx * S / c + 2 * mx * S / d
    d_xx = -S / d
    d_xy = 2 * a / (c * d)
    n = x.shape[-1] * x.shape[-2]
    return (_blur(d_m) + 2 * x * _blur(d_xx) + y * _blur(d_xy)) / n


def paper_loss_intensities(I: np.ndarray, I_gt: np.ndarray, M: np.ndarray, lam: float = SSIM_LAMBDA):
    """L = L_recon + L_SSIM on focal-stack intensities I, I_gt [L][C][H][W]
    with binary plane masks M [L][H][W]:
      L_recon = mean over (l, c, pixels) of d^2 + (M d)^2 + (I_gt d)^2 =
                mean of d^2 (1 + M + I_gt^2), d = I - I_gt;
      L_SSIM  = lambda_1 mean over (l, c) of (1 - SSIM(I_lc, I_gt,lc)).
    Returns (loss, dL/dI)."""
    I = np.asarray(I, dtype=np.float64)
    I_gt = np.asarray(I_gt, dtype=np.float64)
    L, C = I.shape[0], I.shape[1]
    w = 1.0 + np.asarray(M, dtype=np.float64)[:, None] + I_gt * I_gt
    dlt = I - I_gt
    n = I.size
    loss = float(np.sum(dlt * dlt * w) / n)
    g = 2.0 * dlt * w / n
    s_sum = 0.0
    for l in range(L):
        for c in range(C):
            s_sum += ssim(I[l, c], I_gt[l, c])
            g[l, c] -= lam / (L * C) * ssim_grad(I[l, c], I_gt[l, c])
    loss += lam * (1.0 - s_sum / (L * C))
    return loss, g


def paper_loss(P: np.ndarray, I_gt: np.ndarray, M: np.ndarray, pitch: float, wavelengths, plane_z,
               lam: float = SSIM_LAMBDA, band_limit: int = 0, padding: int = 0):
    """The paper's training loss for one view's hologram P [C][H][W]: the
    focal stack I_l = |V_l|^2 of Eq. plane2layer_asm against I_gt, with
    L_recon + L_SSIM.  Returns (loss, dL/dP as g = dL/dRe + j dL/dIm, I)."""
    V = inverse_propagate(P, pitch, wavelengths, plane_z, band_limit, padding)
    I = np.abs(V) ** 2
    loss, gI = paper_loss_intensities(I, I_gt, M, lam)
    gV = 2.0 * gI * V
    return loss, inverse_propagate_adjoint(gV, pitch, wavelengths, plane_z, band_limit, padding), I


def phase_only_loss(U: np.ndarray, phase: np.ndarray, pitch: float, wavelengths, plane_z,
                    lam: float = SSIM_LAMBDA, band_limit: int = 0, padding: int = 0):
    """Objective of the phase-only conversion for one hologram: the target
    fields U[L][C][H][W] (the complex hologram propagated to the planes) against
    U_phi,l = IDFT(H_{-Z_l} DFT(e^{j phase})), phase[C][H][W]:
      L = mean over (l, c, part, pixel) of d^2 + lambda mean over (l, c, part)
          of (1 - SSIM), part = real and imaginary components, d = part(U_phi) - part(U).
    Returns (loss, dL/dphase)."""
    Pphi = np.exp(1j * np.asarray(phase, dtype=np.float64))
    Uphi = inverse_propagate(Pphi, pitch, wavelengths, plane_z, band_limit, padding)
    U = np.asarray(U, dtype=np.complex128)
    # the two parts as 2 L C real images, part-major
    X = np.stack([Uphi.real, Uphi.imag])
    Y = np.stack([U.real, U.imag])
    n = X.size
    d = X - Y
    loss = float(np.sum(d * d) / n)
    g = 2.0 * d / n
    K, L, C = X.shape[0], X.shape[1], X.shape[2]
    s_sum = 0.0
    for k in range(K):
        for l in range(L):
            for c in range(C):
                s_sum += ssim(X[k, l, c], Y[k, l, c])
                g[k, l, c] -= lam / (K * L * C) * ssim_grad(X[k, l, c], Y[k, l, c])
    loss += lam * (1.0 - s_sum / (K * L * C))
    gU = g[0] + 1j * g[1]
    gP = inverse_propagate_adjoint(gU, pitch, wavelengths, plane_z, band_limit, padding)
    # P = e^{j phase}: dL/dphase = gRe (-sin) + gIm cos = Im(conj(P) g)
    return loss, np.imag(np.conj(Pphi) * gP)


def adan_step(p, g, g_prev, m, v, n, step: int, lr: float, beta1=0.9, beta2=0.92, beta3=0.99, eps=1e-8,
              weight_decay=0.0):
    """One step of Adan (Xie et al., Algorithm 1), written with decay factors
    (beta = 1 - the algorithm's small momentum coefficients): at the first step
    m = g, v = 0, n = g^2; at the second v = g - g_prev; afterwards
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2)(g - g_prev),
    n <- b3 n + (1 - b3)(g + b2 (g - g_prev))^2 (m and n also at the second
    step); then p <- (p - lr (m + b2 v) / (sqrt(n) + eps)) / (1 + weight_decay lr).
    Returns new (p, m, v, n)."""
    p, g, m, v, n = (np.asarray(x, dtype=np.float64) for x in (p, g, m, v, n))
    if step == 1:
        m, v, n = g.copy(), np.zeros_like(g), g * g
    else:
        dg = g - np.asarray(g_prev, dtype=np.float64)
        m = beta1 * m + (1 - beta1) * g
        v = dg if step == 2 else beta2 * v + (1 - beta2) * dg
        u = g + beta2 * dg
        n = beta3 * n + (1 - beta3) * u * u
    p = (p - lr * (m + beta2 * v) / (np.sqrt(n) + eps)) / (1.0 + weight_decay * lr)
    return p, m, v, n


def cosine_lr(step: int, total: int, lr0: float, lr_min: float) -> float:
    """Cosine annealing from lr0 at step 0 to lr_min at step ``total``:
    lr_min + (lr0 - lr_min)(1 + cos(pi step / total)) / 2."""
    import math
    t = min(max(step, 0), total)
    return lr_min + (lr0 - lr_min) * (1.0 + math.cos(math.pi * t / total)) / 2.0


# ----------------------------------------------------------------------------
# densification (Algorithm 1) and its counter-based noise
# ----------------------------------------------------------------------------
PHILOX_M = (0xD2511F53, 0xCD9E8D57)   # round multipliers of Philox4x32
PHILOX_W = (0x9E3779B9, 0xBB67AE85)   # Weyl key increments


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): ctr
    [..., 4] and key [..., 2] uint32 -> [..., 4] uint32.  Each round multiplies
    words 0 and 2 by the two constants (64-bit products split into high and low
    halves), permutes and mixes in the key; the key is bumped by the Weyl
    increments between rounds."""
    c = np.array(ctr, dtype=np.uint64) & 0xFFFFFFFF
    k = np.array(key, dtype=np.uint64) & 0xFFFFFFFF
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W[0])) & mask
            k1 = (k1 + np.uint64(PHILOX_W[1])) & mask
        p0 = c0 * np.uint64(PHILOX_M[0])
        p1 = c2 * np.uint64(PHILOX_M[1])
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def philox_words(seed: int, n_words: int, stream: int = 0) -> np.ndarray:
    """n_words uint32 of the stream (seed, stream): block b is
    Philox(counter = (b, stream, 0, 0), key = (seed low, seed high))."""
    nb = (n_words + 3) // 4
    ctr = np.zeros((nb, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nb, dtype=np.uint64)
    ctr[:, 1] = stream & 0xFFFFFFFF
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    return philox4x32_10(ctr, np.broadcast_to(key, (nb, 2))).reshape(-1)[:n_words]


def philox_normals(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n standard normals (float64) from the words of ``philox_words``: each
    word pair (a, b) gives u = (a + 1/2) 2^-32, v = (b + 1/2) 2^-32 and, by
    Box-Muller, sqrt(-2 ln u) (cos 2 pi v, sin 2 pi v)."""
    m = (n + 1) // 2
    w = uniform_of_words(philox_words(seed, 2 * m, stream)).reshape(m, 2)
    u, v = w[:, 0], w[:, 1]
    r = np.sqrt(-2.0 * np.log(u))
    z = np.stack([r * np.cos(2 * np.pi * v), r * np.sin(2 * np.pi * v)], axis=1).reshape(-1)
    return z[:n]


def uniform_of_words(w) -> np.ndarray:
    """The map from 32-bit words to uniforms: u = (w + 1/2) 2^-32, the centre
    of the word's cell of width 2^-32 in [0, 1), so that u lies in the open
    interval (0, 1) (ln u stays finite in Box-Muller) and the map is symmetric
    about 1/2: u(w) + u(2^32 - 1 - w) = 1.  Exact in float64 (33 bits)."""
    return (np.asarray(w, dtype=np.uint32).astype(np.float64) + 0.5) * 2.0 ** -32


def philox_uniforms(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n uniforms in (0, 1) from the words of ``philox_words`` (``uniform_of_words``)."""
    return uniform_of_words(philox_words(seed, n, stream))


DENSIFY_OPTS = dict(grad_threshold=2e-4, split_scale=0.02, prune_opacity=5e-3, prune_scale=0.0,
                    split_shrink=1.6, phase_noise=0.1)
KEEP, PRUNE, CLONE, SPLIT = 0, 1, 2, 3


def densify_accumulate(accum, denom, valid, gmu, H: int, W: int):
    """Add one view's screen-space mean gradients to the densification
    statistics: for every visible Gaussian, accum += |(dL/dmu_x W/2,
    dL/dmu_y H/2)| (the gradient w.r.t. the mean in normalised device
    coordinates) and denom += 1.  In FP32, as the statistic is stored."""
    accum = np.asarray(accum, dtype=np.float32).copy()
    denom = np.asarray(denom, dtype=np.float32).copy()
    vis = np.asarray(valid) != 0
    g = np.asarray(gmu, dtype=np.float64)
    nrm = np.sqrt((g[:, 0] * (W / 2.0)) ** 2 + (g[:, 1] * (H / 2.0)) ** 2)
    accum[vis] += nrm[vis].astype(np.float32)
    denom[vis] += np.float32(1.0)
    return accum, denom


def densify_actions(gauss: dict, accum, denom, opts=None) -> np.ndarray:
    """Per-Gaussian decision of Algorithm 1's densification step, taken in
    FP32 (the precision the statistics are stored in): prune if the opacity
    sigmoid(logit) < prune_opacity or the largest scale exceeds prune_scale
    (when > 0); otherwise, if the mean screen-space gradient accum / denom
    reaches grad_threshold, split when the largest scale exceeds split_scale
    and clone otherwise; else keep."""
    o = {**DENSIFY_OPTS, **(opts or {})}
    f = np.float32
    logit = np.asarray(gauss["opacity_logits"], dtype=f)
    opac = f(1.0) / (f(1.0) + np.exp(-logit))
    smax = np.exp(np.max(np.asarray(gauss["log_scales"], dtype=f), axis=1))
    accum, denom = np.asarray(accum, dtype=f), np.asarray(denom, dtype=f)
    avg = np.where(denom > 0, accum / np.where(denom > 0, denom, f(1.0)), f(0.0))
    prune = opac < f(o["prune_opacity"])
    if o["prune_scale"] > 0:
        prune |= smax > f(o["prune_scale"])
    dens = avg >= f(o["grad_threshold"])
    act = np.full(len(logit), KEEP, dtype=np.int32)
    act[dens & (smax <= f(o["split_scale"]))] = CLONE
    act[dens & (smax > f(o["split_scale"]))] = SPLIT
    act[prune] = PRUNE
    return act


def _rotation(q):
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(gauss: dict, accum, denom, noise, opts=None, extra=()):
    """Algorithm 1's pruning and densification with phase-aware copies.
    Outputs follow the input order: a kept Gaussian once; a clone as the
    original followed by a copy whose phases are perturbed by
    phase_noise * noise[n, 0, 3:]; a split as two children k = 0, 1 with means
    mu + R diag(s) noise[n, k, :3] (a draw from the Gaussian itself), log-scales
    lowered by log(split_shrink), phases perturbed by phase_noise *
    noise[n, k, 3:] and everything else copied; a pruned Gaussian not at all.
    ``noise`` is [N][2][3 + C] standard normals.  ``extra`` arrays (per-Gaussian
    optimiser state) follow kept Gaussians and clone originals, and start at
    zero for copies and children.  Returns (new params, new extras, actions)."""
    o = {**DENSIFY_OPTS, **(opts or {})}
    act = densify_actions(gauss, accum, denom, o)
    p = {k: np.asarray(v, dtype=np.float64) for k, v in gauss.items()}
    C = p["amplitude"].shape[1]
    z = np.asarray(noise, dtype=np.float64).reshape(len(act), 2, 3 + C)
    out = {k: [] for k in p}
    ex_out = [[] for _ in extra]
    shrink = np.log(o["split_shrink"])
    for n, a in enumerate(act):
        if a == PRUNE:
            continue
        if a in (KEEP, CLONE):
            for k in p:
                out[k].append(p[k][n])
            for i, e in enumerate(extra):
                ex_out[i].append(np.asarray(e[n], dtype=np.float64))
        if a == CLONE:
            for k in p:
                out[k].append(p[k][n] + (o["phase_noise"] * z[n, 0, 3:] if k == "phase" else 0.0))
            for i, e in enumerate(extra):
                ex_out[i].append(np.zeros_like(np.asarray(e[n], dtype=np.float64)))
        if a == SPLIT:
            R = _rotation(p["quats"][n])
            s = np.exp(p["log_scales"][n])
            for child in range(2):
                for k in p:
                    if k == "means":
                        out[k].append(p[k][n] + R @ (s * z[n, child, :3]))
                    elif k == "log_scales":
                        out[k].append(p[k][n] - shrink)
                    elif k == "phase":
                        out[k].append(p[k][n] + o["phase_noise"] * z[n, child, 3:])
                    else:
                        out[k].append(p[k][n])
                for i, e in enumerate(extra):
                    ex_out[i].append(np.zeros_like(np.asarray(e[n], dtype=np.float64)))
    shapes = {k: p[k].shape[1:] for k in p}
    newp = {k: (np.array(v) if v else np.zeros((0,) + shapes[k])) for k, v in out.items()}
    newe = [np.array(v) if v else np.zeros((0,) + np.asarray(e).shape[1:]) for v, e in zip(ex_out, extra)]
    return newp, newe, act


# ----------------------------------------------------------------------------
# whole view(s)
# ----------------------------------------------------------------------------
def render(gauss: dict, viewmats, intrs, optics, opts=None):
    """Hologram P[V][C][H][W] and plane fields U[V][L][C][H][W] for V views
    (the optics' band_limit and padding, when present, select the ASM variant)."""
    viewmats = np.asarray(viewmats).reshape(-1, 4, 4)
    intrs = np.asarray(intrs).reshape(-1, 4)
    Ps, Us, Ts, Ns = [], [], [], []
    for v in range(viewmats.shape[0]):
        pr = project(gauss, viewmats[v], intrs[v], optics.H, optics.W, opts)
        U, T, nc = composite(pr, opts)
        Ps.append(propagate_planes(U, optics.pitch, optics.wavelengths, optics.plane_z,
                                   getattr(optics, "band_limit", 0), getattr(optics, "padding", 0)))
        Us.append(U); Ts.append(T); Ns.append(nc)
    return np.stack(Ps), np.stack(Us), np.stack(Ts), np.stack(Ns)


def render_backward(gauss: dict, viewmats, intrs, optics, gP, opts=None, rho_grad: int = 0) -> dict:
    """dL/dparams (float64) for the loss Re<gP, P> summed over views.
    rho_grad = 1: the plane logits also receive the dense plane-weight
    gradient of the planes a Gaussian is not assigned to, through the same
    straight-through rule (elementwise product with softmax(rho'/tau))."""
    viewmats = np.asarray(viewmats).reshape(-1, 4, 4)
    intrs = np.asarray(intrs).reshape(-1, 4)
    acc = None
    dense = None
    for v in range(viewmats.shape[0]):
        pr = project(gauss, viewmats[v], intrs[v], optics.H, optics.W, opts)
        gU = propagate_planes_adjoint(np.asarray(gP[v]), optics.pitch, optics.wavelengths, optics.plane_z,
                                      getattr(optics, "band_limit", 0), getattr(optics, "padding", 0))
        g2d = composite_backward(pr, gU, opts)
        acc = project_backward(gauss, viewmats[v], intrs[v], optics.H, optics.W, g2d, opts, acc)
        if rho_grad:
            d = composite_rho_dense(pr, gU, opts)
            dense = d if dense is None else dense + d
    if rho_grad and dense is not None:
        tau = (opts or DEFAULT_OPTS).get("tau", DEFAULT_OPTS["tau"])
        acc["plane_logits"] = acc["plane_logits"] + dense * ste_softmax(gauss["plane_logits"], tau)
    return acc


def loss_re_inner(P: np.ndarray, gP: np.ndarray) -> float:
    """Scalar Re<gP, P> = sum Re(conj(gP) P): its gradient w.r.t. P in the
    convention g = dL/dRe + j dL/dIm is gP itself."""
    return float(np.sum(np.real(np.conj(gP) * P)))


# ----------------------------------------------------------------------------
# optimiser and learned-initialisation network
# ----------------------------------------------------------------------------
def adam_step(p, g, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns new (p, m, v)."""
    p, g, m, v = (np.asarray(x, dtype=np.float64) for x in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned
    as float64: the 8 high bits of the float32 significand are kept."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    out = (u.astype(np.uint32)).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def mlp_forward(x, Ws, bs, act_round=None):
    """ReLU MLP: h_0 = x, h_{k+1} = relu(h_k W_k^T + b_k) except the last layer
    (linear).  ``act_round="bf16"`` rounds the hidden activations to bfloat16
    before they feed the next layer (the network is defined with BF16
    operands), so that the ReLU decisions are taken on the same values as on
    the GPU.  Returns the output and the list of (layer input, pre-activation)."""
    h = np.asarray(x, dtype=np.float64)
    pre = []
    for k, (Wk, bk) in enumerate(zip(Ws, bs)):
        z = h @ np.asarray(Wk, dtype=np.float64).T + np.asarray(bk, dtype=np.float64)
        pre.append((h, z))
        if k < len(Ws) - 1:
            h = np.maximum(z, 0.0)
            if act_round == "bf16":
                h = round_bf16(h)
        else:
            h = z
    return h, pre


def mlp_backward(x, Ws, bs, gy, act_round=None):
    """Reverse mode of ``mlp_forward`` (the activation rounding passes the
    gradient unchanged): (dL/dW_k, dL/db_k, dL/dx)."""
    _, pre = mlp_forward(x, Ws, bs, act_round)
    g = np.asarray(gy, dtype=np.float64)
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for k in range(len(Ws) - 1, -1, -1):
        h, z = pre[k]
        if k < len(Ws) - 1:
            g = g * (z > 0)
        gW[k] = g.T @ h
        gb[k] = g.sum(axis=0)
        g = g @ np.asarray(Ws[k], dtype=np.float64)
    return gW, gb, g
