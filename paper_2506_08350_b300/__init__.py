"""Python binding of libhcgs (the B300 hologram render path of arXiv 2506.08350).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  There is no CPU fallback; importing this package without the built
library raises.  PyTorch provides device memory and the current stream.

Entry points keep the C names (``hcgs_<name>`` -> ``Context.<name>``):
project, rasterize_planes, asm_propagate, render_view and their _backward
twins, focal_stack_loss, adam_step, mlp_forward, mlp_backward.
``render`` / ``RenderFn`` wrap render_view in a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_int64, c_size_t, c_void_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# HCGS_CHECKED=1 in the environment loads the bounds-checked variant
CHECKED = os.environ.get("HCGS_CHECKED", "0") == "1"
LIB_PATH = os.path.join(_HERE, "_build_checked", "libhcgs_checked.so") if CHECKED else \
    os.path.join(_HERE, "_build", "libhcgs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libhcgs.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'` "
        "or `python paper_2506_08350_b300/build.py`" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "HCGS_OK", -1: "HCGS_ERR_INVALID_ARG", -2: "HCGS_ERR_CUDA", -3: "HCGS_ERR_CAPACITY",
          -4: "HCGS_ERR_UNSUPPORTED_SIZE", -5: "HCGS_ERR_DEVICE_CHECK", -6: "HCGS_ERR_TIMEOUT",
          -7: "HCGS_ERR_STATE"}

EXPORTS = ("hcgs_ctx_create", "hcgs_ctx_destroy", "hcgs_status_string", "hcgs_last_error", "hcgs_ctx_bytes",
           "hcgs_saved_create", "hcgs_saved_release", "hcgs_project", "hcgs_rasterize_planes",
           "hcgs_asm_propagate", "hcgs_asm_propagate_backward", "hcgs_render_view",
           "hcgs_rasterize_planes_backward", "hcgs_project_backward", "hcgs_render_view_backward",
           "hcgs_focal_stack_loss", "hcgs_adam_step", "hcgs_mlp_forward", "hcgs_mlp_backward",
           "hcgs_profile_enable", "hcgs_profile_summary", "hcgs_asm_propagate_noalloc", "hcgs_mlp_mse_loss",
           "hcgs_cast_bf16", "hcgs_init_features", "hcgs_init_targets", "hcgs_init_apply",
           "hcgs_selftest_wait_timeout", "hcgs_paper_loss", "hcgs_paper_loss_intensities", "hcgs_adan_step",
           "hcgs_densify_accumulate", "hcgs_densify_plan", "hcgs_densify_apply", "hcgs_philox",
           "hcgs_phase_only_loss", "hcgs_hologram_phase", "hcgs_phase_hologram", "hcgs_scale",
           "hcgs_is_checked_build", "hcgs_check_status", "hcgs_selftest_device_check",
           "hcgs_adam_step_multi", "hcgs_adan_step_multi")


class HcgsError(RuntimeError):
    pass


class _Optics(ctypes.Structure):
    _fields_ = [("H", c_int), ("W", c_int), ("C", c_int), ("L", c_int), ("pitch_x", c_double),
                ("pitch_y", c_double), ("wavelength", POINTER(c_double)), ("plane_z", POINTER(c_double)),
                ("band_limit", c_int), ("padding", c_int)]


class _RasterOpts(ctypes.Structure):
    _fields_ = [("tile", c_int), ("alpha_min", c_float), ("alpha_max", c_float), ("T_eps", c_float),
                ("cov2d_dilation", c_float), ("near_z", c_float), ("clip_factor", c_float),
                ("ste_tau", c_float), ("order", c_int), ("footprint", c_int), ("rho_grad", c_int)]


class _Gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("amplitude", c_void_p), ("phase", c_void_p),
                ("plane_logits", c_void_p), ("N", c_int)]


class _DensifyOpts(ctypes.Structure):
    _fields_ = [("grad_threshold", c_float), ("split_scale", c_float), ("prune_opacity", c_float),
                ("prune_scale", c_float), ("split_shrink", c_float), ("phase_noise", c_float)]


class _Grads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("amplitude", c_void_p), ("phase", c_void_p),
                ("plane_logits", c_void_p)]


def _sig(name, args):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = c_int
    return f


_P = c_void_p
_lib.hcgs_status_string.argtypes = [c_int]
_lib.hcgs_status_string.restype = ctypes.c_char_p
_lib.hcgs_last_error.argtypes = [_P]
_lib.hcgs_last_error.restype = ctypes.c_char_p
_lib.hcgs_ctx_bytes.argtypes = [_P]
_lib.hcgs_ctx_bytes.restype = c_size_t
_lib.hcgs_ctx_destroy.argtypes = [_P]
_lib.hcgs_ctx_destroy.restype = None
_sig("hcgs_ctx_create", [POINTER(c_void_p), c_int])
_sig("hcgs_saved_create", [_P, POINTER(c_void_p)])
_sig("hcgs_profile_enable", [_P, c_int])
_sig("hcgs_selftest_wait_timeout", [_P, _P])
_sig("hcgs_check_status", [_P, _P])
_sig("hcgs_selftest_device_check", [_P, c_int, _P])
_lib.hcgs_is_checked_build.argtypes = []
_lib.hcgs_is_checked_build.restype = c_int
_sig("hcgs_profile_summary", [_P, c_int, POINTER(c_int), POINTER(ctypes.c_char_p), POINTER(c_double),
                              POINTER(c_int64)])
_sig("hcgs_saved_release", [_P, _P])
_sig("hcgs_project", [_P, POINTER(_Gaussians), c_int, _P, _P, POINTER(_Optics), POINTER(_RasterOpts), _P, _P])
_sig("hcgs_rasterize_planes", [_P, _P, _P, _P, _P, _P])
_sig("hcgs_asm_propagate", [_P, _P, c_int, POINTER(_Optics), c_int, c_int, _P, _P])
_sig("hcgs_asm_propagate_backward", [_P, _P, c_int, POINTER(_Optics), c_int, c_int, _P, _P])
_sig("hcgs_render_view", [_P, POINTER(_Gaussians), c_int, _P, _P, POINTER(_Optics), POINTER(_RasterOpts), _P, _P,
                          _P, _P])
_sig("hcgs_rasterize_planes_backward", [_P, _P, _P, _P])
_sig("hcgs_project_backward", [_P, _P, POINTER(_Gaussians), POINTER(_Grads), c_int, _P])
_sig("hcgs_render_view_backward", [_P, _P, POINTER(_Gaussians), _P, POINTER(_Grads), c_int, _P])
_sig("hcgs_focal_stack_loss", [_P, _P, _P, c_int, POINTER(_Optics), _P, _P, _P, _P])
_sig("hcgs_adam_step", [_P, _P, _P, _P, _P, c_int64, c_int, c_float, c_float, c_float, c_float, _P])
_sig("hcgs_densify_accumulate", [_P, _P, _P, _P, _P])
_sig("hcgs_densify_plan", [_P, POINTER(_Gaussians), _P, _P, POINTER(_DensifyOpts), _P, _P, POINTER(c_int64), _P])
_sig("hcgs_densify_apply", [_P, POINTER(_Gaussians), c_int, c_int, _P, _P, _P, POINTER(_DensifyOpts),
                            POINTER(_Grads), c_int, _P, _P, _P, _P])
_sig("hcgs_philox", [_P, ctypes.c_uint64, ctypes.c_uint32, c_int64, c_int, _P, _P])
_sig("hcgs_phase_only_loss", [_P, _P, _P, c_int, POINTER(_Optics), c_float, _P, _P, _P])
_sig("hcgs_hologram_phase", [_P, _P, c_int64, _P, _P])
_sig("hcgs_phase_hologram", [_P, _P, c_int64, _P, _P])
_sig("hcgs_scale", [_P, _P, c_int64, c_float, _P, _P])
_sig("hcgs_paper_loss", [_P, _P, _P, _P, c_int, POINTER(_Optics), c_float, _P, _P, _P, _P])
_sig("hcgs_paper_loss_intensities", [_P, _P, _P, _P, c_int, c_int, c_int, c_int, c_int, c_float, _P, _P, _P])
_sig("hcgs_adan_step", [_P, _P, _P, _P, _P, _P, _P, c_int64, c_int, c_float, c_float, c_float, c_float, c_float,
                        c_float, _P])
_PP = POINTER(c_void_p)
_sig("hcgs_adam_step_multi", [_P, c_int, _PP, _PP, _PP, _PP, POINTER(c_int64), POINTER(c_float), c_int, c_float,
                              c_float, c_float, _P])
_sig("hcgs_adan_step_multi", [_P, c_int, _PP, _PP, _PP, _PP, _PP, _PP, POINTER(c_int64), POINTER(c_float), c_int,
                              c_float, c_float, c_float, c_float, c_float, _P])
_sig("hcgs_mlp_forward", [_P, _P, c_int] + [_P] * 8 + [_P, _P])
_sig("hcgs_asm_propagate_noalloc", [_P, c_int, POINTER(_Optics), _P, _P])
_sig("hcgs_mlp_mse_loss", [_P, _P, _P, c_int, c_int, _P, _P, _P])
_sig("hcgs_cast_bf16", [_P, _P, _P, c_int64, _P])
_sig("hcgs_init_features", [_P, POINTER(_Gaussians), _P, _P, _P])
_sig("hcgs_init_targets", [_P, _P, _P, c_int, c_int, _P, _P])
_sig("hcgs_init_apply", [_P, _P, c_int, c_int, _P, _P, _P])
_sig("hcgs_mlp_backward", [_P, _P, c_int] + [_P] * 8 + [_P] + [_P] * 8 + [_P])

SSIM_LAMBDA = 0.005  # lambda_1 of the SSIM term (Sec. 4.1, loss paragraph)
# densification (Algorithm 1; the 3DGS rules Sec. 5 adopts); split_scale is
# scene-dependent (3DGS: 1 % of the scene extent; 0.02 m for the 1-3 m scenes here)
DEFAULT_DENSIFY = dict(grad_threshold=2e-4, split_scale=0.02, prune_opacity=5e-3, prune_scale=0.0,
                       split_shrink=1.6, phase_noise=0.1)
DENSIFY_PERIOD = 300

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "amplitude", "phase", "plane_logits")

DEFAULT_OPTS = dict(tile=16, alpha_min=1.0 / 255.0, alpha_max=0.99, T_eps=1e-4, cov2d_dilation=0.3,
                    near_z=0.2, clip_factor=1.3, ste_tau=1e-3, order=0, footprint=0, rho_grad=0)
EXACT_OPTS = dict(DEFAULT_OPTS, alpha_min=0.0, alpha_max=1.0, T_eps=0.0, cov2d_dilation=0.0, clip_factor=0.0)


def _ptrs(ts):
    """A host array of the device pointers of a list of tensors."""
    return (c_void_p * len(ts))(*[_ptr(t) for t in ts])


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return c_void_p(t.data_ptr())


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def make_optics(o):
    """hcgs_optics from any object with H, W, wavelengths, plane_z, pitch (and
    optionally band_limit and padding, default 0)."""
    lam = (c_double * len(o.wavelengths))(*[float(x) for x in o.wavelengths])
    z = (c_double * len(o.plane_z))(*[float(x) for x in o.plane_z])
    s = _Optics(int(o.H), int(o.W), len(o.wavelengths), len(o.plane_z), float(o.pitch), float(o.pitch),
                ctypes.cast(lam, POINTER(c_double)), ctypes.cast(z, POINTER(c_double)),
                int(getattr(o, "band_limit", 0)), int(getattr(o, "padding", 0)))
    s._keep = (lam, z)
    return s


def make_opts(opts=None):
    d = dict(DEFAULT_OPTS)
    d.update(opts or {})
    return _RasterOpts(**{k: d[k] for k, _ in _RasterOpts._fields_})


def _gauss(g):
    for k in PARAM_NAMES:
        if g[k].dtype != torch.float32:
            raise TypeError("%s must be float32" % k)
    N = g["means"].shape[0]
    return _Gaussians(*[_ptr(g[k]) for k in PARAM_NAMES], N)


def _grads(gr):
    return _Grads(*[_ptr(gr[k]) for k in PARAM_NAMES])


class Saved:
    """Forward state (hcgs_saved) reused by the backward."""

    def __init__(self, ctx: "Context"):
        self._ctx = ctx
        h = c_void_p()
        ctx._check(_lib.hcgs_saved_create(ctx.handle, ctypes.byref(h)))
        self.handle = h

    def release(self):
        if self.handle is not None and self._ctx.handle is not None:
            _lib.hcgs_saved_release(self._ctx.handle, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Context:
    """An hcgs_ctx on one device."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = c_void_p()
        rc = _lib.hcgs_ctx_create(ctypes.byref(h), int(device))
        if rc != 0:
            raise HcgsError("hcgs_ctx_create failed: %s" % STATUS.get(rc, rc))
        self.handle = h

    def close(self):
        if self.handle is not None:
            _lib.hcgs_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            msg = _lib.hcgs_last_error(self.handle).decode()
            raise HcgsError("%s (%s)" % (STATUS.get(rc, rc), msg))

    def bytes(self) -> int:
        return int(_lib.hcgs_ctx_bytes(self.handle))

    def selftest_wait_timeout(self):
        """Launches a kernel whose bounded wait runs out (about one second); the
        next project / render_view call then raises HcgsError(HCGS_ERR_TIMEOUT)."""
        self._check(_lib.hcgs_selftest_wait_timeout(self.handle, _stream()))

    def check_status(self):
        """hcgs_check_status on the current stream: raises HcgsError
        (HCGS_ERR_DEVICE_CHECK / HCGS_ERR_TIMEOUT) for what the device recorded."""
        self._check(_lib.hcgs_check_status(self.handle, _stream()))

    def selftest_device_check(self, kind):
        self._check(_lib.hcgs_selftest_device_check(self.handle, int(kind), _stream()))

    def profile_enable(self, on=True):
        self._check(_lib.hcgs_profile_enable(self.handle, int(bool(on))))

    def profile_summary(self, max_kernels=64):
        """{kernel name: (total ms, launches)} since profile_enable, in launch order."""
        names = (ctypes.c_char_p * max_kernels)()
        ms = (c_double * max_kernels)()
        cnt = (c_int64 * max_kernels)()
        n = c_int()
        self._check(_lib.hcgs_profile_summary(self.handle, max_kernels, ctypes.byref(n), names, ms, cnt))
        return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(n.value)}

    # ---- steps ----
    def project(self, g, viewmats, intrinsics, optics, opts, saved: Saved):
        V = viewmats.shape[0]
        self._check(_lib.hcgs_project(self.handle, ctypes.byref(_gauss(g)), V, _ptr(viewmats), _ptr(intrinsics),
                                      ctypes.byref(make_optics(optics)), ctypes.byref(make_opts(opts)),
                                      saved.handle, _stream()))

    def rasterize_planes(self, saved: Saved, U, T_final=None, n_contrib=None):
        self._check(_lib.hcgs_rasterize_planes(self.handle, saved.handle, _ptr(U), _ptr(T_final), _ptr(n_contrib),
                                               _stream()))

    def asm_propagate(self, inp, B, optics, sign, reduce_planes, out):
        self._check(_lib.hcgs_asm_propagate(self.handle, _ptr(inp), int(B), ctypes.byref(make_optics(optics)),
                                            int(sign), int(reduce_planes), _ptr(out), _stream()))

    def asm_propagate_backward(self, g_out, B, optics, sign, reduce_planes, g_in):
        self._check(_lib.hcgs_asm_propagate_backward(self.handle, _ptr(g_out), int(B),
                                                     ctypes.byref(make_optics(optics)), int(sign),
                                                     int(reduce_planes), _ptr(g_in), _stream()))

    def render_view(self, g, viewmats, intrinsics, optics, opts, hologram, planes=None, saved: Saved | None = None):
        V = viewmats.shape[0]
        self._check(_lib.hcgs_render_view(self.handle, ctypes.byref(_gauss(g)), V, _ptr(viewmats),
                                          _ptr(intrinsics), ctypes.byref(make_optics(optics)),
                                          ctypes.byref(make_opts(opts)), _ptr(hologram), _ptr(planes),
                                          saved.handle if saved else None, _stream()))

    def rasterize_planes_backward(self, saved: Saved, gU):
        self._check(_lib.hcgs_rasterize_planes_backward(self.handle, saved.handle, _ptr(gU), _stream()))

    def project_backward(self, saved: Saved, g, grads, accumulate=False):
        self._check(_lib.hcgs_project_backward(self.handle, saved.handle, ctypes.byref(_gauss(g)),
                                               ctypes.byref(_grads(grads)), int(bool(accumulate)), _stream()))

    def render_view_backward(self, saved: Saved, g, g_hologram, grads, accumulate=False):
        self._check(_lib.hcgs_render_view_backward(self.handle, saved.handle, ctypes.byref(_gauss(g)),
                                                   _ptr(g_hologram), ctypes.byref(_grads(grads)),
                                                   int(bool(accumulate)), _stream()))

    def focal_stack_loss(self, hologram, I_gt, B, optics, loss, g_hologram=None, I_out=None):
        self._check(_lib.hcgs_focal_stack_loss(self.handle, _ptr(hologram), _ptr(I_gt), int(B),
                                               ctypes.byref(make_optics(optics)), _ptr(loss), _ptr(g_hologram),
                                               _ptr(I_out), _stream()))

    def paper_loss(self, hologram, I_gt, masks, B, optics, loss, g_hologram=None, I_out=None,
                   lambda_ssim=SSIM_LAMBDA):
        self._check(_lib.hcgs_paper_loss(self.handle, _ptr(hologram), _ptr(I_gt), _ptr(masks), int(B),
                                         ctypes.byref(make_optics(optics)), float(lambda_ssim), _ptr(loss),
                                         _ptr(g_hologram), _ptr(I_out), _stream()))

    def paper_loss_intensities(self, I, I_gt, masks, loss, g_I, lambda_ssim=SSIM_LAMBDA):
        B, L, C, H, W = I.shape
        self._check(_lib.hcgs_paper_loss_intensities(self.handle, _ptr(I), _ptr(I_gt), _ptr(masks), B, L, C, H, W,
                                                     float(lambda_ssim), _ptr(loss), _ptr(g_I), _stream()))

    def adan_step(self, p, g, g_prev, m, v, n, step, lr, beta1=0.9, beta2=0.92, beta3=0.99, eps=1e-8,
                  weight_decay=0.0):
        self._check(_lib.hcgs_adan_step(self.handle, _ptr(p), _ptr(g), _ptr(g_prev), _ptr(m), _ptr(v), _ptr(n),
                                        p.numel(), int(step), float(lr), float(beta1), float(beta2), float(beta3),
                                        float(eps), float(weight_decay), _stream()))

    def adam_step(self, p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(_lib.hcgs_adam_step(self.handle, _ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), int(step),
                                        float(lr), float(beta1), float(beta2), float(eps), _stream()))

    def adam_step_multi(self, ps, gs, ms, vs, step, lrs, beta1=0.9, beta2=0.999, eps=1e-8):
        """adam_step on several parameter arrays (lists of equal length) in one launch."""
        k = len(ps)
        self._check(_lib.hcgs_adam_step_multi(self.handle, k, _ptrs(ps), _ptrs(gs), _ptrs(ms), _ptrs(vs),
                                              (c_int64 * k)(*[t.numel() for t in ps]),
                                              (c_float * k)(*[float(x) for x in lrs]), int(step), float(beta1),
                                              float(beta2), float(eps), _stream()))

    def adan_step_multi(self, ps, gs, g_prevs, ms, vs, ns, step, lrs, beta1=0.9, beta2=0.92, beta3=0.99,
                        eps=1e-8, weight_decay=0.0):
        """adan_step on several parameter arrays (lists of equal length) in one launch."""
        k = len(ps)
        self._check(_lib.hcgs_adan_step_multi(self.handle, k, _ptrs(ps), _ptrs(gs), _ptrs(g_prevs), _ptrs(ms),
                                              _ptrs(vs), _ptrs(ns), (c_int64 * k)(*[t.numel() for t in ps]),
                                              (c_float * k)(*[float(x) for x in lrs]), int(step), float(beta1),
                                              float(beta2), float(beta3), float(eps), float(weight_decay),
                                              _stream()))

    def phase_only_loss(self, U_target, phase, B, optics, loss, g_phase=None, lambda_ssim=SSIM_LAMBDA):
        self._check(_lib.hcgs_phase_only_loss(self.handle, _ptr(U_target), _ptr(phase), int(B),
                                              ctypes.byref(make_optics(optics)), float(lambda_ssim), _ptr(loss),
                                              _ptr(g_phase), _stream()))

    def scale(self, x, s, out):
        """out = s x elementwise (float32 storage; complex arrays as their floats)."""
        n = x.numel() * (2 if x.is_complex() else 1)
        self._check(_lib.hcgs_scale(self.handle, _ptr(x), n, float(s), _ptr(out), _stream()))

    def phase_hologram(self, phase, hologram):
        self._check(_lib.hcgs_phase_hologram(self.handle, _ptr(phase), phase.numel(), _ptr(hologram), _stream()))

    def hologram_phase(self, hologram, phase):
        self._check(_lib.hcgs_hologram_phase(self.handle, _ptr(hologram), hologram.numel(), _ptr(phase), _stream()))

    def philox(self, seed, n, out, kind=1, stream_id=0):
        """n counter-based random numbers into `out` (kind 0: uint32 words as
        int32/uint32 storage, 1: float32 standard normals, 2: float32 uniforms in (0, 1))."""
        self._check(_lib.hcgs_philox(self.handle, int(seed) & (2 ** 64 - 1), int(stream_id) & 0xFFFFFFFF, int(n),
                                     int(kind), _ptr(out), _stream()))

    def densify_accumulate(self, saved, accum, denom):
        self._check(_lib.hcgs_densify_accumulate(self.handle, saved.handle, _ptr(accum), _ptr(denom), _stream()))

    def densify_plan(self, g, accum, denom, opts=None):
        """Returns (action int32 [N], offsets int32 storage of uint32 [N + 1], new count)."""
        import torch
        o = _DensifyOpts(**{**DEFAULT_DENSIFY, **(opts or {})})
        N = g["means"].shape[0]
        dev = g["means"].device
        action = torch.empty(N, dtype=torch.int32, device=dev)
        offsets = torch.empty(N + 1, dtype=torch.int32, device=dev)
        n_out = c_int64(0)
        self._check(_lib.hcgs_densify_plan(self.handle, ctypes.byref(_gauss(g)), _ptr(accum), _ptr(denom),
                                           ctypes.byref(o), _ptr(action), _ptr(offsets), ctypes.byref(n_out),
                                           _stream()))
        return action, offsets, int(n_out.value)

    def densify_apply(self, g, C, L, action, offsets, noise, g_out, opts=None, extras=()):
        """Write the densified Gaussians into g_out (dict of arrays with the new
        count of rows); extras: (in, out) pairs of per-Gaussian float arrays."""
        o = _DensifyOpts(**{**DEFAULT_DENSIFY, **(opts or {})})
        k = len(extras)
        ins = (c_void_p * max(k, 1))(*[_ptr(a) for a, _ in extras])
        outs = (c_void_p * max(k, 1))(*[_ptr(b) for _, b in extras])
        widths = (c_int * max(k, 1))(*[int(a[0].numel()) if a.shape[0] > 0 and a.dim() > 1 else 1
                                       for a, _ in extras])
        self._check(_lib.hcgs_densify_apply(self.handle, ctypes.byref(_gauss(g)), int(C), int(L), _ptr(action),
                                            _ptr(offsets), _ptr(noise), ctypes.byref(o), ctypes.byref(_grads(g_out)),
                                            k, ins, outs, widths, _stream()))

    def mlp_forward(self, x, W, b, y):
        self._check(_lib.hcgs_mlp_forward(self.handle, _ptr(x), x.shape[0], *[_ptr(w) for w in W],
                                          *[_ptr(t) for t in b], _ptr(y), _stream()))

    def mlp_mse_loss(self, y, target, K, loss, gy):
        self._check(_lib.hcgs_mlp_mse_loss(self.handle, _ptr(y), _ptr(target), y.shape[0], int(K), _ptr(loss),
                                           _ptr(gy), _stream()))

    def cast_bf16(self, src, dst):
        self._check(_lib.hcgs_cast_bf16(self.handle, _ptr(src), _ptr(dst), src.numel(), _stream()))

    def init_features(self, g, rgb, x):
        self._check(_lib.hcgs_init_features(self.handle, ctypes.byref(_gauss(g)), _ptr(rgb), _ptr(x), _stream()))

    def init_targets(self, amplitude, phase, target):
        N, C = amplitude.shape
        self._check(_lib.hcgs_init_targets(self.handle, _ptr(amplitude), _ptr(phase), N, C, _ptr(target),
                                           _stream()))

    def init_apply(self, y, amplitude, phase):
        N, C = amplitude.shape
        self._check(_lib.hcgs_init_apply(self.handle, _ptr(y), N, C, _ptr(amplitude), _ptr(phase), _stream()))

    def mlp_backward(self, x, W, b, gy, gW, gb):
        self._check(_lib.hcgs_mlp_backward(self.handle, _ptr(x), x.shape[0], *[_ptr(w) for w in W],
                                           *[_ptr(t) for t in b], _ptr(gy), *[_ptr(t) for t in gW],
                                           *[_ptr(t) for t in gb], _stream()))


def asm_propagate_noalloc(inp, B, optics, out):
    """hcgs_asm_propagate_noalloc: inverse propagation without any device
    allocation (see include/hcgs.h for its size limit and sharing rules)."""
    rc = _lib.hcgs_asm_propagate_noalloc(_ptr(inp), int(B), ctypes.byref(make_optics(optics)), _ptr(out),
                                         _stream())
    if rc != 0:
        raise HcgsError("hcgs_asm_propagate_noalloc: %s" % STATUS.get(rc, rc))


_default_ctx = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context()
    return _default_ctx


class RenderFn(torch.autograd.Function):
    """Hologram of V views as a differentiable function of the Gaussian
    parameters; the backward runs hcgs_render_view_backward."""

    @staticmethod
    def forward(fctx, means, log_scales, quats, opacity_logits, amplitude, phase, plane_logits, viewmats, intr,
                optics, opts, context):
        g = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                 opacity_logits=opacity_logits.contiguous(), amplitude=amplitude.contiguous(),
                 phase=phase.contiguous(), plane_logits=plane_logits.contiguous())
        V = viewmats.shape[0]
        holo = torch.empty((V, len(optics.wavelengths), optics.H, optics.W), dtype=torch.complex64,
                           device=means.device)
        saved = Saved(context)
        context.render_view(g, viewmats.contiguous(), intr.contiguous(), optics, opts, holo, None, saved)
        fctx.saved = saved
        fctx.context = context
        fctx.g = g
        return holo

    @staticmethod
    def backward(fctx, g_holo):
        g = fctx.g
        grads = {k: torch.empty_like(g[k]) for k in PARAM_NAMES}
        fctx.context.render_view_backward(fctx.saved, g, g_holo.contiguous().to(torch.complex64), grads)
        fctx.saved.release()
        return tuple(grads[k] for k in PARAM_NAMES) + (None,) * 5


def render(gauss: dict, viewmats, intrinsics, optics, opts=None, context: Context | None = None):
    """Differentiable hologram [V, C, H, W] (complex64)."""
    context = context or default_context()
    return RenderFn.apply(*[gauss[k] for k in PARAM_NAMES], viewmats, intrinsics, optics, opts, context)


class ASMFn(torch.autograd.Function):
    """Forward recording (plane fields [B, L, C, H, W] -> hologram [B, C, H, W])."""

    @staticmethod
    def forward(fctx, U, optics, context):
        B = U.shape[0]
        out = torch.empty((B,) + tuple(U.shape[2:]), dtype=torch.complex64, device=U.device)
        context.asm_propagate(U.contiguous(), B, optics, 1, 1, out)
        fctx.optics, fctx.context, fctx.shape = optics, context, U.shape
        return out

    @staticmethod
    def backward(fctx, g):
        gU = torch.empty(fctx.shape, dtype=torch.complex64, device=g.device)
        fctx.context.asm_propagate_backward(g.contiguous().to(torch.complex64), fctx.shape[0], fctx.optics, 1, 1,
                                            gU)
        return gU, None, None


def propagate(U, optics, context: Context | None = None):
    return ASMFn.apply(U, optics, context or default_context())
