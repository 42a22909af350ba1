"""Pins for the oracle's reverse mode (Supp. D.4 and Eq. ste).

The analytic gradient of the scalar Re<gP, P> (P the hologram) is checked
against central finite differences of the oracle's own forward pass, which is
pinned separately by closed forms.  Perturbations that would flip a discrete
decision (support, alpha_min, T_eps, the alpha_max clamp) are detected by
comparing the per-pixel contributor counts at theta +- h and skipped.
"""
import numpy as np
import pytest
from scipy.special import softmax

import hcgs_synth as S
import oracle

CLASSES = ("means", "log_scales", "quats", "opacity_logits", "amplitude", "phase")


def _setup(opts, N=14, L=2, C=2, H=28, W=36, seed=0, V=1, ls=-1.7):
    g = S.make_gaussians(N, L, C, H, W, seed=seed, log_scale_mean=ls, log_scale_std=0.3)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    # push the near Gaussians back so that none is culled or huge
    g["means"][:, 2] += 1.0
    optics = S.Optics(H, W, (639e-9, 473e-9)[:C], (0.0, 3e-3, 6e-3)[:L])
    vm, it = S.view_batch(V, H, W, seed=seed)
    gP = S.random_complex((V, C, H, W), seed=2).astype(np.complex128)
    return g, optics, vm, it, gP


def _loss(g, optics, vm, it, gP, opts):
    P, _, _, nc = oracle.render(g, vm, it, optics, opts)
    return oracle.loss_re_inner(P, gP), nc


def _check(opts, picks_per_class=4, V=1, seed=0, rtol=2e-6):
    g, optics, vm, it, gP = _setup(opts, V=V, seed=seed)
    grads = oracle.render_backward(g, vm, it, optics, gP, opts)
    rng = np.random.default_rng(11 + seed)
    checked = 0
    for nm in CLASSES:
        for _ in range(picks_per_class):
            idx = int(rng.integers(g[nm].size))
            th = g[nm].ravel()[idx]
            h = 1e-6 * max(1.0, abs(th))
            gp = {k: v.copy() for k, v in g.items()}
            gm = {k: v.copy() for k, v in g.items()}
            gp[nm].ravel()[idx] += h
            gm[nm].ravel()[idx] -= h
            lp, ncp = _loss(gp, optics, vm, it, gP, opts)
            lm, ncm = _loss(gm, optics, vm, it, gP, opts)
            if not np.array_equal(ncp, ncm):
                continue  # a discrete decision flipped inside the stencil
            fd = (lp - lm) / (2 * h)
            an = grads[nm].ravel()[idx]
            assert abs(fd - an) <= rtol * max(1.0, abs(fd)) + 1e-7, (nm, idx, fd, an)
            checked += 1
    assert checked >= len(CLASSES) * picks_per_class // 2
    return grads


def test_fd_exact_preset():
    _check(oracle.EXACT_OPTS)


def test_fd_default_thresholds():
    _check(oracle.DEFAULT_OPTS, seed=1)


def test_fd_back_to_front_two_views():
    _check(dict(oracle.DEFAULT_OPTS, order=1), V=2, seed=2)


def test_fd_clamped_jacobian():
    # Gaussians pushed far off-axis so that the J clamp (clip factor) is active.
    opts = dict(oracle.DEFAULT_OPTS, clip=0.6)
    g, optics, vm, it, gP = _setup(opts, seed=3)
    g["means"][:4, 0] = 1.6 * g["means"][:4, 2]
    g["means"][4:8, 1] = -1.2 * g["means"][4:8, 2]
    grads = oracle.render_backward(g, vm, it, optics, gP, opts)
    for nm, idx in [("means", 0), ("means", 2), ("means", 13), ("log_scales", 1), ("quats", 17)]:
        th = g[nm].ravel()[idx]
        h = 1e-6 * max(1.0, abs(th))
        gp = {k: v.copy() for k, v in g.items()}
        gm = {k: v.copy() for k, v in g.items()}
        gp[nm].ravel()[idx] += h
        gm[nm].ravel()[idx] -= h
        lp, ncp = _loss(gp, optics, vm, it, gP, opts)
        lm, ncm = _loss(gm, optics, vm, it, gP, opts)
        if not np.array_equal(ncp, ncm):
            continue
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[nm].ravel()[idx]) <= 2e-6 * max(1.0, abs(fd)) + 1e-7


def test_ste_plane_logit_gradient():
    # Eq. ste: dL/drho'_n = dL/drho_n * softmax(rho'_n / tau) (elementwise);
    # dL/drho_{n,l} is o dL/do at the assigned plane (alpha = o G rho) and 0
    # elsewhere.  Includes near-ties, where softmax(rho'/tau) is not one-hot.
    opts = dict(oracle.DEFAULT_OPTS)
    g, optics, vm, it, gP = _setup(opts, seed=4, L=3)
    g["plane_logits"][0] = [0.2, 0.2 + 3e-4, -1.0]
    g["plane_logits"][1] = [0.5, 0.5, 0.5]
    g["plane_logits"][2] = [0.0, -2e-3, 0.0]
    opts_b = dict(opts)
    grads = oracle.render_backward(g, vm, it, optics, gP, opts_b)
    # recover dL/do from the logit gradient: dL/dlogit = dL/do o (1 - o)
    o = 1 / (1 + np.exp(-g["opacity_logits"]))
    dLdo = grads["opacity_logits"] / (o * (1 - o))
    for n in range(g["means"].shape[0]):
        sm = softmax(g["plane_logits"][n] / opts["tau"])
        a = int(np.argmax(g["plane_logits"][n]))
        exp = np.zeros(3)
        exp[a] = o[n] * dLdo[n] * sm[a]
        assert np.allclose(grads["plane_logits"][n], exp, rtol=1e-10, atol=1e-15)
    # the near-tie rows really are soft
    assert 0.2 < softmax(g["plane_logits"][0] / 1e-3)[1] < 0.8


def test_composite_adjoint_dot_product():
    # P12 for the compositor: with every discrete decision frozen, the map
    # w -> U is linear, so <gU, U(w)> = <g_w, w> exactly.
    opts = dict(oracle.DEFAULT_OPTS)
    g, optics, vm, it, _ = _setup(opts, seed=5, N=30)
    pr = oracle.project(g, vm[0], it[0], optics.H, optics.W, opts)
    U, _, _ = oracle.composite(pr, opts)
    gU = S.random_complex(U.shape, seed=9).astype(np.complex128)
    g2 = oracle.composite_backward(pr, gU, opts)
    lhs = np.sum(np.real(np.conj(gU) * U))
    wc = pr["w"][..., 0] + 1j * pr["w"][..., 1]
    gw = g2["w"][..., 0] + 1j * g2["w"][..., 1]
    rhs = np.sum(np.real(np.conj(gw) * wc))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_mlp_reverse_mode():
    rng = np.random.default_rng(0)
    dims = [16, 12, 12, 8, 6]
    Ws = [rng.normal(size=(dims[k + 1], dims[k])) * 0.5 for k in range(4)]
    bs = [rng.normal(size=dims[k + 1]) * 0.1 for k in range(4)]
    x = rng.normal(size=(5, 16))
    gy = rng.normal(size=(5, 6))
    gW, gb, gx = oracle.mlp_backward(x, Ws, bs, gy)
    f = lambda Ws_, bs_, x_: float(np.sum(oracle.mlp_forward(x_, Ws_, bs_)[0] * gy))
    h = 1e-6
    for k in range(4):
        for (i, j) in [(0, 0), (dims[k + 1] - 1, dims[k] - 1)]:
            Wp = [w.copy() for w in Ws]; Wp[k][i, j] += h
            Wm = [w.copy() for w in Ws]; Wm[k][i, j] -= h
            fd = (f(Wp, bs, x) - f(Wm, bs, x)) / (2 * h)
            assert abs(fd - gW[k][i, j]) < 1e-6
    # a single linear layer is a plain matrix product
    y, _ = oracle.mlp_forward(x, Ws[:1], bs[:1])
    assert np.allclose(y, x @ Ws[0].T + bs[0])


def test_bf16_rounding_matches_torch():
    # the oracle's bfloat16 rounding against torch's float32 -> bfloat16 cast
    import torch
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, size=5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.0e38]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    assert np.array_equal(oracle.round_bf16(a), ref)


def test_mlp_bf16_activations_change_only_rounding():
    rng = np.random.default_rng(4)
    dims = [16, 32, 32, 8]
    Ws = [rng.normal(size=(dims[k + 1], dims[k])) / 4 for k in range(3)]
    bs = [rng.normal(size=dims[k + 1]) * 0.1 for k in range(3)]
    x = oracle.round_bf16(rng.normal(size=(50, 16)))
    y0, _ = oracle.mlp_forward(x, Ws, bs)
    y1, pre = oracle.mlp_forward(x, Ws, bs, act_round="bf16")
    assert 0 < np.max(np.abs(y1 - y0)) < 0.05 * np.max(np.abs(y0))
    # the input of layer 2 is exactly bf16-representable
    h = pre[1][0]
    assert np.array_equal(oracle.round_bf16(h), h)


def test_adam_first_step_closed_form():
    # first Adam step: m_hat = g, v_hat = g^2, so p1 = p0 - lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p0 = np.array([1.0, 2.0, 3.0])
    p1, m, v = oracle.adam_step(p0, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
