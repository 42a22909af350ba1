"""Pins for the oracle's version of the paper's training objective.

L = L_recon + L_SSIM (the loss paragraph of Sec. 4.1), the Adan optimiser and
the cosine learning-rate schedule (Sec. 5, implementation).  Each check rests
on something other than the oracle's own formula: a brute-force window sum,
finite differences, reduction to the plain focal-stack loss, and properties
of the optimiser.
"""
import math

import numpy as np

import oracle

PITCH = 8e-6


def _rng(seed):
    return np.random.default_rng(seed)


def _ssim_brute(x, y):
    # SSIM map by explicit window sums over an 11 x 11 neighbourhood, zero
    # outside the image (the window written out from the Gaussian itself)
    H, W = x.shape
    r = 5
    k = np.array([[math.exp(-(i * i + j * j) / (2 * 1.5 ** 2)) for j in range(-r, r + 1)] for i in range(-r, r + 1)])
    k /= k.sum()
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = sxx = syy = sxy = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        wv = k[a + r, b + r]
                        xv, yv = x[ii, jj], y[ii, jj]
                        mx += wv * xv
                        my += wv * yv
                        sxx += wv * xv * xv
                        syy += wv * yv * yv
                        sxy += wv * xv * yv
            vx, vy, cxy = sxx - mx * mx, syy - my * my, sxy - mx * my
            c1, c2 = 0.01 ** 2, 0.03 ** 2
            out[i, j] = (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    return out


def test_ssim_map_matches_brute_force_window_sums():
    x, y = _rng(0).random((13, 17)), _rng(1).random((13, 17))
    assert np.max(np.abs(oracle.ssim_map(x, y) - _ssim_brute(x, y))) < 1e-12


def test_ssim_identity_and_symmetry():
    x, y = _rng(2).random((32, 40)) * 3.0, _rng(3).random((32, 40))
    assert abs(oracle.ssim(x, x) - 1.0) < 1e-12
    assert abs(oracle.ssim(x, y) - oracle.ssim(y, x)) < 1e-14
    assert oracle.ssim(x, y) < 0.5


def test_ssim_gradient_finite_differences():
    x, y = _rng(4).random((12, 15)), _rng(5).random((12, 15))
    g = oracle.ssim_grad(x, y)
    h = 1e-6
    for (i, j) in [(0, 0), (5, 7), (11, 14), (3, 0), (6, 13)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j] += h
        xm[i, j] -= h
        fd = (oracle.ssim(xp, y) - oracle.ssim(xm, y)) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-8 * max(1.0, abs(fd)), (i, j, fd, g[i, j])


def test_recon_loss_reduces_to_plain_focal_stack_loss():
    # with zero targets and masks the weights are 1 and, without the SSIM
    # term, L_recon is the mean squared intensity of the plain loss
    C, H, W = 2, 16, 20
    z = (0.0, 2e-3, 5e-3)
    P = _rng(6).normal(size=(C, H, W)) + 1j * _rng(7).normal(size=(C, H, W))
    Igt = np.zeros((len(z), C, H, W))
    M = np.zeros((len(z), H, W))
    l1, g1, I1 = oracle.paper_loss(P, Igt, M, PITCH, (639e-9, 515e-9), z, lam=0.0)
    l0, g0, I0 = oracle.focal_stack_loss(P, Igt, PITCH, (639e-9, 515e-9), z)
    assert abs(l1 - l0) < 1e-12 * abs(l0)
    assert np.max(np.abs(g1 - g0)) < 1e-12 * np.max(np.abs(g0))


def test_paper_loss_gradient_finite_differences():
    C, H, W = 1, 16, 16
    z = (0.0, 3e-3)
    rng = _rng(8)
    P = rng.normal(size=(C, H, W)) + 1j * rng.normal(size=(C, H, W))
    Igt = rng.random((len(z), C, H, W)) * 2.0
    M = (rng.random((len(z), H, W)) < 0.4).astype(np.float64)
    loss, gP, _ = oracle.paper_loss(P, Igt, M, PITCH, (515e-9,), z, lam=0.5)
    h = 1e-6
    for (c, i, j, part) in [(0, 0, 0, 1.0), (0, 7, 3, 1j), (0, 15, 15, 1.0), (0, 4, 11, 1j)]:
        Pp, Pm = P.copy(), P.copy()
        Pp[c, i, j] += h * part
        Pm[c, i, j] -= h * part
        fd = (oracle.paper_loss(Pp, Igt, M, PITCH, (515e-9,), z, lam=0.5)[0] -
              oracle.paper_loss(Pm, Igt, M, PITCH, (515e-9,), z, lam=0.5)[0]) / (2 * h)
        # g = dL/dRe + j dL/dIm
        want = gP[c, i, j].real if part == 1.0 else gP[c, i, j].imag
        assert abs(fd - want) < 1e-6 * max(1.0, abs(fd)), (c, i, j, fd, want)


def test_recon_loss_weights_reduce_to_scaled_plain_loss():
    # L_recon = mean d^2 + mean (M d)^2 + mean (I_gt d)^2 with d = I - I_gt:
    # with every mask 1 and zero targets it is twice the plain focal-stack
    # loss; with zero masks and a constant target c it is (1 + c^2) times it
    # (lambda_1 = 0 in both; the gradients scale the same way)
    C, H, W = 1, 12, 14
    z = (0.0, 2e-3)
    P = _rng(12).normal(size=(C, H, W)) + 1j * _rng(13).normal(size=(C, H, W))
    zero = np.zeros((len(z), C, H, W))
    l0, g0, _ = oracle.focal_stack_loss(P, zero, PITCH, (515e-9,), z)
    l1, g1, _ = oracle.paper_loss(P, zero, np.ones((len(z), H, W)), PITCH, (515e-9,), z, lam=0.0)
    assert abs(l1 - 2.0 * l0) < 1e-12 * l0
    assert np.max(np.abs(g1 - 2.0 * g0)) < 1e-12 * np.max(np.abs(g0))
    c = 0.7
    Igt = np.full((len(z), C, H, W), c)
    l0, g0, _ = oracle.focal_stack_loss(P, Igt, PITCH, (515e-9,), z)
    l2, g2, _ = oracle.paper_loss(P, Igt, np.zeros((len(z), H, W)), PITCH, (515e-9,), z, lam=0.0)
    assert abs(l2 - (1 + c * c) * l0) < 1e-12 * l0
    assert np.max(np.abs(g2 - (1 + c * c) * g0)) < 1e-12 * np.max(np.abs(g0))


def test_adan_matches_the_algorithm_in_its_authors_notation():
    # Adan as its authors state it (Xie et al., Algorithm 1), with small
    # momentum coefficients a = 1 - beta:
    #   m_k = (1 - a1) m + a1 g_k,  v_k = (1 - a2) v + a2 (g_k - g_{k-1}),
    #   n_k = (1 - a3) n + a3 (g_k + (1 - a2)(g_k - g_{k-1}))^2,
    #   theta <- theta - lr (m_k + (1 - a2) v_k) / (sqrt(n_k) + eps),
    # started with m = g_0, v = 0, n = g_0^2 and v_1 = g_1 - g_0.
    rng = _rng(14)
    a1, a2, a3 = 0.1, 0.08, 0.01
    lr, eps = 0.02, 1e-8
    gs = [rng.normal(size=5) for _ in range(7)]
    th = rng.normal(size=5)
    m, v, n = gs[0].copy(), np.zeros(5), gs[0] ** 2
    th_ref = [th - lr * m / (np.sqrt(n) + eps)]
    for k in range(1, len(gs)):
        dg = gs[k] - gs[k - 1]
        m = (1 - a1) * m + a1 * gs[k]
        v = dg if k == 1 else (1 - a2) * v + a2 * dg
        n = (1 - a3) * n + a3 * (gs[k] + (1 - a2) * dg) ** 2
        th_ref.append(th_ref[-1] - lr * (m + (1 - a2) * v) / (np.sqrt(n) + eps))
    p, mo, vo, no = th.copy(), np.zeros(5), np.zeros(5), np.zeros(5)
    prev = np.zeros(5)
    for k, g in enumerate(gs):
        p, mo, vo, no = oracle.adan_step(p, g, prev, mo, vo, no, k + 1, lr, 1 - a1, 1 - a2, 1 - a3, eps)
        prev = g
        assert np.allclose(p, th_ref[k], rtol=1e-13, atol=1e-15), k


def test_paper_loss_is_a_mean_over_planes_and_channels():
    # both terms are means over (planes, channels): repeating every image
    # along the plane and channel axes leaves the loss unchanged and spreads
    # the gradient evenly over the copies
    rng = _rng(15)
    I = rng.random((2, 1, 12, 14)) * 2.0
    Igt = rng.random((2, 1, 12, 14)) * 2.0
    M = (rng.random((2, 12, 14)) < 0.5).astype(np.float64)
    l1, g1 = oracle.paper_loss_intensities(I, Igt, M, lam=0.7)
    rep = lambda a: np.concatenate([np.concatenate([a, a], axis=1)] * 3, axis=0)
    l6, g6 = oracle.paper_loss_intensities(rep(I), rep(Igt), np.concatenate([M] * 3, axis=0), lam=0.7)
    assert abs(l6 - l1) < 1e-12 * abs(l1)
    assert np.max(np.abs(g6 - rep(g1) / 6.0)) < 1e-12 * np.max(np.abs(g1))


def test_adan_first_step_and_constant_gradient():
    # step 1: m = g, v = 0, n = g^2, so p moves by lr g / (|g| + eps); with a
    # constant gradient the difference terms vanish and every step does the same
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    p = np.zeros(4)
    m = v = n = np.zeros(4)
    lr, eps = 0.01, 1e-8
    prev = np.zeros(4)
    for step in range(1, 6):
        p_new, m, v, n = oracle.adan_step(p, g, prev, m, v, n, step, lr, eps=eps)
        assert np.allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
        assert np.all(v == 0)
        p, prev = p_new, g


def test_adan_is_invariant_to_the_gradient_scale():
    # without eps the update direction and size do not depend on a positive
    # rescaling of all gradients
    rng = _rng(9)
    gs = [rng.normal(size=6) for _ in range(6)]
    out = []
    for scale in (1.0, 37.0):
        p = np.zeros(6)
        m = v = n = np.zeros(6)
        prev = np.zeros(6)
        for step, g in enumerate(gs, start=1):
            p, m, v, n = oracle.adan_step(p, scale * g, scale * prev, m, v, n, step, 0.01, eps=0.0)
            prev = g
        out.append(p)
    assert np.allclose(out[0], out[1], rtol=1e-12, atol=1e-15)


def test_cosine_schedule_endpoints():
    assert oracle.cosine_lr(0, 100, 0.01, 1e-5) == 0.01
    assert abs(oracle.cosine_lr(100, 100, 0.01, 1e-5) - 1e-5) < 1e-18
    assert abs(oracle.cosine_lr(50, 100, 0.01, 1e-5) - (0.01 + 1e-5) / 2) < 1e-15
    assert oracle.cosine_lr(250, 100, 0.01, 1e-5) == oracle.cosine_lr(100, 100, 0.01, 1e-5)


def test_phase_only_loss_vanishes_at_a_phase_only_target():
    # a unit-amplitude target: the optimum is its own phase, loss and
    # gradient vanish there; elsewhere the gradient matches finite differences
    C, H, W = 1, 14, 18
    z = (1e-3, 4e-3)
    rng = _rng(10)
    phi0 = rng.uniform(0, 2 * np.pi, size=(C, H, W))
    U = oracle.inverse_propagate(np.exp(1j * phi0), PITCH, (515e-9,), z)
    loss, g = oracle.phase_only_loss(U, phi0, PITCH, (515e-9,), z, lam=0.3)
    assert abs(loss) < 1e-12 and np.max(np.abs(g)) < 1e-12
    phi = phi0 + rng.normal(0.0, 0.5, size=phi0.shape)
    loss, g = oracle.phase_only_loss(U, phi, PITCH, (515e-9,), z, lam=0.3)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (0, 7, 9), (0, 13, 17), (0, 3, 12)]:
        pp, pm = phi.copy(), phi.copy()
        pp[c, i, j] += h
        pm[c, i, j] -= h
        fd = (oracle.phase_only_loss(U, pp, PITCH, (515e-9,), z, lam=0.3)[0] -
              oracle.phase_only_loss(U, pm, PITCH, (515e-9,), z, lam=0.3)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) < 1e-6 * max(1.0, abs(fd)), (fd, g[c, i, j])


def test_phase_only_loss_without_ssim_is_the_field_mse():
    C, H, W = 2, 10, 12
    z = (0.0, 2e-3)
    rng = _rng(11)
    P = rng.normal(size=(C, H, W)) + 1j * rng.normal(size=(C, H, W))
    U = oracle.inverse_propagate(P, PITCH, (639e-9, 515e-9), z)
    phi = rng.uniform(0, 2 * np.pi, size=(C, H, W))
    Uphi = oracle.inverse_propagate(np.exp(1j * phi), PITCH, (639e-9, 515e-9), z)
    loss, _ = oracle.phase_only_loss(U, phi, PITCH, (639e-9, 515e-9), z, lam=0.0)
    # mean over the real and imaginary parts = half the mean squared complex distance
    assert abs(loss - 0.5 * np.mean(np.abs(Uphi - U) ** 2)) < 1e-12 * loss
