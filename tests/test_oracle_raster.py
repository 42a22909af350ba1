"""Pins for the oracle's projection and complex per-plane compositing.

Closed forms (single Gaussian footprints, a hand-derived three-Gaussian
pixel), library routines (scipy's quaternion rotation, a numerical Jacobian of
the pinhole map), an independent textbook alpha blend (Eq. gaussian_blending)
and invariants stated by the paper (each Gaussian only reaches its own plane;
L = 1 puts every Gaussian on the single plane).
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import hcgs_synth as S
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one(mean, log_s, quat, o, amp, phase, plane_logits):
    f32 = lambda x: np.asarray(x, dtype=np.float64)[None]
    return dict(means=f32(mean), log_scales=f32(log_s), quats=f32(quat),
                opacity_logits=np.array([math.log(o / (1 - o))]), amplitude=f32(amp),
                phase=f32(phase), plane_logits=f32(plane_logits))


def _cat(gs):
    return {k: np.concatenate([g[k] for g in gs], axis=0) for k in gs[0]}


def test_single_gaussian_closed_form():
    # P1: axis-aligned Gaussian on the optical axis at depth z: Sigma' =
    # (f/z)^2 diag(s_x^2, s_y^2); U = c o exp(-1/2 d^T Sigma'^-1 d) e^{j phi}
    # on the assigned plane, zero on the other plane.
    H, W, f, z = 40, 48, 500.0, 2.0
    intr = np.array([f, f, 23.5, 19.5])
    sx, sy = 0.01, 0.02
    g = _one([0, 0, z], np.log([sx, sy, 0.015]), [1, 0, 0, 0], 0.7, [0.8, 0.3], [1.0, 4.0], [0.0, 1.0])
    pr = oracle.project(g, np.eye(4), intr, H, W, oracle.EXACT_OPTS)
    U, T, nc = oracle.composite(pr, oracle.EXACT_OPTS)
    a, b = (f / z * sx) ** 2, (f / z * sy) ** 2
    i = np.arange(H)[:, None] - 19.5
    j = np.arange(W)[None, :] - 23.5
    G = np.exp(-0.5 * (j ** 2 / a + i ** 2 / b))
    for c, (amp, ph) in enumerate([(0.8, 1.0), (0.3, 4.0)]):
        assert np.max(np.abs(U[1, c] - amp * 0.7 * G * np.exp(1j * ph))) < 1e-14
        assert np.all(U[0, c] == 0)
    assert np.max(np.abs(T[1] - (1 - 0.7 * G))) < 1e-14
    assert np.all(T[0] == 1)


def test_rotated_gaussian_closed_form():
    # rotation about the optical axis by theta: Sigma' = (f/z)^2 R2 diag(s^2) R2^T.
    H, W, f, z, th = 36, 36, 400.0, 1.5, 0.6
    intr = np.array([f, f, 17.0, 18.0])
    sx, sy = 0.012, 0.004
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    g = _one([0, 0, z], np.log([sx, sy, 0.01]), q, 0.9, [1.0], [0.0], [0.0])
    pr = oracle.project(g, np.eye(4), intr, H, W, oracle.EXACT_OPTS)
    R2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Sig = (f / z) ** 2 * R2 @ np.diag([sx ** 2, sy ** 2]) @ R2.T
    assert np.allclose(pr["cov"][0], [Sig[0, 0], Sig[0, 1], Sig[1, 1]], rtol=1e-13)
    K = np.linalg.inv(Sig)
    assert np.allclose(pr["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-12)
    U, _, _ = oracle.composite(pr, oracle.EXACT_OPTS)
    i = np.arange(H)[:, None] - 18.0
    j = np.arange(W)[None, :] - 17.0
    G = np.exp(-0.5 * (K[0, 0] * j ** 2 + 2 * K[0, 1] * i * j + K[1, 1] * i ** 2))
    assert np.max(np.abs(U[0, 0] - 0.9 * G)) < 1e-14


def test_projection_matches_numerical_jacobian():
    # Eq. gaussian_projection for an off-axis Gaussian seen by a rotated,
    # translated camera: Sigma' = J W Sigma W^T J^T with J the Jacobian of the
    # pinhole map (here taken by central differences), Sigma from scipy's
    # quaternion rotation, and mu the pinhole image of the mean.
    rng = np.random.default_rng(0)
    H, W = 60, 80
    intr = np.array([70.0, 75.0, 39.5, 29.5])
    M = S.look_at([0.3, -0.2, -0.5], [0.1, 0.2, 2.0])
    for _ in range(5):
        mean = np.array([rng.normal() * 0.3, rng.normal() * 0.3, 2.0 + rng.random()])
        log_s = np.log(0.02 + 0.05 * rng.random(3))
        q = rng.normal(size=4)
        g = _one(mean, log_s, q, 0.5, [1.0], [0.0], [0.0])
        pr = oracle.project(g, M, intr, H, W, oracle.EXACT_OPTS)

        def pin(x):
            t = M[:3, :3] @ x + M[:3, 3]
            return np.array([intr[0] * t[0] / t[2] + intr[2], intr[1] * t[1] / t[2] + intr[3]])

        Jn = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            Jn[:, k] = (pin(mean + e) - pin(mean - e)) / 2e-6
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig3 = Rm @ np.diag(np.exp(2 * log_s)) @ Rm.T
        Sig2 = Jn @ Sig3 @ Jn.T
        assert np.allclose(pr["mu"][0], pin(mean), rtol=1e-12)
        assert np.allclose(pr["cov"][0], [Sig2[0, 0], Sig2[0, 1], Sig2[1, 1]], rtol=1e-7)
        assert abs(pr["depth"][0] - (M[:3, :3] @ mean + M[:3, 3])[2]) < 1e-14


def test_dilation_adds_to_the_2d_covariance():
    # The 2D covariance gets + dilation * I (the low-pass the 3DGS rasterizer
    # applies); the projected mean is untouched.
    H, W = 40, 48
    intr = np.array([300.0, 320.0, 23.5, 19.5])
    g = _one([0.05, -0.03, 2.0], np.log([0.01, 0.02, 0.015]), [0.9, 0.1, -0.3, 0.2], 0.6, [1.0], [0.0], [0.0])
    ex = oracle.project(g, np.eye(4), intr, H, W, oracle.EXACT_OPTS)
    pr = oracle.project(g, np.eye(4), intr, H, W, dict(oracle.EXACT_OPTS, dilation=0.3))
    assert np.allclose(pr["cov"][0] - ex["cov"][0], [0.3, 0.0, 0.3], rtol=0, atol=1e-12)
    assert np.array_equal(pr["mu"][0], ex["mu"][0])


def test_jacobian_clamp_closed_form():
    # Beyond clip * tan(half field of view) the Jacobian of the pinhole map is
    # taken at the clamped position t'_x = lim t_z, so the footprint of an
    # axis-aligned Gaussian far off-axis is J' diag(s^2) J'^T with
    # J' = [[f/z, 0, -f lim / z], [0, f/z, 0]]; the mean still projects exactly.
    H, W, f = 40, 60, 100.0
    intr = np.array([f, f, 29.5, 19.5])
    z, x = 2.0, 1.5                      # x / z = 0.75 beyond lim = 1.3 * 30 / 100 = 0.39
    s = np.array([0.03, 0.02, 0.01])
    g = _one([x, 0.0, z], np.log(s), [1, 0, 0, 0], 0.5, [1.0], [0.0], [0.0])
    pr = oracle.project(g, np.eye(4), intr, H, W, dict(oracle.EXACT_OPTS, clip=1.3))
    lim = 1.3 * (W / 2) / f
    J = np.array([[f / z, 0.0, -f * lim / z], [0.0, f / z, 0.0]])
    Sig = J @ np.diag(s ** 2) @ J.T
    assert np.allclose(pr["cov"][0], [Sig[0, 0], Sig[0, 1], Sig[1, 1]], rtol=1e-12)
    assert abs(pr["mu"][0][0] - (f * x / z + 29.5)) < 1e-12


def test_alpha_max_clamp_and_its_flat_adjoint():
    # alpha = min(alpha_max, o G): a near-opaque Gaussian is clamped around its
    # centre, where the field is c alpha_max e^{j phi}; there alpha does not
    # depend on o or mu, so the adjoint (checked against central differences
    # of the compositing) takes nothing from those pixels.
    H, W, f, z = 24, 28, 300.0, 2.0
    intr = np.array([f, f, 14.0, 11.0])  # the centre falls on pixel (14, 11)
    g = _one([0, 0, z], np.log([0.05, 0.06, 0.02]), [1, 0, 0, 0], 0.999, [0.8], [0.5], [0.0])
    opts = dict(oracle.EXACT_OPTS, alpha_max=0.99)
    pr = oracle.project(g, np.eye(4), intr, H, W, opts)
    U, _, _ = oracle.composite(pr, opts)
    a, b = (f / z * 0.05) ** 2, (f / z * 0.06) ** 2
    i = np.arange(H)[:, None] - 11.0
    j = np.arange(W)[None, :] - 14.0
    G = np.exp(-0.5 * (j ** 2 / a + i ** 2 / b))
    assert np.sum(0.999 * G > 0.99) >= 4  # the clamp is active at some pixels
    assert np.max(np.abs(U[0, 0] - 0.8 * np.minimum(0.99, 0.999 * G) * np.exp(0.5j))) < 1e-14
    gU = S.random_complex(U.shape, seed=4).astype(np.complex128)
    g2 = oracle.composite_backward(pr, gU, opts)

    def loss(key, idx, d):
        p2 = dict(pr)
        p2[key] = pr[key].copy()
        p2[key][idx] += d
        U2, _, _ = oracle.composite(p2, opts)
        return float(np.sum(np.real(np.conj(gU) * U2)))

    h = 1e-7
    for key, idx in (("opac", (0,)), ("mu", (0, 0)), ("mu", (0, 1))):
        fd = (loss(key, idx, h) - loss(key, idx, -h)) / (2 * h)
        assert abs(fd - g2[key][idx]) < 1e-6 * max(1.0, abs(fd)), (key, idx, fd, g2[key][idx])


def test_near_plane_cull():
    # a Gaussian whose camera-space depth is below near_z is culled (it
    # contributes nothing); one just beyond it is projected
    H, W = 16, 16
    intr = np.array([100.0, 100.0, 7.5, 7.5])
    g = _cat([_one([0, 0, 0.15], np.log([0.01] * 3), [1, 0, 0, 0], 0.5, [1.0], [0.0], [0.0]),
              _one([0, 0, 0.25], np.log([0.01] * 3), [1, 0, 0, 0], 0.5, [1.0], [0.0], [0.0])])
    pr = oracle.project(g, np.eye(4), intr, H, W, dict(oracle.EXACT_OPTS, near_z=0.2))
    assert list(pr["valid"]) == [0, 1]
    pr = oracle.project(g, np.eye(4), intr, H, W, dict(oracle.EXACT_OPTS, near_z=0.1))
    assert list(pr["valid"]) == [1, 1]


def test_stop_rule_in_the_adjoint():
    # six Gaussians stacked on the optical axis, o = 0.9 each: at the centre
    # pixel T falls to 1e-5 after the fifth, which stops the walk (T_eps =
    # 1e-4, after the add); the sixth never contributes there.  U is linear in
    # w, so the adjoint's dL/dw must equal the central differences exactly:
    # the fifth Gaussian's is nonzero at the centre, the sixth's only from
    # the pixels its neighbours leave open.
    H, W = 9, 9
    intr = np.array([100.0, 100.0, 4.0, 4.0])
    g = _cat([_one([0, 0, 1.0 + 0.1 * k], np.log([0.01] * 3), [1, 0, 0, 0], 0.9, [0.5 + 0.1 * k], [0.3 * k], [0.0])
              for k in range(6)])
    opts = dict(oracle.EXACT_OPTS, T_eps=1e-4)
    pr = oracle.project(g, np.eye(4), intr, H, W, opts)
    U, T, nc = oracle.composite(pr, opts)
    assert nc[0, 4, 4] == 5 and T[0, 4, 4] < 1e-4
    gU = S.random_complex(U.shape, seed=6).astype(np.complex128)
    g2 = oracle.composite_backward(pr, gU, opts)

    def loss(n, part, d):
        p2 = dict(pr)
        p2["w"] = pr["w"].copy()
        p2["w"][n, 0, part] += d
        U2, _, _ = oracle.composite(p2, opts)
        return float(np.sum(np.real(np.conj(gU) * U2)))

    for n in range(6):
        for part in (0, 1):
            fd = (loss(n, part, 1e-6) - loss(n, part, -1e-6)) / 2e-6
            assert abs(fd - g2["w"][n, 0, part]) < 1e-8 * max(1.0, abs(fd)), (n, part, fd, g2["w"][n, 0, part])


def test_equal_depths_visit_in_index_order():
    # Reading R1: the visiting order is (depth, index) ascending front to back
    # and its exact reverse back to front.  Two Gaussians at the same depth on
    # the same pixel: U = w_a alpha_a + w_b alpha_b (1 - alpha_a) with a the
    # one visited first.
    H, W = 9, 9
    intr = np.array([100.0, 100.0, 4.0, 4.0])
    g = _cat([_one([0, 0, 1.5], np.log([0.01] * 3), [1, 0, 0, 0], 0.6, [1.0], [0.0], [0.0]),
              _one([0, 0, 1.5], np.log([0.01] * 3), [1, 0, 0, 0], 0.3, [0.5], [np.pi / 2], [0.0])])
    w0, w1 = 1.0, 0.5j
    for order, (first, second) in ((0, ((w0, 0.6), (w1, 0.3))), (1, ((w1, 0.3), (w0, 0.6)))):
        opts = dict(oracle.EXACT_OPTS, order=order)
        U, _, _ = oracle.composite(oracle.project(g, np.eye(4), intr, H, W, opts), opts)
        want = first[0] * first[1] + second[0] * second[1] * (1 - first[1])
        assert abs(U[0, 0, 4, 4] - want) < 1e-12, (order, U[0, 0, 4, 4], want)


def test_depth_key_is_rounded_once_to_fp32():
    # Reading R14: the visiting order compares the camera-space depth rounded
    # to FP32, ties by index.  Gaussian 0 sits 2e-8 m behind Gaussian 1 at
    # 1.5 m (FP32 spacing there 1.2e-7 m): equal keys, so index order, 0
    # first.  5e-7 m behind (four FP32 steps): depth order, 1 first.
    H, W = 9, 9
    intr = np.array([100.0, 100.0, 4.0, 4.0])
    opts = dict(oracle.EXACT_OPTS, order=0)
    for dz, first_is_0 in ((2e-8, True), (5e-7, False)):
        g = _cat([_one([0, 0, 1.5 + dz], np.log([0.01] * 3), [1, 0, 0, 0], 0.6, [1.0], [0.0], [0.0]),
                  _one([0, 0, 1.5], np.log([0.01] * 3), [1, 0, 0, 0], 0.3, [0.5], [np.pi / 2], [0.0])])
        pr = oracle.project(g, np.eye(4), intr, H, W, opts)
        U, _, _ = oracle.composite(pr, opts)
        (wa, aa), (wb, ab) = ((1.0, 0.6), (0.5j, 0.3)) if first_is_0 else ((0.5j, 0.3), (1.0, 0.6))
        want = wa * aa + wb * ab * (1 - aa)
        assert abs(U[0, 0, 4, 4] - want) < 1e-9, (dz, U[0, 0, 4, 4], want)
        assert list(oracle.visiting_order(pr)) == ([0, 1] if first_is_0 else [1, 0])


def _golden():
    gs, ex = [], []
    with open(os.path.join(GOLDEN, "three_gaussians_one_pixel.txt")) as fh:
        for line in fh:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "gaussian":
                gs.append(tuple(float(v) for v in p[1:]))
            elif p[0] == "expect":
                ex.append((int(p[1]), complex(float(p[2]), float(p[3])), float(p[4])))
    return gs, ex


def test_three_gaussians_golden_fixture():
    # P2: hand-derived values in tests/golden/three_gaussians_one_pixel.txt.
    gs, ex = _golden()
    H, W = 30, 40
    intr = np.array([100.0, 100.0, 20.0, 15.0])  # mu lands exactly on pixel (15, 20)
    g = _cat([_one([0, 0, d], np.log([0.01, 0.01, 0.01]), [1, 0, 0, 0], o, [a], [ph * np.pi], [0.0])
              for d, o, a, ph in gs])
    for order, U_exp, T_exp in ex:
        opts = dict(oracle.EXACT_OPTS, order=order)
        pr = oracle.project(g, np.eye(4), intr, H, W, opts)
        U, T, nc = oracle.composite(pr, opts)
        assert abs(U[0, 0, 15, 20] - U_exp) < 1e-12
        assert abs(T[0, 15, 20] - T_exp) < 1e-12
        assert nc[0, 15, 20] == 3


def test_thresholds_alpha_min_and_stop_after_add():
    # Algorithm 2: a Gaussian with alpha < alpha_min is skipped; the walk stops
    # once T < T_eps, after the Gaussian that crossed the threshold has added.
    H, W = 10, 10
    intr = np.array([100.0, 100.0, 5.0, 5.0])
    g = _cat([_one([0, 0, 1.0], np.log([0.01] * 3), [1, 0, 0, 0], 0.003, [5.0], [0.0], [0.0]),
              _one([0, 0, 1.5], np.log([0.01] * 3), [1, 0, 0, 0], 0.99995, [1.0], [0.0], [0.0]),
              _one([0, 0, 2.0], np.log([0.01] * 3), [1, 0, 0, 0], 0.5, [1.0], [np.pi / 2], [0.0])])
    base = dict(oracle.EXACT_OPTS, alpha_min=1 / 255, alpha_max=1.0)
    pr = oracle.project(g, np.eye(4), intr, H, W, dict(base, T_eps=1e-4))
    U, T, nc = oracle.composite(pr, dict(base, T_eps=1e-4))
    assert abs(U[0, 0, 5, 5] - 0.99995) < 1e-12 and nc[0, 5, 5] == 1
    U, T, nc = oracle.composite(pr, dict(base, T_eps=1e-5))
    assert abs(U[0, 0, 5, 5] - (0.99995 + 0.5j * 5e-5)) < 1e-12 and nc[0, 5, 5] == 2
    ex = dict(oracle.EXACT_OPTS, T_eps=1e-5)
    U, T, nc = oracle.composite(oracle.project(g, np.eye(4), intr, H, W, ex), ex)
    assert abs(U[0, 0, 5, 5] - (0.003 * 5 + 0.99995 * 0.997 + 0.5j * 0.997 * 5e-5)) < 1e-12


def _scene(N=40, L=2, C=2, H=32, W=40, seed=0, ls=-1.8):
    g = S.make_gaussians(N, L, C, H, W, seed=seed, log_scale_mean=ls, log_scale_std=0.3)
    return {k: v.astype(np.float64) for k, v in g.items()}, S.intrinsics(H, W)


def test_weights_sum_to_one_minus_T():
    # With w = 1 for every Gaussian, U = sum alpha_n T_n = 1 - T_final exactly.
    g, intr = _scene(N=60, L=3, C=1)
    g["amplitude"][:] = 1.0
    g["phase"][:] = 0.0
    pr = oracle.project(g, np.eye(4), intr, 32, 40)
    U, T, _ = oracle.composite(pr)
    assert np.max(np.abs(U[:, 0] - (1 - T))) < 1e-13


def test_plane_independence_and_single_plane():
    # Each Gaussian contributes only to its assigned plane (Sec. 4.1): moving
    # one Gaussian to another plane changes only those two planes.
    g, intr = _scene(N=50, L=4, C=1)
    pr = oracle.project(g, np.eye(4), intr, 32, 40)
    U0, _, _ = oracle.composite(pr)
    n = int(np.argmax(pr["opac"] * (pr["valid"] > 0)))
    src = int(pr["plane"][n])
    dst = (src + 1) % 4
    g2 = {k: v.copy() for k, v in g.items()}
    g2["plane_logits"][n] = -100.0
    g2["plane_logits"][n, dst] = 100.0
    U1, _, _ = oracle.composite(oracle.project(g2, np.eye(4), intr, 32, 40))
    for l in range(4):
        same = np.array_equal(U0[l], U1[l])
        assert same == (l not in (src, dst))
    # L = 1: rho = 1 for all (Eq. hard_assignment); equals putting every
    # Gaussian on plane 0 of an L = 4 scene.
    g1 = {k: v.copy() for k, v in g.items()}
    g1["plane_logits"] = np.zeros((50, 1))
    g4 = {k: v.copy() for k, v in g.items()}
    g4["plane_logits"] = np.tile([1.0, 0.0, 0.0, 0.0], (50, 1))
    Ua, _, _ = oracle.composite(oracle.project(g1, np.eye(4), intr, 32, 40))
    Ub, _, _ = oracle.composite(oracle.project(g4, np.eye(4), intr, 32, 40))
    assert np.array_equal(Ua[0], Ub[0]) and np.all(Ub[1:] == 0)


def test_permutation_invariance():
    g, intr = _scene(N=70, L=2, C=2, seed=3)
    perm = np.random.default_rng(1).permutation(70)
    gp = {k: v[perm] for k, v in g.items()}
    U0, T0, _ = oracle.composite(oracle.project(g, np.eye(4), intr, 32, 40))
    U1, T1, _ = oracle.composite(oracle.project(gp, np.eye(4), intr, 32, 40))
    assert np.array_equal(U0, U1) and np.array_equal(T0, T1)


def test_reduces_to_textbook_alpha_blending():
    # P4: phase 0, amplitude = colour, L = 1: Re U is the 3DGS colour blend of
    # Eq. gaussian_blending.  The blend below is written independently: per
    # pixel, sort by depth and accumulate c alpha T with the same thresholds.
    H, W = 20, 24
    g, intr = _scene(N=25, L=1, C=3, H=H, W=W, seed=5)
    g["phase"][:] = 0.0
    opts = dict(oracle.DEFAULT_OPTS)
    pr = oracle.project(g, np.eye(4), intr, H, W, opts)
    U, _, _ = oracle.composite(pr, opts)
    order = sorted([n for n in range(25) if pr["valid"][n]], key=lambda n: (pr["depth"][n], n))
    ref = np.zeros((3, H, W))
    for i in range(H):
        for j in range(W):
            T, col = 1.0, np.zeros(3)
            for n in order:
                A, B, Cc = pr["conic"][n]
                dx, dy = j - pr["mu"][n][0], i - pr["mu"][n][1]
                a = min(0.99, pr["opac"][n] * math.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + Cc * dy * dy)))
                if a < 1 / 255:
                    continue
                col += g["amplitude"][n] * a * T
                T *= 1 - a
                if T < 1e-4:
                    break
            ref[:, i, j] = col
    assert np.max(np.abs(U[0].real - ref)) < 1e-13
    assert np.max(np.abs(U[0].imag)) < 1e-15


def test_superposition_without_overlap():
    # P11: when no two Gaussians overlap on a plane (T = 1 on every support),
    # the hologram is the sum over Gaussians of IDFT(H_{Z_l(n)} DFT(U_n)),
    # each Gaussian rendered alone (the per-primitive sum of Sec. 5.2).
    H, W = 48, 64
    intr = np.array([300.0, 300.0, 31.5, 23.5])
    gs = []
    for k, (x, y, pl) in enumerate([(-0.15, -0.1, 0), (0.1, -0.1, 1), (-0.1, 0.1, 1), (0.15, 0.08, 0)]):
        gs.append(_one([x, y, 2.0 + 0.1 * k], np.log([0.006, 0.004, 0.005]), [1, 0.2 * k, 0, 0.1], 0.6,
                       [0.5 + 0.1 * k, 1.0], [0.7 * k, 2.0], [1.0 - pl, float(pl)]))
    opts = dict(oracle.DEFAULT_OPTS)
    optics = S.Optics(H, W, (639e-9, 473e-9), (1e-3, 4e-3))
    P, U, _, _ = oracle.render(_cat(gs), np.eye(4)[None], intr[None], optics, opts)
    acc = np.zeros_like(P[0])
    for gg in gs:
        Pn, _, _, _ = oracle.render(gg, np.eye(4)[None], intr[None], optics, opts)
        acc += Pn[0]
    assert np.linalg.norm(P[0] - acc) < 1e-12 * np.linalg.norm(acc)
