"""Pins for the dense plane-weight gradient (the rho_grad = 1 mode).

The dense gradient is dL/drho_{n,l} of the compositing with continuous plane
weights (alpha_eff = alpha rho_l) at the one-hot weights of the argmax planes.
The soft compositing is pinned to the hard one at one-hot weights, and the
dense gradient to central finite differences of the soft compositing in each
unassigned plane weight; the straight-through rule then maps it to the logits.
"""
import numpy as np

import hcgs_synth as S
import oracle

OPTS = dict(oracle.DEFAULT_OPTS)


def _setup(N=24, L=3, C=2, H=28, W=36, seed=0, ls=-1.7):
    g = S.make_gaussians(N, L, C, H, W, seed=seed, log_scale_mean=ls, log_scale_std=0.3)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    g["means"][:, 2] += 1.0
    # spread the plane assignments so that every plane has Gaussians
    g["plane_logits"] = np.random.default_rng(seed).normal(size=(N, L))
    vm, it = S.view_batch(1, H, W, seed=seed)
    pr = oracle.project(g, vm[0], it[0], H, W, OPTS)
    gU = S.random_complex((L, C, H, W), seed=3).astype(np.complex128)
    return g, pr, gU


def _onehot(pr):
    rho = np.zeros((pr["N"], pr["L"]))
    rho[np.arange(pr["N"]), pr["plane"]] = 1.0
    return rho


def test_soft_compositing_at_one_hot_weights_is_the_hard_one():
    g, pr, _ = _setup()
    U, T, _ = oracle.composite(pr, OPTS)
    Us, Ts = oracle.composite_soft(pr, _onehot(pr), OPTS)
    assert np.max(np.abs(U - Us)) < 1e-14 and np.max(np.abs(T - Ts)) < 1e-14


def test_dense_gradient_matches_finite_differences():
    g, pr, gU = _setup()
    d = oracle.composite_rho_dense(pr, gU, OPTS)
    rho0 = _onehot(pr)

    def loss(rho):
        U, _ = oracle.composite_soft(pr, rho, OPTS)
        return float(np.sum(np.real(np.conj(gU) * U)))

    # the assigned plane's entry is zero; pick unassigned ones with the largest values
    assert np.all(d[rho0 == 1] == 0)
    cand = [(n, l) for n in range(pr["N"]) for l in range(pr["L"]) if rho0[n, l] == 0 and pr["valid"][n]]
    cand.sort(key=lambda t: -abs(d[t]))
    assert abs(d[cand[0]]) > 1e-3
    h = 1e-6
    for (n, l) in cand[:8] + cand[-2:]:
        rp, rm = rho0.copy(), rho0.copy()
        rp[n, l] += h
        rm[n, l] -= h
        fd = (loss(rp) - loss(rm)) / (2 * h)
        assert abs(fd - d[n, l]) < 1e-6 * max(1.0, abs(fd)), (n, l, fd, d[n, l])


def test_ste_weights_are_the_tempered_softmax():
    # the straight-through weights of the dense mode: softmax(rho' / tau) per
    # Gaussian, against scipy's softmax
    from scipy.special import softmax
    r = np.random.default_rng(3).normal(size=(7, 5))
    for tau in (1e-3, 0.5, 2.0):
        assert np.allclose(oracle.ste_softmax(r, tau), softmax(r / tau, axis=1), rtol=1e-12, atol=1e-300)


def test_dense_mode_adds_the_unassigned_planes_to_the_logits():
    g, pr, gU = _setup(seed=1)
    optics = S.Optics(28, 36, (639e-9, 473e-9), (0.0, 3e-3, 6e-3))
    vm, it = S.view_batch(1, 28, 36, seed=1)
    gP = S.random_complex((1, 2, 28, 36), seed=2).astype(np.complex128)
    # a larger temperature so that the unassigned logits carry weight
    opts = dict(OPTS, tau=2.0)
    sparse = oracle.render_backward(g, vm, it, optics, gP, opts)
    dense = oracle.render_backward(g, vm, it, optics, gP, opts, rho_grad=1)
    for k in oracle.PARAM_NAMES:
        if k != "plane_logits":
            assert np.allclose(sparse[k], dense[k], rtol=1e-12, atol=1e-15)  # (atomic sums: order may differ)
    pr1 = oracle.project(g, vm[0], it[0], 28, 36, opts)
    gU1 = oracle.propagate_planes_adjoint(gP[0], optics.pitch, optics.wavelengths, optics.plane_z)
    want = sparse["plane_logits"] + oracle.composite_rho_dense(pr1, gU1, opts) * oracle.ste_softmax(
        g["plane_logits"], 2.0)
    assert np.allclose(dense["plane_logits"], want, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(dense["plane_logits"] - sparse["plane_logits"])) > 1e-6
