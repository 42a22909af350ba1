"""Pins for the oracle's band-limited angular spectrum method.

Each check is tied to mathematics that does not come from the oracle itself:
DFT eigenvectors, the analytic Fresnel propagation of a Gaussian beam, energy
conservation, and a brute-force Rayleigh-Sommerfeld convolution (the spatial
kernel whose Fourier transform is the transfer function of Eq.
band_limited_asm_transfer_function, by Weyl's identity).
"""
import math

import numpy as np
import pytest

import oracle

PITCH = 8e-6
LAM = 515e-9


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_fft_matches_naive_dft():
    # numpy's FFT is the library step the oracle relies on; check it against
    # the literal DFT sum on non-power-of-two lengths used by 1080 x 1920.
    rng = np.random.default_rng(0)
    for n in (8, 12, 15, 27, 60, 135):
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        k = np.arange(n)
        D = np.exp(-2j * np.pi * np.outer(k, k) / n)
        assert rel(np.fft.fft(x), D @ x) < 1e-12


def test_frequencies_fft_order():
    f = oracle.frequencies(6, 1.0)
    assert np.allclose(f * 6, [0, 1, 2, -3, -2, -1])
    f = oracle.frequencies(5, 2.0)
    assert np.allclose(f * 10, [0, 1, 2, -2, -1])


def test_transfer_function_values():
    # H at DC is exp(j 2 pi z / lambda); outside the evanescent cut it is 0.
    z = 1e-3
    H = oracle.transfer_function(4, 4, PITCH, LAM, z)
    assert abs(H[0, 0] - np.exp(2j * np.pi * z / LAM)) < 1e-12
    # large pitch-to-wavelength ratio: every bin is propagating, |H| = 1
    assert np.allclose(np.abs(H), 1.0)
    # a pitch below lambda/2 puts the Nyquist bins past 1/lambda: H = 0 there
    Hs = oracle.transfer_function(8, 8, 0.2e-6, LAM, z)
    fx = oracle.frequencies(8, 0.2e-6)
    mask = (fx[None, :] ** 2 + fx[:, None] ** 2) > 1.0 / LAM ** 2
    assert mask.any() and np.all(Hs[mask] == 0)


@pytest.mark.parametrize("k0,m0", [(0, 0), (3, -5), (17, 40), (-64, 1)])
def test_plane_wave_is_eigenvector(k0, m0):
    # P5: exp(j 2 pi (k0 j / W + m0 i / H)) is a DFT eigenvector; ASM scales it
    # by H(f_k0, f_m0) = exp(j 2 pi z sqrt(1/lambda^2 - f^2)).
    Hh, Ww, z = 96, 128, 5e-3
    i = np.arange(Hh)[:, None]
    j = np.arange(Ww)[None, :]
    u = np.exp(2j * np.pi * (k0 * j / Ww + m0 * i / Hh))
    out = oracle.propagate(u, PITCH, LAM, z)
    fx, fy = k0 / (Ww * PITCH), m0 / (Hh * PITCH)
    h = np.exp(2j * np.pi * z * math.sqrt(1 / LAM ** 2 - fx ** 2 - fy ** 2))
    assert rel(out, h * u) < 1e-12


def test_z_zero_is_identity():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(60, 90)) + 1j * rng.normal(size=(60, 90))
    assert rel(oracle.propagate(u, PITCH, LAM, 0.0), u) < 1e-13


def test_parseval_energy():
    # P7: |H| = 1 on the whole grid at these pitches, so energy is conserved.
    rng = np.random.default_rng(2)
    u = rng.normal(size=(64, 80)) + 1j * rng.normal(size=(64, 80))
    out = oracle.propagate(u, PITCH, LAM, 7e-3)
    assert abs(np.linalg.norm(out) / np.linalg.norm(u) - 1) < 1e-12


def test_round_trip():
    # P8: z then -z is the identity inside the propagating band.
    rng = np.random.default_rng(3)
    u = rng.normal(size=(72, 48)) + 1j * rng.normal(size=(72, 48))
    back = oracle.propagate(oracle.propagate(u, PITCH, LAM, 4e-3), PITCH, LAM, -4e-3)
    assert rel(back, u) < 1e-12


@pytest.mark.parametrize("z", [1e-3, 5e-3, 10e-3])
def test_gaussian_beam_fresnel(z):
    # P9: a sampled Gaussian exp(-r^2 / 2 s^2) propagates (paraxially) to
    #   exp(j k z) (s^2 / s_z^2) exp(-r^2 / (2 s_z^2)),  s_z^2 = s^2 + j z / k.
    # The exact ASM differs from the paraxial result by the phase term
    # pi lambda^3 z f^4 / 4 weighted by the spectrum exp(-2 pi^2 s^2 f^2);
    # aliasing and wrap-around are below exp(-80) here.
    n, s_px = 256, 10.0
    s = s_px * PITCH
    k = 2 * np.pi / LAM
    x = (np.arange(n) - n / 2) * PITCH
    X, Y = np.meshgrid(x, x)
    r2 = X ** 2 + Y ** 2
    u0 = np.exp(-r2 / (2 * s ** 2))
    out = oracle.propagate(u0, PITCH, LAM, z)
    sz2 = s ** 2 + 1j * z / k
    ref = np.exp(1j * k * z) * (s ** 2 / sz2) * np.exp(-r2 / (2 * sz2))
    # Predicted size of that difference: the power spectrum exp(-4 pi^2 s^2 f^2)
    # makes f a 2D Gaussian with per-axis variance 1/(8 pi^2 s^2), so
    # f^2 = var * chi2_2 and E[f^8] = 384 var^4; the rms relative error is
    # (pi lambda^3 z / 4) sqrt(384) var^2.
    var = 1.0 / (8 * np.pi ** 2 * s ** 2)
    pred = np.pi * LAM ** 3 * z / 4 * math.sqrt(384.0) * var ** 2
    err = rel(out, ref)
    assert 0.5 * pred < err < 1.5 * pred, (err, pred)
    # a sign mistake in the propagation phase would be far off
    wrong = np.exp(-1j * k * z) * (s ** 2 / np.conj(sz2)) * np.exp(-r2 / (2 * np.conj(sz2)))
    assert rel(out, wrong) > 1e-3


def _rs_brute(u0, pitch, lam, z, out_idx):
    """Direct Rayleigh-Sommerfeld (first kind) sum:
    U(x) = sum_x' u0(x') z e^{jkR} (1 - jkR) / (2 pi R^3) dx^2."""
    n = u0.shape[0]
    k = 2 * np.pi / lam
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    src = u0.ravel()
    ys = ii.ravel() * pitch
    xs = jj.ravel() * pitch
    res = np.zeros(len(out_idx), dtype=np.complex128)
    for t, (i, j) in enumerate(out_idx):
        dx = j * pitch - xs
        dy = i * pitch - ys
        R = np.sqrt(dx * dx + dy * dy + z * z)
        h = z * np.exp(1j * k * R) * (1 - 1j * k * R) / (2 * np.pi * R ** 3)
        res[t] = np.sum(src * h) * pitch * pitch
    return res


def _asm_padded(u0, pitch, lam, z):
    # the oracle's zero-padded mode: the field centred in a 2n x 2n grid of
    # zeros, propagated, and the centre cropped back
    return oracle.propagate(u0, pitch, lam, z, padding=1)


def test_rayleigh_sommerfeld_brute_force():
    # P10: the ASM on a 2x zero-padded grid equals the brute-force RS
    # convolution for a smooth source under the sampling condition
    # r_max / R <= lambda / (2 dx), at two resolutions of the same source.
    z = 50e-3
    errs = []
    for refine in (1, 2):
        n = 32 * refine
        pitch = 16e-6 / refine
        s = 4.0 * 16e-6 / 2  # same physical width at both resolutions
        c = (n - 1) / 2
        i = np.arange(n)
        I, J = np.meshgrid(i, i, indexing="ij")
        u0 = np.exp(-(((I - c) * pitch) ** 2 + ((J - c) * pitch) ** 2) / (2 * s ** 2)).astype(np.complex128)
        asm = _asm_padded(u0, pitch, LAM, z)
        rng = np.random.default_rng(4)
        idx = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(48, 2))]
        idx += [(n // 2, n // 2), (0, 0), (n - 1, n // 3)]
        bf = _rs_brute(u0, pitch, LAM, z, idx)
        a = np.array([asm[p] for p in idx])
        errs.append(rel(a, bf))
    assert max(errs) < 1e-6, errs


def test_adjoint_dot_product():
    # P12: <g, A u> = <A^H g, u> (real part) for the multi-plane propagation.
    rng = np.random.default_rng(5)
    L, C, H, W = 3, 2, 24, 40
    wl, zs = (639e-9, 473e-9), (0.0, 2e-3, 6e-3)
    u = rng.normal(size=(L, C, H, W)) + 1j * rng.normal(size=(L, C, H, W))
    g = rng.normal(size=(C, H, W)) + 1j * rng.normal(size=(C, H, W))
    Au = oracle.propagate_planes(u, PITCH, wl, zs)
    Ag = oracle.propagate_planes_adjoint(g, PITCH, wl, zs)
    lhs = np.sum(np.real(np.conj(g) * Au))
    rhs = np.sum(np.real(np.conj(Ag) * u))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_plane_sum_matches_frequency_domain_sum():
    # Eq. sum_planes taken after each inverse transform equals the sum taken
    # in the frequency domain (linearity); the GPU path uses the latter.
    rng = np.random.default_rng(6)
    L, H, W = 4, 30, 20
    u = rng.normal(size=(L, 1, H, W)) + 1j * rng.normal(size=(L, 1, H, W))
    zs = (0.0, 1e-3, 3e-3, 9e-3)
    P = oracle.propagate_planes(u, PITCH, (LAM,), zs)[0]
    S = sum(oracle.transfer_function(H, W, PITCH, LAM, zs[l]) * np.fft.fft2(u[l, 0]) for l in range(L))
    assert rel(P, np.fft.ifft2(S)) < 1e-13


def test_inverse_propagation_and_loss():
    # plane wave through forward then inverse propagation: |V|^2 is |a|^2;
    # and the loss gradient agrees with central differences.
    Hh, Ww, zs = 16, 24, (0.0, 3e-3)
    i = np.arange(Hh)[:, None]
    j = np.arange(Ww)[None, :]
    a = 0.7 - 0.2j
    P = (a * np.exp(2j * np.pi * (2 * j / Ww - 3 * i / Hh)))[None]
    V = oracle.inverse_propagate(P, PITCH, (LAM,), zs)
    assert np.allclose(np.abs(V) ** 2, abs(a) ** 2, atol=1e-13)
    rng = np.random.default_rng(7)
    P = rng.normal(size=(1, Hh, Ww)) + 1j * rng.normal(size=(1, Hh, Ww))
    Igt = rng.random((2, 1, Hh, Ww))
    loss, gP, _ = oracle.focal_stack_loss(P, Igt, PITCH, (LAM,), zs)
    for (c, y, x) in [(0, 1, 2), (0, 7, 13), (0, 15, 23)]:
        for part in (1.0, 1j):
            h = 1e-6
            Pp = P.copy(); Pp[c, y, x] += h * part
            Pm = P.copy(); Pm[c, y, x] -= h * part
            fd = (oracle.focal_stack_loss(Pp, Igt, PITCH, (LAM,), zs)[0]
                  - oracle.focal_stack_loss(Pm, Igt, PITCH, (LAM,), zs)[0]) / (2 * h)
            an = gP[c, y, x].real if part == 1.0 else gP[c, y, x].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
    # zero field: the loss is the mean of I_gt^2 and the gradient vanishes
    l0, g0, _ = oracle.focal_stack_loss(np.zeros_like(P), Igt, PITCH, (LAM,), zs)
    assert abs(l0 - np.mean(Igt ** 2)) < 1e-15 and np.all(g0 == 0)


def test_fp32_phase_formation_misses_the_bound_at_10mm():
    # Negative control for the precision split of the propagation: at z = 10 mm
    # the phase 2 pi z sqrt(1/lambda^2 - f^2) is ~1.2e5 rad, where FP32 values
    # are 2^-7 rad apart, so a table whose phase is formed in FP32 misses the
    # 1e-4 parity bound; formed in FP64 (reduced mod 2 pi) and only then
    # rounded to complex64, it stays far below it.
    H = W = 128
    z = 10e-3
    rng = np.random.default_rng(7)
    u = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
    ref = oracle.propagate(u, PITCH, LAM, z)
    fx = oracle.frequencies(W, PITCH).astype(np.float32)[None, :]
    fy = oracle.frequencies(H, PITCH).astype(np.float32)[:, None]
    arg32 = np.float32(1.0) / np.float32(LAM) ** 2 - (fx * fx + fy * fy)
    phase32 = np.float32(2.0 * np.pi) * np.float32(z) * np.sqrt(arg32)
    assert phase32.dtype == np.float32 and float(phase32.max()) > 1e5
    h32 = np.exp(1j * phase32.astype(np.float64))
    bad = np.fft.ifft2(h32 * np.fft.fft2(u))
    h64 = oracle.transfer_function(H, W, PITCH, LAM, z).astype(np.complex64).astype(np.complex128)
    good = np.fft.ifft2(h64 * np.fft.fft2(u))
    assert rel(bad, ref) > 1e-3
    assert rel(good, ref) < 1e-6


def test_band_limit_is_the_unaliased_phase_region():
    # band_limit = 1: the kept frequencies are those where the sampled phase
    # of the transfer function does not alias, i.e. where the phase changes
    # by at most pi between neighbouring frequency samples.  The phase
    # increments are computed here numerically from 2 pi z sqrt(1/lambda^2 -
    # f^2) on the sample grid, independently of the limit's closed form; the
    # two may disagree only at the first sample past the boundary.
    n, z = 96, 30e-3
    f = oracle.frequencies(n, PITCH)
    du = 1.0 / (n * PITCH)
    phase = lambda x: 2.0 * np.pi * z * np.sqrt(np.maximum(1.0 / LAM ** 2 - x ** 2, 0.0))
    step = np.abs(phase(f + 0.5 * du) - phase(f - 0.5 * du))
    unaliased = step <= np.pi
    Hb = oracle.transfer_function(1, n, PITCH, LAM, z, band_limit=1)[0]
    kept = np.abs(Hb) > 0
    assert 0 < kept.sum() < n  # the limit is active at this distance and grid
    edge = np.abs(f[kept]).max()
    near_edge = np.abs(np.abs(f) - edge) <= 1.0001 * du
    assert np.all((kept == unaliased) | near_edge)
    assert np.array_equal(kept, np.abs(f) <= edge)  # one contiguous band
    # the kept set is symmetric and inside it the plain transfer function is unchanged
    H0 = oracle.transfer_function(1, n, PITCH, LAM, z, band_limit=0)[0]
    assert np.array_equal(Hb[kept], H0[kept])
    assert np.array_equal(kept, kept[(-np.arange(n)) % n])


def test_band_limit_applies_per_axis():
    # the limit on f_y comes from the grid's own frequency spacing along y:
    # on a 96 x 48 grid the kept f_y (column f_x = 0) are those of a 96-sample
    # axis and the kept f_x (row f_y = 0) those of a 48-sample axis
    z = 30e-3
    Hb = oracle.transfer_function(96, 48, PITCH, LAM, z, band_limit=1)
    ky = np.abs(Hb[:, 0]) > 0
    kx = np.abs(Hb[0, :]) > 0
    assert np.array_equal(ky, np.abs(oracle.transfer_function(1, 96, PITCH, LAM, z, band_limit=1)[0]) > 0)
    assert np.array_equal(kx, np.abs(oracle.transfer_function(1, 48, PITCH, LAM, z, band_limit=1)[0]) > 0)
    assert ky.sum() < 96 and kx.sum() < 48


def test_band_limit_inactive_on_the_paper_shaped_grids():
    # At 8 um pitch the limit lies above the grid's highest frequency for the
    # workloads' sizes and distances, so band_limit = 1 changes nothing there.
    for (H, W, z) in ((1080, 1920, 12e-3), (512, 512, 10e-3), (256, 256, 5e-3)):
        for lam in (639e-9, 515e-9, 473e-9):
            a = oracle.transfer_function(H, W, PITCH, lam, z, band_limit=0)
            b = oracle.transfer_function(H, W, PITCH, lam, z, band_limit=1)
            assert np.array_equal(a, b)


def test_zero_padding_is_the_embedding_done_by_hand():
    # padding = 1 equals propagating an explicit zero embedding on the 2x
    # grid and cropping the window the field occupied (odd sizes included)
    rng = np.random.default_rng(12)
    for H, W in ((16, 24), (15, 9)):
        u = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
        big = np.zeros((2 * H, 2 * W), dtype=np.complex128)
        big[H // 2:H // 2 + H, W // 2:W // 2 + W] = u
        ref = oracle.propagate(big, PITCH, LAM, 3e-3)[H // 2:H // 2 + H, W // 2:W // 2 + W]
        assert np.max(np.abs(oracle.propagate(u, PITCH, LAM, 3e-3, padding=1) - ref)) < 1e-12


def test_zero_padding_removes_the_wrap_around_of_an_edge_source():
    # a smooth source near the left edge (fully inside the grid: a truncated
    # source would radiate outside the band): the padded ASM matches the
    # brute-force (non-periodic) Rayleigh-Sommerfeld sum on both edges, while
    # the circular ASM puts light on the far (right) edge that the
    # non-periodic diffraction integral does not have
    n, pitch, z = 48, 16e-6, 60e-3
    s = 2 * 16e-6
    i = np.arange(n)
    I, J = np.meshgrid(i, i, indexing="ij")
    u0 = np.exp(-(((I - n / 2) * pitch) ** 2 + ((J - 12) * pitch) ** 2) / (2 * s ** 2)).astype(np.complex128)
    idx = [(n // 2, j) for j in (0, 2, 5, 10, n - 6, n - 3, n - 1)]
    bf = _rs_brute(u0, pitch, LAM, z, idx)
    pad = oracle.propagate(u0, pitch, LAM, z, padding=1)
    circ = oracle.propagate(u0, pitch, LAM, z)
    ep = rel(np.array([pad[p] for p in idx]), bf)
    ec = rel(np.array([circ[p] for p in idx]), bf)
    assert ep < 1e-6 and ec > 0.1, (ep, ec)


@pytest.mark.parametrize("band_limit", [0, 1])
def test_adjoint_dot_product_zero_padded(band_limit):
    rng = np.random.default_rng(13)
    L, C, H, W = 2, 2, 12, 20
    wl, zs = (639e-9, 473e-9), (1e-3, 6e-3)
    u = rng.normal(size=(L, C, H, W)) + 1j * rng.normal(size=(L, C, H, W))
    g = rng.normal(size=(C, H, W)) + 1j * rng.normal(size=(C, H, W))
    Au = oracle.propagate_planes(u, PITCH, wl, zs, band_limit, padding=1)
    Ag = oracle.propagate_planes_adjoint(g, PITCH, wl, zs, band_limit, padding=1)
    assert abs(np.sum(np.real(np.conj(g) * Au)) - np.sum(np.real(np.conj(Ag) * u))) < 1e-10 * np.sum(np.abs(g * Au))
    # and the inverse propagation against its adjoint
    P = rng.normal(size=(C, H, W)) + 1j * rng.normal(size=(C, H, W))
    gV = rng.normal(size=(L, C, H, W)) + 1j * rng.normal(size=(L, C, H, W))
    V = oracle.inverse_propagate(P, PITCH, wl, zs, band_limit, padding=1)
    gP = oracle.inverse_propagate_adjoint(gV, PITCH, wl, zs, band_limit, padding=1)
    assert abs(np.sum(np.real(np.conj(gV) * V)) - np.sum(np.real(np.conj(gP) * P))) < 1e-10 * np.sum(np.abs(gV * V))
