"""GPU parity of the phase-only hologram conversion (Sec. 6) against the FP64
oracle: the objective and its phase gradient (circular and zero-padded, with
the band limit), the phase <-> hologram helpers, and a conversion run on a
rendered hologram."""
import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import cams, cams_dev, complex_dev, dev, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("B,H,W,C,L,bl,pad,lam", [(2, 64, 80, 2, 3, 0, 0, 0.005), (1, 45, 96, 1, 2, 1, 1, 0.5),
                                                  (1, 256, 256, 3, 2, 0, 0, 0.0)])
def test_phase_only_loss_and_gradient(P, ctx, B, H, W, C, L, bl, pad, lam):
    o = S.Optics(H, W, S.WAVELENGTHS_RGB[:C], tuple(float(z) for z in np.linspace(0.0, 6e-3, L)),
                 band_limit=bl, padding=pad)
    Pn = S.random_complex((B, C, H, W), seed=3)
    phase = S.random_real((B, C, H, W), seed=4, lo=-np.pi, hi=np.pi)
    U = torch.empty((B, L, C, H, W), dtype=torch.complex64, device="cuda")
    ctx.asm_propagate(complex_dev(Pn), B, o, -1, 0, U)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.empty((B, C, H, W), dtype=torch.float32, device="cuda")
    ctx.phase_only_loss(U, torch.from_numpy(phase).cuda(), B, o, loss, g, lambda_ssim=lam)
    Uh = U.cpu().numpy().astype(np.complex128)
    refs = [oracle.phase_only_loss(Uh[b], phase[b].astype(np.float64), o.pitch, o.wavelengths, o.plane_z, lam, bl,
                                   pad) for b in range(B)]
    l_ref = float(np.mean([r[0] for r in refs]))
    g_ref = np.stack([r[1] / B for r in refs])
    assert abs(float(loss.item()) - l_ref) < 1e-5 * abs(l_ref) + 4e-7 * lam, (float(loss.item()), l_ref)
    assert rel(g.cpu().numpy(), g_ref) < 1e-4


def test_phase_helpers(P, ctx):
    Pn = S.random_complex((3, 17, 29), seed=5)
    ph = torch.empty((3, 17, 29), dtype=torch.float32, device="cuda")
    ctx.hologram_phase(complex_dev(Pn), ph)
    assert np.max(np.abs(ph.cpu().numpy() - np.angle(Pn.astype(np.complex128)))) < 1e-6
    h = torch.empty((3, 17, 29), dtype=torch.complex64, device="cuda")
    ctx.phase_hologram(ph, h)
    assert np.max(np.abs(h.cpu().numpy() - np.exp(1j * ph.cpu().numpy().astype(np.float64)))) < 1e-6


def test_conversion_of_a_rendered_hologram(P, ctx):
    # With a propagation that is unitary inside the band, the field error
    # summed over the planes is L times the error on the hologram plane, which
    # the complex hologram's own phase minimises pixel by pixel: from that
    # start the optimisation only refines (SSIM term, band edges); from
    # uniform random phases it must find its way to the same level.
    from paper_2506_08350_b300.phase_only import convert
    o = S.Optics(256, 256, S.WAVELENGTHS_RGB, (0.0, 2e-3, 4e-3, 6e-3))
    g = S.make_gaussians(20_000, o.L, o.C, o.H, o.W, seed=1)
    vm, it = cams(1, o.H, o.W, seed=0)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    ctx.render_view(dev(g), vmd, itd, o, P.DEFAULT_OPTS, holo)
    _, rep_h = convert(ctx, holo, o, steps=100)
    phase, rep_r = convert(ctx, holo, o, steps=600, lr=0.05, init="random")
    print("phase-only conversion from the hologram's phase:", rep_h)
    print("phase-only conversion from random phases:", rep_r)
    assert phase.shape == (1, o.C, o.H, o.W)
    assert rep_h["loss_end"] <= rep_h["loss_start"] * (1 + 1e-6)
    assert rep_r["loss_end"] < 0.5 * rep_r["loss_start"], rep_r
    assert rep_r["loss_end"] < 1.25 * rep_h["loss_end"], (rep_r, rep_h)
    assert rep_r["psnr_end"] > rep_r["psnr_start"] + 3.0, rep_r
