"""GPU parity of the zero-padded (linear-convolution) propagation against the
FP64 oracle: forward recording, inverse propagation and both adjoints, with
and without the band limit; the render path and the two losses on padded
optics; and the size checks of the padded grid."""
import dataclasses

import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import cams, cams_dev, complex_dev, dev, oracle_opts, rel

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


# padded grids: 2H x 2W = 128 x 160, 90 x 192 (odd half-offsets: H = 45), 1024 x 1024
@pytest.mark.parametrize("H,W,L,C,B,bl", [(64, 80, 2, 2, 1, 0), (45, 96, 3, 1, 2, 1), (512, 512, 2, 1, 1, 0),
                                          (64, 80, 2, 2, 1, 1)])
def test_padded_asm_all_directions(P, ctx, H, W, L, C, B, bl):
    wl = S.WAVELENGTHS_RGB[:C]
    z = tuple(float(v) for v in np.linspace(1e-3, 20e-3, L))
    o = S.Optics(H, W, wl, z, band_limit=bl, padding=1)
    U = S.random_complex((B, L, C, H, W), seed=1)
    Pn = S.random_complex((B, C, H, W), seed=2)
    out = torch.empty((B, C, H, W), dtype=torch.complex64, device="cuda")
    ctx.asm_propagate(complex_dev(U), B, o, 1, 1, out)
    inv = torch.empty((B, L, C, H, W), dtype=torch.complex64, device="cuda")
    ctx.asm_propagate(complex_dev(Pn), B, o, -1, 0, inv)
    gU = torch.empty((B, L, C, H, W), dtype=torch.complex64, device="cuda")
    ctx.asm_propagate_backward(complex_dev(Pn), B, o, 1, 1, gU)
    gP = torch.empty((B, C, H, W), dtype=torch.complex64, device="cuda")
    ctx.asm_propagate_backward(complex_dev(U), B, o, -1, 0, gP)
    for b in range(B):
        U64, P64 = U[b].astype(np.complex128), Pn[b].astype(np.complex128)
        assert rel(out.cpu().numpy()[b], oracle.propagate_planes(U64, o.pitch, wl, z, bl, padding=1)) < 1e-5
        assert rel(inv.cpu().numpy()[b], oracle.inverse_propagate(P64, o.pitch, wl, z, bl, padding=1)) < 1e-5
        assert rel(gU.cpu().numpy()[b], oracle.propagate_planes_adjoint(P64, o.pitch, wl, z, bl, padding=1)) < 1e-5
        assert rel(gP.cpu().numpy()[b], oracle.inverse_propagate_adjoint(U64, o.pitch, wl, z, bl, padding=1)) < 1e-5
    # padding changes the result (the circular version wraps light around)
    circ = torch.empty_like(out)
    ctx.asm_propagate(complex_dev(U), B, dataclasses.replace(o, padding=0), 1, 1, circ)
    assert rel(circ.cpu().numpy(), out.cpu().numpy()) > 1e-3


def test_padded_render_forward_and_backward(P, ctx):
    o = S.Optics(48, 80, (639e-9, 473e-9), (0.0, 3e-3, 7e-3), padding=1)
    g = S.make_gaussians(300, o.L, o.C, o.H, o.W, seed=7, log_scale_mean=-2.8, log_scale_std=0.4)
    g["means"][:, 2] += 0.5
    V = 2
    vm, it = cams(V, o.H, o.W, seed=2)
    gd = dev(g)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((V, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
    Po, _, _, _ = oracle.render(g, vm.astype(np.float64), it.astype(np.float64), o, oracle_opts(P.DEFAULT_OPTS))
    assert rel(holo.cpu().numpy(), Po) < 1e-4
    gP = S.random_complex((V, o.C, o.H, o.W), seed=2)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(gP), grads)
    saved.release()
    ref = oracle.render_backward(g, vm.astype(np.float64), it.astype(np.float64), o, gP.astype(np.complex128),
                                 oracle_opts(P.DEFAULT_OPTS))
    for k in P.PARAM_NAMES:
        assert rel(grads[k].cpu().numpy(), ref[k]) < 1e-3, k


@pytest.mark.parametrize("objective", ["mse", "paper"])
def test_padded_losses(P, ctx, objective):
    o = S.Optics(64, 96, (639e-9, 515e-9), (0.0, 2e-3, 6e-3), padding=1)
    Pn = S.random_complex((1, o.C, o.H, o.W), seed=4)
    Igt = S.random_real((1, o.L, o.C, o.H, o.W), seed=5)
    M = S.plane_masks(1, o.L, o.H, o.W, seed=6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gP = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    Iout = torch.empty((1, o.L, o.C, o.H, o.W), dtype=torch.float32, device="cuda")
    P64, I64 = Pn[0].astype(np.complex128), Igt[0].astype(np.float64)
    if objective == "mse":
        ctx.focal_stack_loss(complex_dev(Pn), torch.from_numpy(Igt).cuda(), 1, o, loss, gP, Iout)
        l_ref, g_ref, I_ref = oracle.focal_stack_loss(P64, I64, o.pitch, o.wavelengths, o.plane_z, padding=1)
    else:
        ctx.paper_loss(complex_dev(Pn), torch.from_numpy(Igt).cuda(), torch.from_numpy(M).cuda(), 1, o, loss, gP,
                       Iout, lambda_ssim=0.5)
        l_ref, g_ref, I_ref = oracle.paper_loss(P64, I64, M[0].astype(np.float64), o.pitch, o.wavelengths,
                                                o.plane_z, lam=0.5, padding=1)
    assert abs(float(loss.item()) - l_ref) < 1e-5 * abs(l_ref)
    assert rel(Iout.cpu().numpy()[0], I_ref) < 1e-5
    assert rel(gP.cpu().numpy()[0], g_ref) < 1e-4


def test_padded_grid_size_is_checked(P, ctx):
    # 1080 x 2560: 2W = 5120 exceeds the longest supported transform
    o = S.Optics(1080, 2560, (515e-9,), (0.0,), padding=1)
    x = torch.zeros((1, 1, 1, o.H, o.W), dtype=torch.complex64, device="cuda")
    y = torch.zeros((1, 1, o.H, o.W), dtype=torch.complex64, device="cuda")
    with pytest.raises(P.HcgsError, match="UNSUPPORTED_SIZE"):
        ctx.asm_propagate(x, 1, o, 1, 1, y)
