"""GPU parity of the paper's training objective and optimiser against the
FP64 oracle: L_recon + L_SSIM on intensities (hcgs_paper_loss_intensities),
the whole loss through the inverse propagation (hcgs_paper_loss), and the
Adan step (hcgs_adan_step)."""
import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import complex_dev, rel

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


def _oracle_views(fn, B, *per_view):
    """Average a per-view oracle loss over B views: the loss is the mean of
    the views' losses and each view's gradient carries a factor 1/B."""
    losses, grads, rest = [], [], []
    for b in range(B):
        out = fn(*[a[b] if a is not None else None for a in per_view])
        losses.append(out[0])
        grads.append(out[1] / B)
        rest.append(out[2:])
    return float(np.mean(losses)), np.stack(grads), rest


# B, L, C, H, W: several 32 x 32 tiles with ragged tails, a single pixel,
# one-pixel-high and narrow images
SHAPES = [(2, 3, 2, 70, 45), (1, 2, 3, 33, 97), (1, 1, 1, 1, 1), (1, 2, 1, 1, 40), (2, 1, 2, 50, 3),
          (1, 4, 3, 128, 128)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("lam,with_masks", [(0.005, True), (0.5, True), (0.5, False), (0.0, True)])
def test_paper_loss_intensities(P, ctx, shape, lam, with_masks):
    B, L, C, H, W = shape
    I = S.random_real(shape, seed=11, hi=2.0)
    Igt = S.random_real(shape, seed=12)
    M = S.plane_masks(B, L, H, W, seed=13) if with_masks else None
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gI = torch.empty(shape, dtype=torch.float32, device="cuda")
    Md = torch.from_numpy(M).cuda() if with_masks else None
    ctx.paper_loss_intensities(torch.from_numpy(I).cuda(), torch.from_numpy(Igt).cuda(), Md, loss, gI,
                               lambda_ssim=lam)
    Mo = M if with_masks else np.zeros((B, L, H, W))
    l_ref, g_ref, _ = _oracle_views(lambda i, t, m: oracle.paper_loss_intensities(i, t, m, lam), B,
                                    I.astype(np.float64), Igt.astype(np.float64), Mo.astype(np.float64))
    # the kernel forms S in FP32: near S = 1 each value carries an absolute
    # error of a few units in the last place of 1 (6e-8), so the SSIM term
    # has an absolute error bound of about lambda * 4e-7 besides the relative one
    assert abs(float(loss.item()) - l_ref) < 2e-6 * abs(l_ref) + 4e-7 * lam, (float(loss.item()), l_ref)
    e = rel(gI.cpu().numpy(), g_ref)
    assert e < 2e-5, e


def test_paper_loss_intensities_ssim_term_alone(P, ctx):
    # identical images: L_recon and 1 - SSIM vanish, and so does the gradient
    # (SSIM is at its maximum); with lambda large the SSIM gradient dominates
    shape = (1, 2, 2, 40, 70)
    I = S.random_real(shape, seed=21)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gI = torch.empty(shape, dtype=torch.float32, device="cuda")
    It = torch.from_numpy(I).cuda()
    ctx.paper_loss_intensities(It, It.clone(), None, loss, gI, lambda_ssim=1.0)
    assert abs(float(loss.item())) < 1e-6
    assert float(gI.abs().max()) < 1e-7  # terms of size ~1e-3 cancel
    I2 = S.random_real(shape, seed=22)
    ctx.paper_loss_intensities(torch.from_numpy(I2).cuda(), It, None, loss, gI, lambda_ssim=100.0)
    l_ref, g_ref, _ = _oracle_views(lambda i, t: oracle.paper_loss_intensities(i, t, np.zeros((2, 40, 70)), 100.0),
                                    1, I2.astype(np.float64), I.astype(np.float64))
    assert abs(float(loss.item()) - l_ref) < 2e-6 * l_ref + 4e-7 * 100.0
    assert rel(gI.cpu().numpy(), g_ref) < 2e-5


@pytest.mark.parametrize("B,H,W,C,L", [(1, 64, 80, 2, 3), (2, 48, 64, 3, 2), (1, 256, 256, 1, 4),
                                       (1, 1080, 1920, 3, 8)])
def test_paper_loss(P, ctx, B, H, W, C, L):
    o = S.Optics(H, W, (639e-9, 515e-9, 473e-9)[:C], tuple(float(z) for z in np.linspace(0.0, 1e-2, L)))
    Pn = S.random_complex((B, o.C, o.H, o.W), seed=4)
    Igt = S.random_real((B, o.L, o.C, o.H, o.W), seed=5)
    M = S.plane_masks(B, o.L, o.H, o.W, seed=6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gP = torch.empty((B, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    Iout = torch.empty((B, o.L, o.C, o.H, o.W), dtype=torch.float32, device="cuda")
    ctx.paper_loss(complex_dev(Pn), torch.from_numpy(Igt).cuda(), torch.from_numpy(M).cuda(), B, o, loss, gP, Iout)
    l_ref, g_ref, rest = _oracle_views(
        lambda p, t, m: oracle.paper_loss(p, t, m, o.pitch, o.wavelengths, o.plane_z), B,
        Pn.astype(np.complex128), Igt.astype(np.float64), M.astype(np.float64))
    I_ref = np.stack([r[0] for r in rest])
    assert abs(float(loss.item()) - l_ref) < 1e-5 * abs(l_ref), (float(loss.item()), l_ref)
    assert rel(Iout.cpu().numpy(), I_ref) < 1e-5
    e = rel(gP.cpu().numpy(), g_ref)
    assert e < 1e-4, e
    # without the optional outputs the loss is the same
    loss2 = torch.zeros(1, dtype=torch.float32, device="cuda")
    ctx.paper_loss(complex_dev(Pn), torch.from_numpy(Igt).cuda(), torch.from_numpy(M).cuda(), B, o, loss2)
    assert float(loss2.item()) == float(loss.item())


def test_paper_loss_reduces_to_focal_stack_loss(P, ctx):
    # no masks, no SSIM, zero targets: the weights are 1 and the loss is the
    # plain focal-stack loss on the same propagation
    o = S.Optics(64, 96, (639e-9, 515e-9), (0.0, 2e-3, 5e-3))
    Pn = complex_dev(S.random_complex((1, o.C, o.H, o.W), seed=7))
    Igt = torch.zeros((1, o.L, o.C, o.H, o.W), dtype=torch.float32, device="cuda")
    l1, l2 = (torch.zeros(1, dtype=torch.float32, device="cuda") for _ in range(2))
    g1, g2 = (torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda") for _ in range(2))
    ctx.paper_loss(Pn, Igt, None, 1, o, l1, g1, lambda_ssim=0.0)
    ctx.focal_stack_loss(Pn, Igt, 1, o, l2, g2)
    assert abs(float(l1.item()) - float(l2.item())) < 1e-6 * float(l2.item())
    assert rel(g1.cpu().numpy(), g2.cpu().numpy()) < 1e-6


def test_adan_steps(P, ctx):
    rng = np.random.default_rng(3)
    n = 100003  # ragged: not a multiple of the block
    p = rng.normal(size=n).astype(np.float32)
    gs = [rng.normal(size=n).astype(np.float32) for _ in range(5)]
    pt = torch.from_numpy(p.copy()).cuda()
    gp, m, v, nn = (torch.full((n,), 7.0, dtype=torch.float32, device="cuda") for _ in range(4))  # any state
    pr = p.astype(np.float64)
    mr = vr = nr = np.zeros(n)
    prev = np.zeros(n)
    for step, g in enumerate(gs, start=1):
        lr = oracle.cosine_lr(step, 5, 1e-2, 1e-5)
        ctx.adan_step(pt, torch.from_numpy(g).cuda(), gp, m, v, nn, step, lr, weight_decay=0.02)
        pr, mr, vr, nr = oracle.adan_step(pr, g, prev, mr, vr, nr, step, lr, weight_decay=0.02)
        prev = g.astype(np.float64)
    assert rel(pt.cpu().numpy(), pr) < 1e-6
    assert rel(m.cpu().numpy(), mr) < 1e-6
    assert rel(v.cpu().numpy(), vr) < 1e-5
    assert rel(nn.cpu().numpy(), nr) < 1e-6
    assert np.array_equal(gp.cpu().numpy(), gs[-1])
