"""Finite differences at configuration c2: 1080 x 1920, three wavelengths, 8
planes over 0-10 mm, 100k Gaussians, one view.

The GPU adjoint of the whole render path (hcgs_render_view_backward, for the
loss Re<gP, P>) is compared with central differences of the FP64 oracle's
forward on 64 random parameters, plane logits excluded (their forward is
piecewise constant; the straight-through rule is pinned on the CPU).

Only the perturbed Gaussian's footprint can change when one of its
parameters moves by a small h: its own contribution, and, through T, the
contributions of the Gaussians behind it on its plane at the same pixels.
So with gU = ASM^H gP (FP64, once) the difference of the loss is
Re<gU, U(theta + h) - U(theta - h)> summed over the rows of the footprint's
bounding box, which the oracle composites on its own.  A parameter whose
perturbation changes a discrete decision is replaced by another draw: a
contributor that appears or goes at an alpha_min / T_eps threshold (seen in
the contributor counts), or a depth that moves past a neighbour's on the
same plane (seen in the visiting order; with ~5e4 Gaussians per metre of
depth on a plane, a step of 2e-5 m in a mean's depth does this often enough
to matter).
"""
import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import cams, cams_dev, complex_dev, dev, oracle_opts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_PARAMS = 64
CLASSES = (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("amplitude", 3), ("phase", 3))


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


def test_render_adjoint_vs_oracle_finite_differences_c2(P):
    wl = S.workload("c2_1080p_L8_N100k")
    o = wl.optics
    g = S.make_gaussians(wl.N, o.L, o.C, o.H, o.W, seed=0)
    vm, it = cams(1, o.H, o.W, seed=0)
    gP = S.random_complex((1, o.C, o.H, o.W), seed=2)

    # GPU: the whole path forward and adjoint
    ctx = P.Context(0)
    gd = dev(g)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(gP), grads)
    torch.cuda.synchronize()
    ggpu = {k: grads[k].cpu().numpy().astype(np.float64) for k in P.PARAM_NAMES}
    saved.release()
    ctx.close()

    # oracle: FP64 on the float32 values the GPU saw
    g64 = {k: np.asarray(g[k], dtype=np.float32).astype(np.float64) for k in P.PARAM_NAMES}
    v64, i64 = vm[0].astype(np.float64), it[0].astype(np.float64)
    opts = oracle_opts(P.DEFAULT_OPTS)
    gU = oracle.propagate_planes_adjoint(gP[0].astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
    pr0 = oracle.project(g64, v64, i64, o.H, o.W, opts)
    # candidates: visible Gaussians whose support box (x0, x1, y0, y1) meets
    # the image and spans at most 160 rows
    bb = pr0["bbox"]
    ok = (pr0["valid"] == 1) & (bb[:, 1] > bb[:, 0]) & (bb[:, 3] > bb[:, 2]) & np.all(np.isfinite(bb), axis=1)
    ok &= (bb[:, 1] >= 0) & (bb[:, 0] < o.W) & (bb[:, 3] >= 0) & (bb[:, 2] < o.H) & (bb[:, 3] - bb[:, 2] <= 160)
    y0 = np.floor(np.where(ok, bb[:, 2], 0)).astype(int)
    y1 = np.ceil(np.where(ok, bb[:, 3], 0)).astype(int) + 1
    cand = np.nonzero(ok)[0]
    assert cand.size > 1000

    def window_loss(gg, n, r0, r1):
        pr = oracle.project(gg, v64, i64, o.H, o.W, opts)
        l = pr0["plane"][n]
        # only plane l can change: leave the other planes' Gaussians out
        pr["valid"] = np.where(pr["plane"] == l, pr["valid"], 0).astype(np.int32)
        U, _, nc = oracle.composite(pr, opts, rows=(r0, r1))
        order = oracle.visiting_order(pr)
        return float(np.sum(np.real(np.conj(gU[l, :, r0:r1]) * U[l, :, r0:r1]))), nc[l, r0:r1].copy(), order

    rng = np.random.default_rng(1)
    per_class = {name: [] for name, _ in CLASSES}
    want = {name: N_PARAMS // len(CLASSES) + (1 if i < N_PARAMS % len(CLASSES) else 0)
            for i, (name, _) in enumerate(CLASSES)}
    tries = 0
    while any(len(per_class[k]) < want[k] for k in want):
        tries += 1
        assert tries < 20 * N_PARAMS, "too many draws change a discrete decision"
        name = [k for k in want if len(per_class[k]) < want[k]][0]
        width = dict(CLASSES)[name]
        n = int(rng.choice(cand))
        j = int(rng.integers(width))
        r0, r1 = max(0, y0[n] - 2), min(o.H, y1[n] + 2)
        theta = g64[name][n].reshape(-1)[j] if g64[name].ndim > 1 else g64[name][n]
        h = 1e-5 * max(1.0, abs(theta))
        vals, ncs, orders = [], [], []
        for sgn in (1.0, -1.0):
            gg = {k: v.copy() for k, v in g64.items()}
            if gg[name].ndim > 1:
                gg[name][n, j] += sgn * h
            else:
                gg[name][n] += sgn * h
            lv, nc, order = window_loss(gg, n, r0, r1)
            vals.append(lv)
            ncs.append(nc)
            orders.append(order)
        if not np.array_equal(ncs[0], ncs[1]):
            continue  # a contributor crossed a threshold: resample
        if not np.array_equal(orders[0], orders[1]):
            continue  # the depth moved past a neighbour's: the order is piecewise constant
        fd = (vals[0] - vals[1]) / (2.0 * h)
        gv = ggpu[name][n, j] if ggpu[name].ndim > 1 else ggpu[name][n]
        per_class[name].append((fd, gv, n, j))

    worst = []
    report = []
    for name, pairs in per_class.items():
        fd = np.array([a for a, _, _, _ in pairs])
        gv = np.array([b for _, b, _, _ in pairs])
        scale = np.sqrt(np.mean(fd ** 2))
        class_rel = np.linalg.norm(gv - fd) / max(np.linalg.norm(fd), 1e-300)
        bad = sorted(pairs, key=lambda t: -abs(t[1] - t[0]))[:5]
        report.append((name, round(float(class_rel), 6), [(round(a, 6), round(b, 6), n, j) for a, b, n, j in bad]))
        for a, b, n, j in pairs:
            worst.append((abs(b - a) / max(abs(a), 0.05 * scale), name, a, b, n, j))
    print("per class: rel L2 and the five largest |gpu - fd| (fd, gpu, gaussian, component):")
    for r in report:
        print("  ", r)
    for name, class_rel, _ in report:
        assert class_rel < 1e-3, report
    for e, name, a, b, n, j in worst:
        scale = np.sqrt(np.mean(np.array([t[0] for t in per_class[name]]) ** 2))
        assert abs(b - a) <= 1e-2 * abs(a) + 1e-3 * scale, (name, a, b, n, j)
    print("worst per-parameter error (relative to max(|fd|, 5 % of class rms)):", max(worst))
