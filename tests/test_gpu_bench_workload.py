"""Parity at full size, in the launch configuration the bench times: 16
views of 1080 x 1920, three wavelengths, 12 planes over 0-12 mm, rendered
and differentiated in one batch, at 1M Gaussians (the bench workload; FP32
path, FP16x2 and BF16x2 footprint tiers) and at 2M Gaussians (configuration
c4; all three tiers), so that the instance buffers sized from the
device's instance count and the strip lists are exercised at the largest
configuration; and the training configuration's render (c3: one view of
512 x 512, three wavelengths, 8 planes, 500k Gaussians; all three tiers).

The FP64 oracle cannot composite 16 full views in a test's time, so the
outputs are sampled where it can compute them exactly:
* the plane fields of one view on a band of image rows (all planes and
  channels; the oracle composites just those rows);
* that view's hologram from the GPU's own plane fields through the oracle's
  propagation (all 36 plane-channels at full size; FP32 path);
* the parameter gradients of the Gaussians whose support lies inside the
  band, with the upstream gradient nonzero on that view only: their
  gradients depend on the band's pixels alone, which the oracle's adjoint
  covers.
"""
import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import cams, cams_dev, complex_dev, dev, oracle_opts, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# relative L2 bounds (fields, gradients): 1e-4 / 1e-3 for the FP32 path
# (gradients are sums of many FP32 terms accumulated by atomics), 1e-2 for
# both reduced-precision tiers
TOL = {0: (1e-4, 1e-3), 1: (1e-2, 1e-2), 2: (1e-2, 1e-2)}
# workload: (footprint tiers, sampled view, row band)
WORKLOADS = {"1080p_rgb_L12_N1M_V16": ((0, 1, 2), 5, 480, 576),
             "c4_1080p_L12_N2M_V16": ((0, 1, 2), 5, 480, 576),
             "c3_512_L8_N500k": ((0, 1, 2), 0, 224, 288)}
CASES = [(w, fp) for w, spec in WORKLOADS.items() for fp in spec[0]]


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


_CASES = {}


def _case(P, name):
    # one oracle sample per workload, kept for the module (tiers share it)
    if name in _CASES:
        return _CASES[name]
    _CASES.clear()
    _, V0, R0, R1 = WORKLOADS[name]
    wl = S.workload(name)
    o = wl.optics
    g = S.make_gaussians(wl.N, o.L, o.C, o.H, o.W, seed=0)
    vm, it = cams(wl.V, o.H, o.W, seed=0)
    gP = np.zeros((wl.V, o.C, o.H, o.W), dtype=np.complex64)
    gP[V0] = S.random_complex((o.C, o.H, o.W), seed=2)
    # oracle, FP64 on the float32 values the GPU sees
    g64 = {k: np.asarray(g[k], dtype=np.float32).astype(np.float64) for k in P.PARAM_NAMES}
    v64, i64 = vm[V0].astype(np.float64), it[V0].astype(np.float64)
    oo = oracle_opts(dict(P.DEFAULT_OPTS))
    pr = oracle.project(g64, v64, i64, o.H, o.W, oo)
    Uo, _, _ = oracle.composite(pr, oo, rows=(R0, R1))
    band = Uo[:, :, R0:R1].copy()
    del Uo
    gU = oracle.propagate_planes_adjoint(gP[V0].astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
    g2d = oracle.composite_backward(pr, gU, oo, rows=(R0, R1))
    del gU
    go = oracle.project_backward(g64, v64, i64, o.H, o.W, g2d, oo)
    bb = pr["bbox"]  # x0, x1, y0, y1 of the support ellipse
    sel = (pr["valid"] == 1) & np.all(np.isfinite(bb), axis=1) & (bb[:, 1] > bb[:, 0]) & (bb[:, 3] > bb[:, 2])
    sel &= (bb[:, 1] >= 0) & (bb[:, 0] < o.W - 1) & (bb[:, 2] >= R0) & (bb[:, 3] <= R1 - 1)
    _CASES[name] = dict(wl=wl, o=o, g=g, vm=vm, it=it, gP=gP, band=band, go=go, sel=sel, V0=V0, R0=R0, R1=R1)
    return _CASES[name]


@pytest.mark.parametrize("workload,footprint", CASES)
def test_full_size_sampled_parity(P, workload, footprint):
    case = _case(P, workload)
    wl, o = case["wl"], case["o"]
    V0, R0, R1 = case["V0"], case["R0"], case["R1"]
    opts = dict(P.DEFAULT_OPTS, footprint=footprint)
    ctx = P.Context(0)
    gd = dev(case["g"])
    vmd, itd = cams_dev(case["vm"], case["it"])
    holo = torch.empty((wl.V, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    U = torch.empty((wl.V, o.L, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, opts, holo, U, saved)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(case["gP"]), grads)
    torch.cuda.synchronize()
    Uv = U[V0].cpu().numpy()
    hv = holo[V0].cpu().numpy()
    ggpu = {k: grads[k].cpu().numpy().astype(np.float64) for k in P.PARAM_NAMES}
    saved.release()
    del U, holo, grads, gd
    ctx.close()

    tol_f, tol_g = TOL[footprint]
    e_band = rel(Uv[:, :, R0:R1], case["band"])
    sel, go = case["sel"], case["go"]
    errs = {k: rel(ggpu[k][sel], go[k][sel]) for k in P.PARAM_NAMES}
    msg = "%s, footprint tier %d, view %d rows %d-%d: plane fields %.3e" % (workload, footprint, V0, R0, R1, e_band)
    if footprint == 0:
        # the view's hologram from the GPU's plane fields
        Po = oracle.propagate_planes(Uv.astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
        e_holo = rel(hv, Po)
        msg += ", hologram %.3e" % e_holo
        assert e_holo < 1e-5, e_holo
    print(msg + "; %d Gaussians inside the band:" % int(sel.sum()), {k: "%.2e" % v for k, v in errs.items()})
    assert e_band < tol_f, e_band
    assert int(sel.sum()) > 500
    for k, e in errs.items():
        assert e < tol_g, (k, e)
