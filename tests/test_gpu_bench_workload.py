"""Parity at the bench workload's full size, in the launch configuration the
bench times: 16 views of 1080 x 1920, three wavelengths, 12 planes over
0-12 mm, 1M Gaussians, rendered and differentiated in one batch.

The FP64 oracle cannot composite 16 full views in a test's time, so the
outputs are sampled where it can compute them exactly:
* the plane fields of one view on a band of image rows (all planes and
  channels; the oracle composites just those rows);
* that view's hologram from the GPU's own plane fields through the oracle's
  propagation (all 36 plane-channels at full size);
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

V0, R0, R1 = 5, 480, 576  # sampled view and row band


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


def test_bench_workload_sampled_parity(P):
    wl = S.workload("1080p_rgb_L12_N1M_V16")
    o = wl.optics
    g = S.make_gaussians(wl.N, o.L, o.C, o.H, o.W, seed=0)
    vm, it = cams(wl.V, o.H, o.W, seed=0)
    opts = dict(P.DEFAULT_OPTS)

    # GPU: the whole batch forward and adjoint, as the bench launches it
    ctx = P.Context(0)
    gd = dev(g)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((wl.V, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    U = torch.empty((wl.V, o.L, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, opts, holo, U, saved)
    gP = np.zeros((wl.V, o.C, o.H, o.W), dtype=np.complex64)
    gP[V0] = S.random_complex((o.C, o.H, o.W), seed=2)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(gP), grads)
    torch.cuda.synchronize()
    Uv = U[V0].cpu().numpy()
    hv = holo[V0].cpu().numpy()
    ggpu = {k: grads[k].cpu().numpy().astype(np.float64) for k in P.PARAM_NAMES}
    saved.release()
    del U, holo, grads, gd
    ctx.close()

    # oracle, FP64 on the float32 values the GPU saw
    g64 = {k: np.asarray(g[k], dtype=np.float32).astype(np.float64) for k in P.PARAM_NAMES}
    v64, i64 = vm[V0].astype(np.float64), it[V0].astype(np.float64)
    oo = oracle_opts(opts)
    pr = oracle.project(g64, v64, i64, o.H, o.W, oo)

    # plane fields on the band
    Uo, _, _ = oracle.composite(pr, oo, rows=(R0, R1))
    e_band = rel(Uv[:, :, R0:R1], Uo[:, :, R0:R1])
    del Uo

    # the view's hologram from the GPU's plane fields
    Po = oracle.propagate_planes(Uv.astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
    e_holo = rel(hv, Po)
    del Po, Uv

    # gradients of the Gaussians whose support lies inside the band
    gU = oracle.propagate_planes_adjoint(gP[V0].astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
    g2d = oracle.composite_backward(pr, gU, oo, rows=(R0, R1))
    del gU
    go = oracle.project_backward(g64, v64, i64, o.H, o.W, g2d, oo)
    bb = pr["bbox"]  # x0, x1, y0, y1 of the support ellipse
    sel = (pr["valid"] == 1) & np.all(np.isfinite(bb), axis=1) & (bb[:, 1] > bb[:, 0]) & (bb[:, 3] > bb[:, 2])
    sel &= (bb[:, 1] >= 0) & (bb[:, 0] < o.W - 1) & (bb[:, 2] >= R0) & (bb[:, 3] <= R1 - 1)
    n_sel = int(sel.sum())
    errs = {k: rel(ggpu[k][sel], go[k][sel]) for k in P.PARAM_NAMES}
    print("bench workload, view %d rows %d-%d: plane fields %.3e, hologram %.3e; %d Gaussians inside the band:"
          % (V0, R0, R1, e_band, e_holo, n_sel), {k: "%.2e" % v for k, v in errs.items()})
    assert e_band < 1e-4, e_band
    assert e_holo < 1e-5, e_holo
    assert n_sel > 500, n_sel
    for k, e in errs.items():
        assert e < 1e-3, (k, e)
