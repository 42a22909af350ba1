"""GPU parity of the dense plane-weight gradient mode (rho_grad = 1) against
the FP64 oracle: every parameter gradient of the whole render path, the plane
logits now carrying the unassigned planes' terms through the straight-through
rule (a temperature large enough for them to matter)."""
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


@pytest.mark.parametrize("opts_name,order", [("default", 0), ("default", 1), ("exact", 0)])
def test_dense_rho_gradient_vs_oracle(P, ctx, opts_name, order):
    o = S.Optics(48, 80, (639e-9, 473e-9), (0.0, 3e-3, 7e-3))
    g = S.make_gaussians(300, o.L, o.C, o.H, o.W, seed=7, log_scale_mean=-2.8, log_scale_std=0.4)
    g["means"][:, 2] += 0.5
    g["plane_logits"] = np.random.default_rng(3).normal(size=g["plane_logits"].shape).astype(np.float32)
    base = {"default": P.DEFAULT_OPTS, "exact": P.EXACT_OPTS}[opts_name]
    opts = dict(base, order=order, ste_tau=2.0, rho_grad=1)
    V = 2
    vm, it = cams(V, o.H, o.W, seed=2)
    gd = dev(g)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((V, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    gP = S.random_complex((V, o.C, o.H, o.W), seed=2)
    grads, grads0 = ({k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES} for _ in range(2))
    for gr, rg in ((grads, 1), (grads0, 0)):
        saved = P.Saved(ctx)
        ctx.render_view(gd, vmd, itd, o, dict(opts, rho_grad=rg), holo, None, saved)
        ctx.render_view_backward(saved, gd, complex_dev(gP), gr)
        saved.release()
    oo = oracle_opts(dict(opts, rho_grad=0))
    ref = oracle.render_backward(g, vm.astype(np.float64), it.astype(np.float64), o, gP.astype(np.complex128), oo,
                                 rho_grad=1)
    for k in P.PARAM_NAMES:
        e = rel(grads[k].cpu().numpy(), ref[k])
        print(opts_name, order, k, "%.3e" % e)
        assert e < 1e-3, (k, e)
        if k != "plane_logits":
            assert rel(grads[k].cpu().numpy(), grads0[k].cpu().numpy()) < 1e-5, k  # atomics: order may differ
    # the dense terms change the logits' gradient
    assert rel(grads["plane_logits"].cpu().numpy(), grads0["plane_logits"].cpu().numpy()) > 1e-2
