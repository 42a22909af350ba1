"""GPU parity of the densification step (Algorithm 1) and its noise against
the oracle: Philox words bit for bit, normals to rounding, the per-Gaussian
decisions exactly, the new arrays element by element, the screen-space
statistics of a rendered view; and a ring run with densification on."""

import numpy as np
import pytest

import hcgs_synth as S
import oracle
from gpu_common import cams, cams_dev, complex_dev, dev, oracle_opts, rel

pytestmark = pytest.mark.gpu

# densification threshold on the mean NDC gradient norm for the ring test's
# loss scale (the 3DGS default 2e-4 belongs to a per-image L1 loss)
DENSIFY_THRESHOLD = 1e-3

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

@pytest.mark.parametrize("seed,stream,n", [(0, 0, 1001), (2 ** 40 + 7, 5, 4096), (123, 0xFFFFFFFF, 3)])
def test_philox_words_and_normals(P, ctx, seed, stream, n):
    w = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.philox(seed, n, w, kind=0, stream_id=stream)
    got = w.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.philox_words(seed, n, stream))
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx.philox(seed, n, z, kind=1, stream_id=stream)
    ref = oracle.philox_normals(seed, n, stream)
    assert np.max(np.abs(z.cpu().numpy() - ref) / np.maximum(1.0, np.abs(ref))) < 1e-6
    # uniforms bit for bit: the FP64 value (w + 1/2) 2^-32 is exact, and both
    # sides round it once to FP32
    ctx.philox(seed, n, z, kind=2, stream_id=stream)
    ref_u = oracle.philox_uniforms(seed, n, stream).astype(np.float32)
    assert np.array_equal(z.cpu().numpy().view(np.uint32), ref_u.view(np.uint32))

def _scene(n, C=3, L=4, seed=0):
    rng = np.random.default_rng(seed)
    g = S.make_gaussians(n, L, C, 64, 64, seed=seed)
    g["log_scales"] = rng.normal(-4.0, 0.6, size=(n, 3)).astype(np.float32)
    g["opacity_logits"] = rng.normal(0.0, 3.0, size=n).astype(np.float32)
    accum = rng.uniform(0, 6e-4, size=n).astype(np.float32)
    denom = rng.integers(0, 3, size=n).astype(np.float32)
    return g, accum, denom

@pytest.mark.parametrize("n,prune_scale", [(5003, 0.0), (777, 0.05), (1, 0.0)])
def test_densify_plan_and_apply(P, ctx, n, prune_scale):
    C, L = 3, 4
    g, accum, denom = _scene(n, C, L, seed=n)
    o = dict(P.DEFAULT_DENSIFY, prune_scale=prune_scale)
    gd = dev(g)
    act, off, n_new = ctx.densify_plan(gd, torch.from_numpy(accum).cuda(), torch.from_numpy(denom).cuda(), o)
    ref_act = oracle.densify_actions(g, accum, denom, o)
    assert np.array_equal(act.cpu().numpy(), ref_act)
    per = np.array([1, 0, 2, 2])[ref_act]
    assert n_new == per.sum()
    assert np.array_equal(off.cpu().numpy().view(np.uint32), np.concatenate([[0], np.cumsum(per)]))
    if n_new == 0:
        return
    noise = torch.empty((n, 2, 3 + C), dtype=torch.float32, device="cuda")
    ctx.philox(9, noise.numel(), noise, kind=1, stream_id=300)
    m1 = torch.from_numpy(np.random.default_rng(1).normal(size=(n, 3)).astype(np.float32)).cuda()
    m2 = torch.from_numpy(np.random.default_rng(2).normal(size=n).astype(np.float32)).cuda()
    out = {k: torch.empty((n_new,) + tuple(v.shape[1:]), dtype=torch.float32, device="cuda") for k, v in gd.items()}
    o1, o2 = torch.empty((n_new, 3), device="cuda"), torch.empty(n_new, device="cuda")
    ctx.densify_apply(gd, C, L, act, off, noise, out, o, extras=[(m1, o1), (m2, o2)])
    newp, (e1, e2), _ = oracle.densify(g, accum, denom, noise.cpu().numpy(), o,
                                       extra=(m1.cpu().numpy(), m2.cpu().numpy()))
    for k in P.PARAM_NAMES:
        got = out[k].cpu().numpy()
        assert got.shape == newp[k].shape, k
        assert np.allclose(got, newp[k], rtol=2e-6, atol=2e-6), (k, np.max(np.abs(got - newp[k])))
    assert np.array_equal(o1.cpu().numpy(), e1.astype(np.float32))
    assert np.array_equal(o2.cpu().numpy(), e2.astype(np.float32))

def test_densify_all_pruned_and_empty(P, ctx):
    g, accum, denom = _scene(50)
    g["opacity_logits"][:] = -10.0
    act, off, n_new = ctx.densify_plan(dev(g), torch.from_numpy(accum).cuda(), torch.from_numpy(denom).cuda())
    assert n_new == 0 and np.all(act.cpu().numpy() == oracle.PRUNE)
    g0 = {k: v[:0] for k, v in g.items()}
    e = torch.zeros(0, device="cuda")
    act, off, n_new = ctx.densify_plan(dev(g0), e, e)
    assert n_new == 0 and off.cpu().numpy()[0] == 0

def test_densify_statistics_of_a_rendered_view(P, ctx):
    o = S.Optics(48, 80, (639e-9, 473e-9), (0.0, 3e-3, 7e-3))
    g = S.make_gaussians(300, o.L, o.C, o.H, o.W, seed=7, log_scale_mean=-2.8, log_scale_std=0.4)
    g["means"][:, 2] += 0.5
    V = 2
    vm, it = cams(V, o.H, o.W, seed=2)
    gd = dev(g)
    vmd, itd = cams_dev(vm, it)
    holo = torch.empty((V, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
    gP = S.random_complex((V, o.C, o.H, o.W), seed=2)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(gP), grads)
    accum = torch.full((300,), 0.5, device="cuda")  # statistics add to what is there
    denom = torch.ones(300, device="cuda")
    ctx.densify_accumulate(saved, accum, denom)
    saved.release()
    opts = oracle_opts(P.DEFAULT_OPTS)
    g64 = {k: np.asarray(g[k], dtype=np.float32).astype(np.float64) for k in P.PARAM_NAMES}
    ra, rd = np.full(300, 0.5, dtype=np.float32), np.ones(300, dtype=np.float32)
    for v in range(V):
        pr = oracle.project(g64, vm[v].astype(np.float64), it[v].astype(np.float64), o.H, o.W, opts)
        gU = oracle.propagate_planes_adjoint(gP[v].astype(np.complex128), o.pitch, o.wavelengths, o.plane_z)
        gb = oracle.composite_backward(pr, gU, opts)
        ra, rd = oracle.densify_accumulate(ra, rd, pr["valid"], gb["mu"], o.H, o.W)
    assert np.array_equal(denom.cpu().numpy(), rd)
    assert rel(accum.cpu().numpy() - 0.5, ra - 0.5) < 1e-3

def test_ring_run_with_densification(P):
    # the reduced ring configuration with the paper's recipe and densification
    # at step 300 (the paper's period), then 150 more steps: the count changes
    # as the statistics dictate and the focal-stack PSNR still rises
    from paper_2506_08350_b300.train import ring_run
    c = P.Context(0)
    o = S.workload("c3_512_L8_N500k").optics
    dens = dict(grad_threshold=DENSIFY_THRESHOLD, split_scale=0.02, prune_opacity=0.01)
    r = ring_run(c, o, 50_000, steps=450, n_views=10, objective="paper", optimizer="adan", anneal=True,
                 densify=dens)
    print("ring run with densification:", {k: v for k, v in r.items() if k != "densify"})
    for d in r["densify"]:
        print("  ", d)
    assert len(r["densify"]) == 1
    d = r["densify"][0]
    assert d["n_after"] == d["keep"] + 2 * (d["clone"] + d["split"]) == r["N_end"]
    assert d["clone"] + d["split"] > 0
    assert r["psnr_end"] > r["psnr_start"] + 1.0, r
    c.close()
