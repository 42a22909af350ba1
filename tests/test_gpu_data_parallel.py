"""The data-parallel partition of the path, checked on one GPU.

Views are independent problems, so a batch of views may be split into
shards rendered one after another (or on different GPUs), with the
per-Gaussian gradients summed afterwards; and a data-parallel training step
on two ranks (one view each, gradients summed over the ranks before the
optimiser step) must take the same step as one process that sums the two
views' gradients itself.  The ranks are two processes over a gloo group on
one GPU; their kernels never wait on one another (the only exchange is the
gloo all-reduce of the gradient arrays, on the host).
"""
import socket

import numpy as np
import pytest

import hcgs_synth as S
from gpu_common import cams, cams_dev, complex_dev, dev, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


def test_view_shards_sum_to_the_batch_gradient(P):
    o = S.Optics(72, 120, S.WAVELENGTHS_RGB, (0.0, 3e-3, 6e-3, 9e-3))
    g = S.make_gaussians(3000, o.L, o.C, o.H, o.W, seed=5, log_scale_mean=-3.4)
    V = 4
    vm, it = cams(V, o.H, o.W, seed=2)
    gP = S.random_complex((V, o.C, o.H, o.W), seed=8)
    ctx = P.Context(0)
    gd = dev(g)

    def grads_of(views):
        vmd, itd = cams_dev(vm[views], it[views])
        n = len(views)
        holo = torch.empty((n, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
        saved = P.Saved(ctx)
        ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
        out = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
        ctx.render_view_backward(saved, gd, complex_dev(gP[views]), out)
        torch.cuda.synchronize()
        saved.release()
        return {k: out[k].cpu().numpy().astype(np.float64) for k in P.PARAM_NAMES}, holo.cpu().numpy()

    whole, holo = grads_of(list(range(V)))
    a, ha = grads_of([0, 1])
    b, hb = grads_of([2, 3])
    ctx.close()
    # the shards' holograms are the batch's, bit for bit (views do not interact)
    assert np.array_equal(np.concatenate([ha, hb]), holo)
    for k in P.PARAM_NAMES:
        e = rel(a[k] + b[k], whole[k])
        assert e < 1e-5, (k, e)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_training_step_matches_one_process(P):
    import torch.multiprocessing as mp

    import dp_worker
    from paper_2506_08350_b300.train import HologramTrainer
    steps, world = 2, 2
    mctx = mp.get_context("spawn")
    q = mctx.Queue()
    port = _free_port()
    procs = [mctx.Process(target=dp_worker.run, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = dict(q.get(timeout=600) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    # one process: both views' gradients, summed, then the same update
    o, g, vm, it, Igt = dp_worker.scene()
    ctx = P.Context(0)
    params = {k: torch.from_numpy(g[k]).cuda() for k in P.PARAM_NAMES}
    tr = HologramTrainer(ctx, params, o, data_parallel=False)
    for _ in range(steps):
        acc = None
        for r in range(world):
            tr.gradients(torch.from_numpy(vm[r:r + 1]).cuda(), torch.from_numpy(it[r:r + 1]).cuda(),
                         torch.from_numpy(Igt[r]).cuda())
            acc = {k: tr.g[k].clone() for k in P.PARAM_NAMES} if acc is None else \
                {k: acc[k] + tr.g[k] for k in P.PARAM_NAMES}
        for k in P.PARAM_NAMES:
            tr.g[k].copy_(acc[k])
        tr.apply_gradients()
    torch.cuda.synchronize()
    want = {k: params[k].cpu().numpy() for k in P.PARAM_NAMES}
    ctx.close()
    for r in range(world):
        for k in P.PARAM_NAMES:
            # both ranks hold the same parameters, those of the one-process step
            e = rel(res[r][k], want[k])
            assert e < 1e-5, (r, k, e)
