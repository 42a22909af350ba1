"""Rank of the two-process data-parallel training test (imported by spawned
processes): one view per rank, gradients summed over a gloo group."""
import os


def scene():
    """The shared synthetic problem: optics, Gaussians, two views, targets."""
    import numpy as np

    import hcgs_synth as S
    o = S.Optics(48, 80, S.WAVELENGTHS_RGB[:2], (0.0, 2e-3, 4e-3))
    g = S.make_gaussians(600, o.L, o.C, o.H, o.W, seed=21, log_scale_mean=-3.2)
    vm, it = S.view_batch(2, o.H, o.W, seed=4)
    Igt = S.random_real((2, 1, o.L, o.C, o.H, o.W), seed=9)
    return o, g, vm.astype(np.float32), it.astype(np.float32), Igt


def run(rank, world, port, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        import paper_2506_08350_b300 as P
        from paper_2506_08350_b300.train import HologramTrainer
        o, g, vm, it, Igt = scene()
        ctx = P.Context(0)
        params = {k: torch.from_numpy(g[k]).cuda() for k in P.PARAM_NAMES}
        tr = HologramTrainer(ctx, params, o, data_parallel=True)
        v = torch.from_numpy(vm[rank:rank + 1]).cuda()
        i = torch.from_numpy(it[rank:rank + 1]).cuda()
        t = torch.from_numpy(Igt[rank]).cuda()
        for _ in range(steps):
            tr.step(v, i, t)
        torch.cuda.synchronize()
        q.put((rank, {k: params[k].cpu().numpy() for k in P.PARAM_NAMES}))
        ctx.close()
    finally:
        dist.destroy_process_group()
