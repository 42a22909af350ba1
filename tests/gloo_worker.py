"""Worker of the two-rank CPU test (imported by spawned processes)."""
import os


def run(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2506_08350_b300 import PARAM_NAMES
        from paper_2506_08350_b300.parallel import allreduce_gradients, max_over_ranks, rank_seeds
        # the bench's step time: each rank reports its own, all agree on the largest
        m = max_over_ranks(10.0 + 3.0 * rank)
        # the data-parallel training step's exchange: per-Gaussian gradients summed
        grads = {k: torch.full((7, 3), float(rank + 1)) + torch.arange(21.0).reshape(7, 3) for k in PARAM_NAMES}
        allreduce_gradients(grads)
        want = sum(range(1, world + 1)) + world * torch.arange(21.0).reshape(7, 3)
        ok = all(torch.equal(grads[k], want) for k in PARAM_NAMES)
        q.put((rank, m, ok, rank_seeds(rank)))
    finally:
        dist.destroy_process_group()
