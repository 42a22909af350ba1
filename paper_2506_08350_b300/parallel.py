"""One process per GPU (torch.distributed): how the path shards.

Views are independent problems.  Rendering and the benchmark give each rank
its own batch of views (and, for the synthetic workloads, its own scene and
upstream-gradient draws), with no collective on the data path; the only
cross-rank step is the time each rank reports, reduced to the maximum.  A
training step across ranks takes different views on each rank and sums the
per-Gaussian gradient arrays before the optimiser step: one all-reduce per
step of N (11 + 2C + L) floats (the parameters of Sec. 3: mean, log-scale,
rotation, opacity, amplitude and phase per wavelength, plane logits).
"""
from __future__ import annotations

from . import PARAM_NAMES


def rank_seeds(rank: int) -> dict:
    """Seeds of the synthetic inputs of one rank (scene, views, upstream
    gradient); distinct per rank, so that ranks render independent views."""
    return {"scene": int(rank), "views": int(rank), "grad": 2 + int(rank)}


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the
    step time the bench reports), or ``value`` without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_gradients(grads: dict, group=None) -> None:
    """Sums the gradient arrays over the ranks, in place (the data-parallel
    training step's one exchange).  A no-op without a process group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return
    for k in PARAM_NAMES:
        dist.all_reduce(grads[k], op=dist.ReduceOp.SUM, group=group)
