"""The multi-process pieces of the path, on the CPU: two ranks over gloo.

Views are independent problems: each rank renders its own views (distinct
input seeds), the bench reduces the ranks' step times to the maximum, and a
data-parallel training step sums the per-Gaussian gradients over the ranks.
"""
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo():
    import torch.multiprocessing as mp

    import gloo_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=gloo_worker.run, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 13.0 for r in res)  # max over ranks
    assert all(r[2] for r in res)  # gradients summed on every rank
    assert res[0][3] != res[1][3]  # independent inputs per rank
