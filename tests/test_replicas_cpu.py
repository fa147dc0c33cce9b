"""The replica (multi-process) host logic of bench.py on CPU ranks over gloo.

Every GB300 machine here has one GPU, so `bench.py --gpus N` runs N independent replicas;
the only cross-rank steps are the barrier and the max-over-ranks of the step time.
This test runs them with world_size 2 on the gloo backend.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.replica_env()
        dist.barrier()
        slowest = bench.max_over_ranks(1.0 + 2.0 * r, w)  # rank 1 is the slow replica
        out.put((r, w, lr, slowest))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for r, w, lr, slowest in res:
        assert w == 2 and lr == r and slowest == 3.0


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5
