"""The N > 1 path of bench.py: independent replicas, one per rank, joined only
by the max-over-ranks time and the sum of converged solves (no data-path
collective).  Runs as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed (10 + 5 r) ms and converged (100 + r) solves
    t, c = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 100 + rank, device="cpu")
    out[rank] = (t, c)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_time_max_and_count_sum():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        assert res[r] == (15.0, 201)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7) == (12.5, 7)
