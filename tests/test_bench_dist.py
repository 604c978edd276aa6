"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the GPU runs use NCCL), each timing
its own replica; the reported time is the slowest rank's and the rate counts both replicas; the
reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t_local = [1.5, 2.25][rank]
    t = bench.max_over_ranks(t_local, ws, device="cpu")
    rate = bench.whole_job_rate(ws, 1000, 10, t)
    env = bench.dist_env()

    class A:  # the reference arm's arguments
        gpus, steps, warmup = ws, 1, 0

    ref_rc = bench.run_reference(A()) if rank == 1 else None  # rank 1 must return without work
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, rate, env, ref_rc))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, env, ref_rc in out:
        assert t == 2.25                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000 * 10 / 2.25)
        assert env == (2, rank, rank)
    assert out[1][4] == 0                     # the reference arm: rank 1 exits 0 without running
