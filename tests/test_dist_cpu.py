"""The benchmark's multi-rank host logic on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) set up the process group, agree on the maximum
of their step times, compute the whole-job throughput from it, and the
reference arm returns on rank 1 without doing any work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_setup(False)
    assert (r, w, local) == (rank, world, rank)
    t_ms = 100.0 * (rank + 1)  # rank 1 is the slower one
    t_max = bench.max_over_ranks(t_ms, w, False)
    value = bench.job_throughput(10, w, t_max)

    class Args:
        workload, steps, warmup = "vessels", 1, 3
    rc = bench.run_reference(Args) if rank == 1 else 0  # rank 1 must return at once, without oracle work
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((rank, t_max, value, rc))


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(out.get(timeout=5) for _ in range(world))
    for rank, t_max, value, rc in res:
        assert t_max == 200.0
        assert value == pytest.approx(10 * 2 / 0.2)
        assert rc == 0
