"""The multi-process (N > 1) path of bench.py on CPU: two gloo ranks run the
rendezvous, barrier and whole-job aggregation that torchrun uses on GPUs
(independent replicas, no data-path collective): value = the units of all
ranks over the slowest rank's time."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # rank k processed 1000 (k + 1) units in 10 (k + 1) ms
    value, ms_max = bench.job_rate(1000 * (rank + 1), 10.0 * (rank + 1), w)
    launches = bench.allreduce_sum(7, w)
    out.put((rank, value, ms_max, launches))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_whole_job_rate_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(1000 * (k + 1) for k in range(world))
    slowest = 10.0 * world
    for rank, value, ms_max, launches in res:
        assert ms_max == slowest
        assert value == pytest.approx(total / (slowest / 1e3))
        assert launches == 7 * world
    assert sorted(r[0] for r in res) == list(range(world))
