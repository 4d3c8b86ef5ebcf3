"""The multi-GPU path of bench.py is replicas only: every rank advances its
own instance, and the whole-job value is the units all ranks processed over
the slowest rank's time.  Its host logic (rank environment, maximum over
ranks, aggregation) runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench._dist_env()
    ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    value = bench.replicas_rate(w, 1000.0, slowest / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, slowest, value))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(60)
    assert [p.exitcode for p in procs] == [0, 0]
    # both ranks see the slower rank's 150 ms; 2 ranks x 1000 units / 0.15 s
    for r, (rank, world, local, slowest, value) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == 150.0
        assert value == pytest.approx(2 * 1000.0 / 0.150, rel=1e-12)


def test_one_process_keeps_its_own_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replicas_rate(1, 500.0, 0.25) == 2000.0
