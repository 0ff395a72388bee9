"""The N > 1 bench path on CPU: world size 2 over gloo (replicas only -- the
filter's columns are independent, so ranks exchange nothing but the final
timing reduction)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.replica_max_ms(times[rank], torch.device("cpu"))
        val = bench.replica_throughput(1e12, world, ms)
        dist.barrier()
        out_q.put((rank, ms, val))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(100.0, 250.0), (80.0, 40.0)])
def test_replica_timing_is_max_over_ranks(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in results:
        assert ms == max(times)
        assert abs(val - 2 * 1e12 / (max(times) * 1e-3) / 1e9) < 1e-6


def test_single_process_is_identity():
    import bench
    assert bench.replica_max_ms(12.5, torch.device("cpu")) == 12.5
    assert bench.replica_throughput(2e9, 1, 1000.0) == 2.0
