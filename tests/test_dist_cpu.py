"""The bench's multi-GPU path is replicas only (a frame does not shard): N
ranks each render the same frame, the step time is the slowest rank's, and
the whole-job throughput is N x pixels / that time; the reference arm runs on
rank 0 alone.  These run the same helpers as world-size-2 gloo process groups
on the CPU (no GPU, no collective on the data path beyond the timing max)."""
import importlib.util
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    b = _bench()
    d = b.dist_init("gloo")
    ws2, r2, _ = b.dist_env()
    local_ms = [2.0, 5.0][rank]
    tput, ms = b.replica_throughput(ws2, 1000.0, local_ms, d)
    d.barrier()

    class A:
        steps, warmup, gpus = 1, 0, ws
    # the reference arm: rank 0 alone works; the others return at once
    ref_ran = None
    if rank != 0:
        b.run_reference(A())  # must return without running the oracle
        ref_ran = False
    q.put((rank, ws2, r2, tput, ms, ref_ran))
    dist.destroy_process_group()


def test_replica_timing_max_over_ranks_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r2, tput, ms, ref_ran in res:
        assert ws == 2 and r2 == rank
        assert ms == 5.0                     # the slowest rank bounds the step
        assert tput == pytest.approx(2 * 1000.0 / 5e-3)  # both replicas' units
    assert res[1][5] is False


def test_single_process_has_no_collective():
    b = _bench()
    tput, ms = b.replica_throughput(1, 500.0, 4.0, None)
    assert ms == 4.0 and tput == pytest.approx(500.0 / 4e-3)
