"""The N > 1 path of bench.py (replicas: one right-hand side per rank, no data
exchange) on CPU with two gloo ranks: every rank gets its own right-hand side,
the timed region is the slowest rank's, and the whole-job rate counts all ranks'
solves."""
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


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench._dist()
        ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, got_ws, device="cpu")
        rate = bench.whole_job_rate(3 * bench.NSHIFT, got_ws, ms_max)
        q.put((got_rank, got_ws, bench.replica_rhs_seed(got_rank), ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert out[0][2] != out[1][2]                               # each replica its own right-hand side
    assert all(o[3] == 150.0 for o in out)                      # max over ranks on every rank
    assert all(abs(o[4] - 2 * 3 * bench.NSHIFT / 0.150) < 1e-9 for o in out)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(24, 1, 500.0) == 48.0
