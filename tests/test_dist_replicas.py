"""Host logic of bench.py on CPU.  The N > 1 path (replicas: one right-hand side
per rank, no data exchange) with two gloo ranks: every rank gets its own
right-hand side, the timed region is the slowest rank's, and the whole-job rate
counts all ranks' solves.  The reference arm's JSON line (the oracle on the host)."""
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


def test_reference_arm_line(oracle_lib, monkeypatch):
    """bench.py --impl reference times the oracle on the host and prints the contract's keys
    (the default form's workload shrunk to 4^3x8 with 2 right-hand sides, one step)."""
    import argparse
    import bench
    monkeypatch.setitem(bench.FORMS, "hybrid", dict(dims=(8, 4, 4, 4), nrhs=2, seeds=(11, 12), lattice="4^3x8",
                                                    batch=2))
    monkeypatch.setattr(bench, "oracle_full_iters", lambda name: 50)
    line = bench.run_reference(argparse.Namespace(steps=1, warmup=1, form="hybrid"))
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]


def test_kernel_base_name_and_clock_parsing(tmp_path):
    """Host helpers of the bench line: kernel names as CUPTI writes them, and the clock
    record (median SM clock under load, throttle reasons seen) from nvidia-smi's CSV."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for name, base in (("void <unnamed>::k_hop_odd_s16<1, 3, 1, 128, 3>(Geom, SiteTermF, const int2 *)",
                        "k_hop_odd_s16"),
                       ("<unnamed>::k_pupdate_s(int, const <unnamed>::MMSCoef *, unsigned long)", "k_pupdate_s"),
                       ("void (anonymous namespace)::k_hop_even<double2, 1>(Geom, SiteTerm)", "k_hop_even"),
                       ("k_resid32(long, const float2 *, const float2 *, float2 *, double *)", "k_resid32")):
        assert bench.kernel_base_name(name) == base
    cs = bench.ClockSampler.__new__(bench.ClockSampler)   # no nvidia-smi: feed a recorded CSV
    f = open(tmp_path / "clocks.csv", "w+")
    f.write("0, 2070, 2070, 700.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "0, 2070, 2070, 1310.2, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "garbled line\n")
    f.flush()
    cs.f, cs.p = f, None
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
    class _Done:                                          # a finished sampler process
        def terminate(self):
            pass

        def wait(self):
            return 0
    cs.p = _Done()
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
