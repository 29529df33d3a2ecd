"""Host logic of bench.py's multi-rank run, on CPU with the gloo backend (world size 2):
the whole-job rate is all ranks' units over the slowest rank's time, and the
reference arm runs on rank 0 only."""
import argparse
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [0.5, 2.0][rank]                     # rank 1 is the slow one
        q.put((rank, bench.whole_job(local, 1000.0, dist)))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_uses_the_slowest_rank_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for r in (0, 1):
        slowest, rate = out[r]
        assert slowest == 2.0
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_rank_rate():
    import bench
    assert bench.whole_job(0.25, 100.0) == (0.25, 400.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    a = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(a) is None
    assert capsys.readouterr().out == ""


def test_workload_defaults(monkeypatch):
    """The low-Mach workload defaults to FP64 (its 1e-5 deviations are below FP32
    resolution); the others to FP32; an explicit --precision wins."""
    import bench
    for argv, want in ((["bench.py"], "f32"), (["bench.py", "--workload", "tables"], "f32"),
                       (["bench.py", "--workload", "luo"], "f64"),
                       (["bench.py", "--workload", "luo", "--precision", "f32"], "f32")):
        monkeypatch.setattr("sys.argv", argv)
        assert bench.parse().precision == want, argv
    import workloads as W
    luo = W.luo_runs()
    assert [lab["k"] for lab, _ in luo] == [0.03, 0.1, 1.0, 10.0]
    assert all(p["Qy"] == 0 and p["Qx"] == 2 and p["half"] == 1 and p["Pr"] == 1.0 for _, p in luo)
    tab = W.paper_tables(reduced=True)
    assert len(tab) == 20 and all(p["Qy"] == 0 for _, p in tab)


def test_clock_summary_parses_throttle_reasons():
    """bench.Clocks.summary: the median SM clock under load, the maximum, and every
    throttle reason that was active in any sample (from nvidia-smi's CSV lines)."""
    import bench
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2070, 1000.0, 0x8, Active, Not Active, Active, Not Active"]
    assert bench.Clocks(0).summary()["reasons"] == ["no samples"]
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0
