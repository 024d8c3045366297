"""The benchmark's multi-GPU path is replicas only (one workload per rank, no
collective on the data path): the whole-job rate is the units of all ranks over
the slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    D = bench.Dist(world, rank, backend="gloo")
    units = 12 * (rank + 1)           # ranks may process different amounts
    seconds = 0.5 + rank              # the slowest rank sets the time
    value, t_max = bench.whole_job_rate(D, units, seconds)
    D.barrier()
    out[rank] = (value, t_max)
    D.close()


def test_whole_job_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        value, t_max = out[r]
        assert t_max == pytest.approx(1.5)
        assert value == pytest.approx((12 + 24) / 1.5)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    D = bench.Dist(1, 0)
    assert bench.whole_job_rate(D, 24, 2.0) == (12.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 exits without work and prints nothing."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(None, bench.WORKLOADS["4^4"], "4^4")
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero(monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the contract's keys: the oracle's
    rate as value, cpu_baseline describing the same run, an e2e with no copies."""
    import json
    import types
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(types.SimpleNamespace(steps=1, warmup=0), bench.WORKLOADS["4^4"], "4^4")
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the steps are real: value x ms_per_step is the work one step did, and the steps ran
    assert d["value"] * d["ms_per_step"] / 1000.0 == pytest.approx(d["solves_per_step"])
    # both arms describe the workload with the same config
    assert d["config"] == bench.bench_config(bench.WORKLOADS["4^4"], "4^4", 1)


def test_reference_arm_steps_take_the_time_they_claim(monkeypatch):
    """ms_per_step x steps is the wall time the timed steps took (within the warm-up's share)."""
    import json
    import time
    import types
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    t0 = time.perf_counter()
    with redirect_stdout(buf):
        bench.reference_arm(types.SimpleNamespace(steps=3, warmup=1), bench.WORKLOADS["4^4"], "4^4")
    wall = time.perf_counter() - t0
    d = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert d["steps"] == 3
    assert d["ms_per_step"] * d["steps"] / 1000.0 <= wall


def test_roofline_entry_arithmetic():
    """The roofline entry picks the bandwidth class with the largest summed event time (never the
    latency-bound second-stage reduction), divides bytes per launch by the average duration, and
    scales the measured DRAM ratio by the average launch's bytes (null where none was measured)."""
    sys.path.insert(0, ROOT)
    import bench
    kt = {"k_reduce": {"ms": 99.0, "launches": 10, "bytes": 1e6},
          "k_dcgs_update<float2>": {"ms": 20.0, "launches": 10, "bytes": 10 * 6.8e7},
          "k_hw<float,float2>": {"ms": 15.0, "launches": 30, "bytes": 30 * 1e7}}
    r = bench.roofline(kt, 6800.0, "measured", 0.1)
    assert r["kernel"] == "k_dcgs_update<float2>" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6.8e7 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert r["traffic"] == pytest.approx(bench.DRAM_PER_ALGORITHMIC_BYTE["k_dcgs_update<float2>"] * 6.8e7)
    assert r["share_of_timed"] == pytest.approx(0.2)
    kt["k_hw<float,float2>"]["ms"] = 50.0
    r = bench.roofline(kt, 6800.0, "measured", 0.1)
    assert r["kernel"] == "k_hw<float,float2>" and r["traffic"] is None


def test_solve_roofline_arithmetic():
    """The whole-solve entry: the counted bytes of every timed class per step over the headline
    step time, against the HBM peak; no entry without steps or time."""
    sys.path.insert(0, ROOT)
    import bench
    kt = {"k_reduce": {"ms": 1.0, "launches": 10, "bytes": 2e6},
          "k_dcgs_update<float2>": {"ms": 20.0, "launches": 10, "bytes": 6e9},
          "k_hw<float,float2>": {"ms": 15.0, "launches": 30, "bytes": 2e9}}
    r = bench.solve_roofline(kt, 2, 0.001, 6800.0, "measured")
    assert r["bytes_per_step"] == pytest.approx((2e6 + 6e9 + 2e9) / 2)
    assert r["achieved"] == pytest.approx((2e6 + 6e9 + 2e9) / 2 / 0.001 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0) and r["unit"] == "GB/s"
    assert bench.solve_roofline(kt, 0, 0.001, 6800.0, "measured") is None
    assert bench.solve_roofline(kt, 2, 0.0, 6800.0, "measured") is None


def test_clock_summary_parses_samples():
    """Median SM clock under load, the maximum, and the throttle reasons seen in any sample."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 712.3, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1399.0, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
               "[N/A], garbage"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_workload_inputs():
    """The default workload's sources are the 12 spin-colour point sources at site 0 (column
    3 spin + colour is the unit vector of that component), and its name states the sizes."""
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    w = bench.WORKLOADS["10^4"]
    B = bench.sources(w)
    assert B.shape == (12, 12 * 10 ** 4)
    assert np.array_equal(B[:, :12], np.eye(12)) and not np.any(B[:, 12:])
    name = bench.workload_name(w, "10^4")
    assert "lattice 10x10x10x10" in name and "FOM-LR(30,40)" in name and "12 point sources" in name
