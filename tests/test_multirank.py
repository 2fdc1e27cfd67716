"""The bench's host logic on CPU: the multi-rank path (gloo, world size 2)
where every rank times its own replica, the job reports the slowest rank's
time and the reference arm runs on rank 0 only; and the clock record that
flags throttling."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.0 + 0.5 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(torch, mine, "cpu")
        out.put((rank, slowest, bench.whole_job_mlups(world, 1000, 10, slowest)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_and_whole_job_value():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [1.5, 1.5]
    # 2 ranks x 1000 cells x 10 steps in 1.5 s
    assert res[0][2] == pytest.approx(2 * 1000 * 10 / 1.5 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle on a bounded slab of the
    workload and prints one JSON line with the contract's keys."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--size", "16",
                                      "--steps", "2", "--warmup", "1"])
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_clock_summary_flags_throttling():
    """The clock record beside every bench line: median SM clock, maximum,
    and each throttle reason seen active in any sample (nvidia-smi CSV in
    the sampler's field order); unparsable lines are skipped."""
    import bench
    ok = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active"] * 4
    s = bench.ClockSampler.summarize(ok + ["[N/A], 2070, 0, x, x, x, x", "garbage"])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}
    hot = ok + ["1800, 2070, 1400.0, Not Active, Active, Not Active, Active",
                "1700, 2070, 1400.0, Active, Not Active, Not Active, Not Active"]
    s = bench.ClockSampler.summarize(hot)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 2070.0 and s["samples"] == 6
    assert bench.ClockSampler.summarize([]) is None
