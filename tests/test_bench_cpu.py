"""Host-side checks of bench.py (no GPU): the reference arm's JSON line, rank-0-only output,
the roofline helpers, clock/throttle parsing, and the multi-rank timing reduction run as two
gloo processes on the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def run_bench(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, env=env, cwd=ROOT)
    return r


def test_reference_arm_json_line():
    r = run_bench(["--impl", "reference", "--N", "10", "--steps", "2", "--warmup", "1", "--cpu-seconds", "0.05"])
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_only_rank0_prints():
    r = run_bench(["--impl", "reference", "--N", "10", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.05"],
                  env_extra={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_roofline_helpers(tmp_path, monkeypatch):
    # algorithmic counts per unit: N + 7 FP32 ops per Pauli string, 16 N tensor FLOPs per Pauli
    # string, 4.7 N + 8 FP32 ops per mana point
    assert bench.ops_per_string(20) == 27 and bench.ops_per_string(22) == 29
    assert bench.tensor_flops_per_string(22) == 4 * (128 + 64 + 128)
    assert bench.tensor_alg_flops_per_string(22) == 352
    assert bench.mana_ops_per_point(11) == pytest.approx(59.7)
    assert bench.fp32_peak_ops(152, 2070.0) == pytest.approx(152 * 128 * 2.07e9)
    assert bench.aggregate_rate(4, 5, 1e9, 2.0) == pytest.approx(1e10)
    assert bench.max_over_ranks(1.5, 1) == 1.5
    # measured peak from the file if present, else the stated fallback
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak("bf16_tflops", 1900.0) == (1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1901.0}))
    assert bench.measured_peak("bf16_tflops", 1900.0) == (1901.0, "measured")


def test_clock_sampler_summary_flags_throttling():
    cs = bench.ClockSampler(0)
    cs.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1995, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 1800, 2070, 1350.0, 0x8, Active, Not Active, Not Active, Active"]
    s = cs.summary()
    assert s["sm_mhz"] == 1995 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max = bench.max_over_ranks(times[rank], world)
        out.put((rank, t_max, bench.aggregate_rate(world, 3, 2.0 ** 20, t_max)))
    finally:
        dist.destroy_process_group()


def test_multi_rank_timing_takes_the_slowest_rank():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.25, 2.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate in res:
        assert t_max == 2.5  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 3 * 2.0 ** 20 / 2.5)  # whole-job aggregate (weak scaling)


def test_new_rows_child_reports_failures_without_raising():
    # the default run times the newer workloads in a child process; a child that fails (here:
    # no GPU) or overruns its limit must give an error entry, never an exception
    import bench
    out = bench.new_rows_in_child(timeout_s=0.001)
    assert "error" in out and "timed out" in out["error"]
    import torch
    if not torch.cuda.is_available():
        out = bench.new_rows_in_child(timeout_s=300)
        assert isinstance(out, dict) and "error" in out
