"""Benchmark of the exact-SRE hot path (and its CPU oracle as the reference arm).

Default workload (one step = one complete exact M_2 of one state, every X-string):
  N = 20 qubits, complex64 state of a seeded brick-wall circuit of Haar-random two-qubit
  gates on |0...0> (depth 10, open chain, seed 2001 -- the paper's Eq. randC workload),
  FP32 CUDA-core Walsh-Hadamard path, 4^20 = 1.1e12 Pauli strings per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--N 20] [--path cudacore|tensor] [--no-cpu-baseline] [--no-lines] [--extra] [--xstrings K]

The same line carries the metric's other configurations ("lines"): exact M2 at N = 22 on the
CUDA-core and the tensor-core paths and exact mana at N = 11, each with its clocks, roofline
fraction and error against an independent value.

Multi-GPU (torchrun, one rank per GPU): the X-strings are independent (Sec. 3.1.2; Sec. 4.1
splits them over ranks and GPUs), so the ranks split the one state's X-strings into
chunk-aligned slices, all-gather the per-chunk FP64 sums over NCCL and combine them in chunk
order ("scaling": "strong": the work per step is fixed); rank 0 prints the JSON line with the
max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pauli strings/s for exact SRE (N=20,22 qubits) & mana (N=11); % of roofline"
UNIT = "Pauli strings/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--N", type=int, default=20)
    ap.add_argument("--path", default="cudacore", choices=["cudacore", "tensor", "auto"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extra", action="store_true",
                    help="also time N=22, mana N=11, MC N=28, batched, thermodynamic integration N=20, "
                         "mixed-state mana N=8, even-sector SRE N=20, qudit mana d=5, mana gradient")
    ap.add_argument("--only", default="",
                    help="run just the named --extra workloads (comma-separated, e.g. ti_N20_L10) and print them")
    ap.add_argument("--no-lines", action="store_true",
                    help="skip the metric's other configurations (N = 22 on both paths, mana N = 11)")
    ap.add_argument("--no-new-rows", action="store_true",
                    help="skip the separate-process timing of the Algorithm 3 / 6, sector and qudit workloads")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--shape", default="",
                    help="profiling aid: UPW,TPT,R,LAG pins the two-pass task shape (no tuning launches)")
    ap.add_argument("--xstrings", type=int, default=0,
                    help="profiling aid: each step evaluates only the first K X-strings of the "
                         "workload (per-X-string sums) instead of the full M_2")
    return ap.parse_args()


def workload_state(N: int):
    import numpy as np
    from paper_2601_07824_gb300 import inputs
    if N == 20:
        return inputs.brickwork_haar(20, 10, seed=2001, dtype=np.complex64), \
            "brickwork Haar circuit on |0>^20, depth 10, open chain, seed 2001"
    return inputs.brickwork_haar(N, 10, seed=2000 + N, dtype=np.complex64), \
        f"brickwork Haar circuit on |0>^{N}, depth 10, open chain, seed {2000 + N}"


# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu capture of this
# exact command on the current kernel (profiles/); absent (null) when no capture matches it.
TRAFFIC = {(20, 0): 254603761408 + 951125725952}  # sre_twopass<10, 9, 2>, N = 20, one full M2


def ops_per_string(N: int) -> int:
    # Algorithmic FP32 operations per Pauli string (FMA counted once) of the method's real
    # transform (u = Re v + Im v of length 2^N): N butterfly stages, the pair product and u,
    # and the |c|^4 / |c|^2 reduction -- N + 7.  (The kernels' half-length complex form issues
    # N + 4: N - 1 stages, 2 for the pair product, 3 for the reduction.)
    return N + 7


def mana_ops_per_point(N: int) -> float:
    # radix-3 transform: ~14 FP32 operations per 3 complex values per digit (4.7 per value and
    # digit), plus ~8 for the pair product and |chi| -- about 60 at N = 11
    return 4.7 * N + 8.0


def fp32_peak_ops(sm_count: int, mhz: float) -> float:
    return sm_count * 128 * mhz * 1e6


def tensor_flops_per_string(N: int) -> int:
    # tensor-core path as issued: each Pauli string is one real value of the half-length
    # transform; its Kronecker blocks are K = 128, 64 and 128 wide (pass 1: 7 + 6 bits, pass 2:
    # 7 bits), each applied to the hi and the lo operand: 2 (hi, lo) x 2 (multiply-add) x
    # (128 + 64 + 128)
    return 4 * (128 + 64 + 128)


def tensor_alg_flops_per_string(N: int) -> int:
    # algorithmic tensor work of the method: H_16 blocks (4 bits each) on hi/lo operands,
    # 2 x 2 x 16 = 64 FLOPs per value per 4 stages -> 16 N per Pauli string
    return 16 * N


def golden_value(key: str):
    """A stored FP64 oracle value for a full-size workload (tests/golden/oracle_full_size.json,
    written by tests/golden/make_full_size_values.py), or None."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_full_size.json")) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def measured_peak(key: str, fallback: float):
    """A peak from MEASURED_PEAKS.json (driver-written) and where it came from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get(key)
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return fallback, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def max_over_ranks(t_local: float, world: int, device=None) -> float:
    """The slowest rank's time (all-reduce MAX over the default process group when world > 1)."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, steps: int, units_per_step: float, t_max: float) -> float:
    """Whole-job throughput: every rank processes `units_per_step` per step (weak scaling)."""
    return world * steps * units_per_step / t_max


def _calibrate(oracle, psi_np, dim, threads, rng):
    """Seconds per X-string of the oracle on this host (probe grown until it takes >= 0.3 s)."""
    count = max(threads, 4)
    while True:
        probe = rng.integers(0, dim, count)
        t0 = time.perf_counter()
        oracle.sre_terms_list(psi_np, probe, threads)
        dt = time.perf_counter() - t0
        if dt >= 0.3 or count >= (1 << 20):
            return dt / count
        count *= 4


def cpu_baseline(psi_np, N: int, seconds: float):
    """The FP64 oracle (as it stands) on a bounded sample of X-strings of the same workload."""
    import numpy as np
    import oracle
    threads = oracle.num_threads(0)
    dim = 2 ** N
    rng = np.random.default_rng(12345)
    # calibrate on a handful of X-strings, then size the sample to ~`seconds` of CPU work
    per_a = _calibrate(oracle, psi_np, dim, threads, rng)
    count = int(max(threads, min(1 << 22, seconds / max(per_a, 1e-9))))
    a = rng.integers(0, dim, count)
    t0 = time.perf_counter()
    oracle.sre_terms_list(psi_np, a, threads)
    dt = time.perf_counter() - t0
    return {"value": count * dim / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{count} uniformly drawn X-strings of the N={N} workload (each a full "
                      f"2^{N}-point FP64 Walsh-Hadamard transform), {dt:.1f} s"}, dt


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on this host, same metric and config."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    N = args.N
    psi, desc = workload_state(N)
    threads = oracle.num_threads(0)
    dim = 2 ** N
    rng = np.random.default_rng(777)
    per_a = _calibrate(oracle, psi, dim, threads, rng)
    # whole run ~ 8 x --cpu-seconds (120 s by default), split over the steps
    budget = max(0.05, 8.0 * args.cpu_seconds / max(1, args.steps + args.warmup))
    count = int(max(threads, budget / max(per_a, 1e-9)))
    times = []
    for s in range(args.warmup + args.steps):
        a = rng.integers(0, dim, count)
        t0 = time.perf_counter()
        oracle.sre_terms_list(psi, a, threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * count * dim / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"exact M2, N={N}: {desc}; complex64 amplitudes read in FP64",
                   "N": N, "n": 2, "step": f"{count} X-strings (bounded sample of the 2^{N})"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{count} X-strings per step, {args.steps} timed steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    import paper_2601_07824_gb300 as hm
    from paper_2601_07824_gb300 import _lib

    if args.only:
        if rank == 0:
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            print(json.dumps({"extra": extra_workloads(hm, dev, sms, args.only)}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    N = args.N
    psi_np, desc = workload_state(N)
    psi = torch.from_numpy(psi_np).to(dev)
    ctx = _lib.context(local)
    if args.shape:
        upw, tpt, R, lag = (int(v) for v in args.shape.split(","))
        ctx.set_twopass_shape(N, 2.0, upw, tpt, R, lag)
    path = {"cudacore": _lib.PATH_CUDACORE, "tensor": _lib.PATH_TENSOR, "auto": _lib.PATH_AUTO}[args.path]
    ctx.set_path(path)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    M = ln = None
    if args.xstrings > 0:
        alist = torch.arange(args.xstrings, dtype=torch.int64, device=dev)
        step = lambda: (hm.sre_terms(psi, 2.0, alist), None)  # noqa: E731
    elif world > 1:
        # one state split by X-string over the ranks (strong scaling): each rank evaluates its
        # slice, the ranks all-gather the per-chunk FP64 triples (NCCL) and combine them in order
        from paper_2601_07824_gb300 import shard
        step = lambda: shard.sre_sharded(psi, 2.0, path=path)  # noqa: E731
    else:
        step = lambda: hm.sre(psi, 2.0)  # noqa: E731
    for _ in range(args.warmup):
        M, ln = step()
    barrier()
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)  # evict L2 between steps (the state is smaller than L2)
            ev[s][0].record(stream)
            M, ln = step()
            ev[s][1].record(stream)
        barrier()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, world, dev)
    strings_per_step = 4.0 ** N if args.xstrings <= 0 else float(args.xstrings) * 2 ** N
    if args.xstrings > 0:
        M = ln = None
    sharded = world > 1 and args.xstrings <= 0
    # sharded: the ranks share one state's 4^N strings per step; otherwise every rank does its own
    value = (args.steps * strings_per_step / t_max) if sharded else aggregate_rate(world, args.steps, strings_per_step,
                                                                                   t_max)
    clocks = clk.summary()

    # end-to-end: the C-ABI host-buffer call, H2D copy from pinned memory inside the timed region
    e2e = None
    if not args.no_e2e and args.xstrings <= 0:
        host = torch.from_numpy(psi_np).pin_memory()
        if sharded:
            # every rank copies the state from pinned host memory, evaluates its slice, and the
            # combined result comes back to the host (sre_combine runs on host doubles)
            dst = torch.empty_like(psi)

            def e2e_step():
                dst.copy_(host, non_blocking=True)
                return shard.sre_sharded(dst, 2.0, path=path)
        else:
            def e2e_step():
                return hm.sre_host(host.numpy(), 2.0, device=local)
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": (args.steps * strings_per_step / te) if sharded
               else aggregate_rate(world, args.steps, strings_per_step, te), "unit": UNIT,
               "h2d_bytes_per_step": int(psi_np.nbytes), "d2h_bytes_per_step": 3 * 8 + 4}

    line = None
    if rank == 0:
        avg_s = t_local / args.steps
        mhz_max = 2070.0
        if args.path == "tensor" and 21 <= N <= 24:
            # tensor-core path (21 <= N <= 24): tensor-pipe FLOPs against the measured dense
            # fp16/bf16 peak (same rate for both types); smaller N runs the CUDA-core kernels
            peak, src = measured_peak("bf16_tflops", 1900.0)
            peak *= 1e12
            achieved = tensor_flops_per_string(N) * strings_per_step / avg_s
            roof = {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "note": f"{tensor_flops_per_string(N)} fp16 tensor FLOPs per Pauli string (blocks of K = "
                            f"128, 64, 128 on hi and lo operands); peak = {src} dense bf16 burst"}
        else:
            achieved = ops_per_string(N) * strings_per_step / avg_s
            peak = fp32_peak_ops(sm_count, mhz_max)
            roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": TRAFFIC.get((N, args.xstrings)),
                    "note": f"algorithmic FP32 ops (FMA = 1) = N + 7 = {ops_per_string(N)} per Pauli string "
                            f"(the kernel issues N + 4); peak = {sm_count} SMs x 128 lanes x {mhz_max:.0f} MHz; "
                            "kernel time = CUDA events around the call on its stream"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"exact M2, N={N}: {desc}; complex64; {args.path} Walsh-Hadamard path"
                                    + (f"; first {args.xstrings} X-strings only (profiling)" if args.xstrings > 0 else "")),
                       "N": N, "n": 2, "strings_per_step": strings_per_step,
                       "parallelism": (f"X-strings split over {world} ranks (chunk-aligned slices, NCCL all-gather "
                                       "of per-chunk FP64 sums)") if sharded else "one state per GPU",
                       "l2": f"state ({psi_np.nbytes >> 20} MiB) is smaller than L2: a 256 MiB buffer is written between steps",
                       "M2": M, "lost_norm": ln,
                       "twopass_shape": (dict(zip(("units_per_pass1_warp", "tiles_per_pass2_task", "ring_slots",
                                                   "xstrings_per_batch", "pass2_lag"), ctx.twopass_shape(N, 2.0)))
                                         if 16 <= N <= 24 else None)},
            "roofline": roof,
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": e2e,
        }
        if clocks.get("sm_mhz") and roof["bound"] == "alu":
            line["roofline"]["frac_at_measured_clock"] = achieved / fp32_peak_ops(sm_count, clocks["sm_mhz"])
        ref = golden_value("sre_brickwork_N20_depth10_seed2001") if (N == 20 and args.xstrings <= 0) else None
        if ref and M is not None:
            line["error"] = {"vs": "FP64 oracle on the same complex64 amplitudes (tests/golden/oracle_full_size.json)",
                             "M2_oracle": ref["M2"], "abs_dM2": abs(M - ref["M2"]),
                             "rel_dM2": abs(M - ref["M2"]) / max(1.0, abs(ref["M2"])),
                             "abs_dlost_norm": abs(ln - ref["lost_norm"])}
    if world > 1:
        dist.barrier()
    if rank == 0 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(psi_np, N, args.cpu_seconds)
        line["cpu_baseline"] = cb
    if rank == 0 and world == 1 and not args.no_lines and args.xstrings <= 0:
        line["lines"] = metric_lines(hm, dev, sm_count, flush)
    if rank == 0 and args.extra:
        line["extra"] = extra_workloads(hm, dev, sm_count)
    if rank == 0 and world == 1 and not args.no_new_rows:
        line["new_rows"] = new_rows_in_child()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def metric_lines(hm, dev, sm_count, flush, reps: int = 3, frac_log2: int = 3):
    """The metric's other configurations, after the headline, each with a warm-up, `reps` timed
    repeats (CUDA events; L2 flushed between repeats), clocks sampled during its repeats, a
    roofline fraction and an error against an independent value:
      * exact M2 at N = 22 (i.i.d. Gaussian state, seed 2201) on the FP32 CUDA-core path and
        on the tensor-core path, each timed on the X-strings [0, 2^22 / 2^frac_log2) through
        hadamag_sre_slice (the same kernels; a full sum takes 2^frac_log2 times as long);
        error: the same slice of |T>^22, whose per-X-string sums are 2^-|a| (closed form);
      * exact mana of N = 11 qutrits (Gaussian, seed 1101), whole sum; error against the
        stored FP64 oracle value, and the Strange-state closed form N log2(5/3)."""
    import math

    import numpy as np
    import torch
    from paper_2601_07824_gb300 import _lib, inputs
    out = {}
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        fn()  # warm-up (buffers sized, autotune)
        torch.cuda.synchronize(dev)
        ts, r = [], None
        with ClockSampler(dev.index or 0) as clk:
            for k in range(reps):
                flush.fill_(k & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = fn()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1) / 1e3)
        return ts, r, clk.summary()

    N = 22
    a1 = 2 ** (N - frac_log2)
    strings = float(a1) * 2 ** N
    psi = torch.from_numpy(inputs.gaussian_state(N, 2201, dtype=np.complex64)).to(dev)
    tst = torch.from_numpy(inputs.t_state_product(N, dtype=np.complex64)).to(dev)
    want_S2, want_S1 = 1.5 ** (N - frac_log2), float(a1)  # sum over a < a1 of 2^-|a|, and of 1
    tpeak, tsrc = measured_peak("bf16_tflops", 1900.0)
    res = {}
    for name, path in (("cudacore", _lib.PATH_CUDACORE), ("tensor", _lib.PATH_TENSOR)):
        try:
            ts, ch, clocks = timed(lambda p=path: hm.sre_slice(psi, 2.0, 0, a1, path=p))
            t = statistics.median(ts)
            rate = strings / t
            tch = hm.sre_slice(tst, 2.0, 0, a1, path=path).cpu().numpy()
            S2, S1 = float(np.sum(tch[:, 0])), float(np.sum(tch[:, 1]))
            d = {"value": rate, "unit": UNIT, "s_per_call": t, "s_all": ts, "clocks": clocks,
                 "workload": f"exact M2 sums, N = 22 Gaussian (seed 2201), X-strings [0, 2^{N - frac_log2}) of "
                             f"2^{N} ({strings:.3e} Pauli strings per call), {name} path",
                 "S2_slice": float(np.sum(ch[:, 0].cpu().numpy())),
                 "error": {"vs": "closed form on |T>^22 over the same slice: S2 = 1.5^19, S1 = 2^19",
                           "rel_dS2": abs(S2 / want_S2 - 1.0), "rel_dS1": abs(S1 / want_S1 - 1.0),
                           "equiv_abs_dM2": abs(S2 / want_S2 - 1.0) / math.log(2.0)}}
            if name == "tensor":
                d["roofline"] = {"bound": "tensor", "unit": "TFLOP/s", "peak": tpeak, "peak_source": f"{tsrc} bf16 burst",
                                 "achieved": tensor_alg_flops_per_string(N) * rate / 1e12,
                                 "frac": tensor_alg_flops_per_string(N) * rate / (tpeak * 1e12),
                                 "count": f"{tensor_alg_flops_per_string(N)} FLOPs per Pauli string (16 N, H_16 "
                                          "blocks on hi/lo operands)",
                                 "frac_issued_blocks": tensor_flops_per_string(N) * rate / (tpeak * 1e12),
                                 "issued": f"{tensor_flops_per_string(N)} FLOPs per Pauli string (blocks K = 128, 64, "
                                           "128 on hi and lo)"}
            else:
                pk = fp32_peak_ops(sm_count, 2070.0)
                d["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": pk / 1e12,
                                 "achieved": ops_per_string(N) * rate / 1e12, "frac": ops_per_string(N) * rate / pk,
                                 "count": f"N + 7 = {ops_per_string(N)} FP32 ops per Pauli string"}
            res[name] = d
            out[f"sre_N22_{name}"] = d
        except Exception as e:  # noqa: BLE001
            out[f"sre_N22_{name}"] = {"error": str(e)}
    if "cudacore" in res and "tensor" in res:
        out["sre_N22_tensor_over_cudacore"] = res["tensor"]["value"] / res["cudacore"]["value"]
        out["sre_N22_rel_dS2_tensor_vs_cudacore"] = abs(res["tensor"]["S2_slice"] / res["cudacore"]["S2_slice"] - 1.0)
    del psi, tst

    try:
        Nq = 11
        q = torch.from_numpy(inputs.gaussian_state(Nq, 1101, d=3, dtype=np.complex64)).to(dev)
        ts, r, clocks = timed(lambda: hm.mana(q))
        t = statistics.median(ts)
        pts = 9.0 ** Nq
        pk = fp32_peak_ops(sm_count, 2070.0)
        d = {"value": pts / t, "unit": "phase-space points/s", "s_per_call": t, "s_all": ts, "clocks": clocks,
             "workload": "exact mana, N = 11 qutrits, Gaussian (seed 1101), complex64, all 9^11 points",
             "mana": r[0],
             "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": pk / 1e12,
                          "achieved": mana_ops_per_point(Nq) * pts / t / 1e12,
                          "frac": mana_ops_per_point(Nq) * pts / t / pk,
                          "count": f"4.7 N + 8 = {mana_ops_per_point(Nq):.1f} FP32 ops per point"}}
        ref = golden_value("mana_gaussian_N11_seed1101")
        strange = hm.mana(torch.from_numpy(inputs.strange_product(Nq, dtype=np.complex64)).to(dev))[0]
        d["error"] = {"strange_closed_form_abs_dmana": abs(strange - Nq * math.log2(5.0 / 3.0))}
        if ref:
            d["error"].update({"vs": "FP64 oracle (tests/golden/oracle_full_size.json)", "mana_oracle": ref["mana"],
                               "abs_dmana": abs(r[0] - ref["mana"])})
        out["mana_N11"] = d
    except Exception as e:  # noqa: BLE001
        out["mana_N11"] = {"error": str(e)}
    return out


NEW_ROWS = ("batched_64_fwd_bwd", "ti_N20_L10", "mana_mixed_N8_of_10", "sre_even_sector_N20_u1", "mana_qudit_d5_N6",
            "mana_grad_d3_N9")


def new_rows_in_child(timeout_s: float = 480.0):
    """Times the Algorithm 3 / Algorithm 6, even-sector, qudit and mana-gradient workloads (the
    --extra lines of those rows) in a separate process, after the headline measurement: a CUDA
    error there cannot reach the headline's context, and a time limit bounds it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--only", ",".join(NEW_ROWS)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout_s:.0f} s"}
    for ln in reversed(r.stdout.strip().splitlines()):
        try:
            return json.loads(ln)["extra"]
        except (ValueError, KeyError):
            continue
    return {"error": f"exit {r.returncode}: " + (r.stderr.strip().splitlines() or [""])[-1][:200]}


def extra_workloads(hm, dev, sm_count, only: str = ""):
    """The other configurations, one timed call each (not part of the headline value); with
    `only`, just the workload of that name."""
    import numpy as np
    import torch
    from paper_2601_07824_gb300 import _lib, inputs
    out = {}

    def timed(fn, reps=1, warm=True):
        if warm:
            fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) / reps, r

    wanted = set(only.split(",")) if only else None

    def guard(key, fn):
        if wanted is not None and key not in wanted:
            return
        try:
            out[key] = fn()
        except Exception as e:  # noqa: BLE001
            out[key] = {"error": str(e)}

    tpeak, tsrc = measured_peak("bf16_tflops_sustained", 1700.0)

    # exact M2 at N = 22 (Gaussian state): FP32 CUDA-core path vs tensor-core path
    psi22 = torch.from_numpy(inputs.gaussian_state(22, 2201, dtype=np.complex64)).to(dev) \
        if wanted is None or wanted & {"sre_N22_cudacore", "sre_N22_tensor"} else None
    res = {}
    for name, p in (("cudacore", _lib.PATH_CUDACORE), ("tensor", _lib.PATH_TENSOR)):
        def run22(p=p, name=name):
            dt, r = timed(lambda: hm.sre(psi22, 2.0, path=p), warm=False)
            rate = 4.0 ** 22 / dt
            d = {"strings_per_s": rate, "s": dt, "M2": r[0], "lost_norm": r[1]}
            if name == "tensor":
                d["tensor_frac_of_sustained_peak"] = tensor_flops_per_string(22) * rate / (tpeak * 1e12)
                d["peak_source"] = tsrc
            else:
                d["alu_frac"] = ops_per_string(22) * rate / fp32_peak_ops(sm_count, 2070.0)
            res[name] = d
            return d
        guard(f"sre_N22_{name}", run22)
    if "cudacore" in res and "tensor" in res:
        out["sre_N22_tensor_over_cudacore"] = res["tensor"]["strings_per_s"] / res["cudacore"]["strings_per_s"]
        out["sre_N22_rel_dM2"] = abs(res["tensor"]["M2"] - res["cudacore"]["M2"]) / res["cudacore"]["M2"]
    del psi22

    # exact mana of an N = 11 qutrit Gaussian state
    def mana11():
        q = torch.from_numpy(inputs.gaussian_state(11, 1101, d=3, dtype=np.complex64)).to(dev)
        dt, r = timed(lambda: hm.mana(q), reps=3)
        return {"points_per_s": 9.0 ** 11 / dt, "s": dt, "mana": r[0]}
    guard("mana_N11", mana11)

    # Monte-Carlo M2 at N = 28 with 4096 sampled X-strings (plus the exact a = 0 row)
    def mc28():
        psi = torch.from_numpy(inputs.gaussian_state(28, 2801, dtype=np.complex64)).to(dev)
        dt, r = timed(lambda: hm.sre_mc(psi, 4096, 2802), warm=False)
        return {"strings_per_s": 4097 * 2.0 ** 28 / dt, "s": dt, "M2": r[0], "stderr": r[1],
                "hbm_state_reads_GBps": 4097 * 2 * psi.numel() * 8 / dt / 1e9}
    guard("mc_N28", mc28)

    # batched forward + backward: 64 states, N uniform in 10..18, one persistent launch, against
    # a loop of single-state calls over the same states (forward + backward, and forward only)
    def batched():
        Ns, states = inputs.batched_ladder_states(64, 10, 18, 8, seed=4001)
        ts = [torch.from_numpy(x).to(dev) for x in states]
        strings = sum(4.0 ** n for n in Ns)
        dt, _ = timed(lambda: hm.sre_batched(ts, want_grad=True), reps=2)
        dl, _ = timed(lambda: [hm.sre_grad(t) for t in ts], reps=2)
        df, _ = timed(lambda: hm.sre_batched(ts, want_grad=False), reps=2)
        dlf, _ = timed(lambda: [hm.sre(t, 2.0) for t in ts], reps=2)
        return {"strings_per_s": strings / dt, "s": dt, "states": len(Ns),
                "loop_fwd_bwd_s": dl, "speedup_over_loop": dl / dt,
                "fwd_only_s": df, "loop_fwd_only_s": dlf, "fwd_speedup_over_loop": dlf / df}
    guard("batched_64_fwd_bwd", batched)

    # thermodynamic-integration M2 (Algorithm 3) on the N = 20 brickwork state: L = 10 chains,
    # 200 burn-in + 2000 recorded steps, one per-X evaluation per chain and step
    def ti20():
        psi = torch.from_numpy(inputs.brickwork_haar(20, 10, seed=2001, dtype=np.complex64)).to(dev)
        L, n_s, burn = 10, 2000, 200
        dt, r = timed(lambda: hm.sre_ti(psi, L, n_s, 2002, burn_in=burn))
        evals = L * (n_s + burn + 1)
        rate = evals * 2.0 ** 20 / dt
        return {"strings_per_s": rate, "alu_frac": ops_per_string(20) * rate / fp32_peak_ops(sm_count, 2070.0),
                "evaluations_per_s": evals / dt,
                "steps_per_s": (n_s + burn) / dt, "s": dt, "M2": r[0], "dM2": r[1], "L": L, "n_s": n_s,
                "burn_in": burn}
    guard("ti_N20_L10", ti20)

    # mixed-state mana (Algorithm 6's W) of the Sec. 3.3.3 example: the 8-qutrit marginal (sites
    # 0..7) of a 10-qutrit brick-wall Haar state of depth 3; rho is 9^8 complex64 = 344 MB
    # (larger than L2), read once per call
    def mixed8():
        psi = torch.from_numpy(inputs.brickwork_haar(10, 3, seed=1001, d=3, dtype=np.complex64)).to(dev)
        keep = list(range(8))
        t_rdm, rho = timed(lambda: hm.reduced_density_matrix(psi, keep), reps=3)
        dt, r = timed(lambda: hm.mana_mixed(rho), reps=3)
        pts = 9.0 ** 8
        hbm, hsrc = measured_peak("hbm_gbs", 6800.0)
        return {"points_per_s": pts / dt, "s": dt, "mana": r[0], "rho_read_GBps": pts * 8 / dt / 1e9,
                "hbm_frac": pts * 8 / dt / 1e9 / hbm, "peak_source": hsrc,
                "rdm_s": t_rdm, "rdm_tflops": 8.0 * 9.0 ** 8 * 3.0 ** 2 / t_rdm / 1e12}
    guard("mana_mixed_N8_of_10", mixed8)

    # even-weight X-sectors only (U(1) state at half filling, N = 20): half the work of the full sum
    def even20():
        psi = torch.from_numpy(inputs.u1_state(20, 10, 2003, dtype=np.complex64)).to(dev)
        t_full, rf = timed(lambda: hm.sre(psi, 2.0))
        t_even, re_ = timed(lambda: hm.sre_even_sector(psi, 2.0))
        return {"full_s": t_full, "even_s": t_even, "speedup": t_full / t_even, "M2_full": rf[0], "M2_even": re_[0],
                "even_strings_per_s": 2.0 ** 39 / t_even,
                "alu_frac": ops_per_string(20) * 2.0 ** 39 / t_even / fp32_peak_ops(sm_count, 2070.0)}
    guard("sre_even_sector_N20_u1", even20)

    # odd-prime qudits: mana at d = 5, N = 6, and the qutrit mana gradient at N = 9
    def qudit5():
        psi = torch.from_numpy(inputs.gaussian_state(6, 501, d=5, dtype=np.complex64)).to(dev)
        dt, r = timed(lambda: hm.mana_qudit(psi, 5), reps=3)
        # N d complex multiply-adds (4 FMAs) per point in the direct d-point sums
        return {"points_per_s": 25.0 ** 6 / dt, "s": dt, "mana": r[0],
                "alu_frac": 4 * 6 * 5 * 25.0 ** 6 / dt / fp32_peak_ops(sm_count, 2070.0)}
    guard("mana_qudit_d5_N6", qudit5)

    def grad3():
        psi = torch.from_numpy(inputs.gaussian_state(9, 901, d=3, dtype=np.complex64)).to(dev)
        dt, r = timed(lambda: hm.mana_grad(psi, 3), reps=3)
        # two transforms of N d complex multiply-adds (4 FMAs each) per point
        return {"points_per_s": 9.0 ** 9 / dt, "s": dt, "mana": r[0],
                "alu_frac": 2 * 4 * 9 * 3 * 9.0 ** 9 / dt / fp32_peak_ops(sm_count, 2070.0)}
    guard("mana_grad_d3_N9", grad3)
    return out


if __name__ == "__main__":
    main()
