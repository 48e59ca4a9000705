"""Benchmark of the direct-summation hot path on one (or N replica) GB300 GPUs.

Workload: an N = 2^20 Plummer sphere with log-normal masses (sigma 0.5,
total mass 1), eps = 4/N, seed 1003; one step = one full evaluation of
acceleration, jerk and potential of all N i-particles against all N
j-particles in mixed precision (the j images are rebuilt from the FP64 state
by the device predictor, then the force kernel and, if the launch splits j,
the reduction).  Metric: pair interactions per second (N^2 per step, Eq. 3's
convention), with the k = 60 GFLOP/s figure and the fraction of FP32 peak.

Alongside: the FP64 GPU path on an i-subset, the eps = 0 / r_min = 1e-6
guarded variant, the end-to-end rate through the host-pointer C ABI (uploads
and result downloads inside the timed region), the FP64 CPU oracle on a
bounded i-subset (which also gives the per-particle error of the mixed
results), SM clocks sampled during the timed region, and the roofline entry.

The default line also carries the other workloads as sub-records ("small",
"block", "ensemble", "adjoint"), each with its own clock sample and a parity
summary against the oracle; --no-sub leaves them out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--no-sub]
  python bench.py --workload small|block|ensemble|adjoint   (the other workloads, one JSON line each)

Multi-GPU runs (torchrun, one rank per GPU) are replicas by default: every
rank evaluates its own copy of the workload; value = all ranks' pairs / max
time.  --parallel jsplit shares one evaluation among the ranks instead (each
sums its part of the j tiles; the partial sums are all-gathered over NCCL and
added in part order): value = N^2 per step / max time, strong scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair interactions/s (acc+jerk+pot) mixed vs FP64 GPU at <=1e-6 rel force err"
UNIT = "pair interactions/s"
N_DEFAULT = 1 << 20
L2_FLUSH_BYTES = 256 << 20


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("force_mixed.cu", "pair_mixed.cuh", "tma.cuh", "kirin_internal.cuh"):
        with open(os.path.join(ROOT, "paper_0707_0438_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            # a region shorter than the sampling period still gets its first sample
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                self.tmp.flush()
                if os.path.getsize(self.tmp.name) > 0:
                    break
                time.sleep(0.02)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        with open(self.tmp.name) as f:
            rows = [r.split(",") for r in f.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


def replica_rate(local_seconds: float, units_per_step: float, steps: int, world: int, dist=None, device=None):
    """Whole-job rate of `world` replicas: every rank did `steps` steps of `units_per_step`;
    the job took as long as the slowest rank (MAX over ranks).  Returns (rate, max_seconds)."""
    t_max = float(local_seconds)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return world * units_per_step * steps / t_max, t_max


def _fp32_peak_tflops(nsm: int, mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return nsm * 128 * 2 * mhz * 1e6 / 1e12


def _sub_roofline(rate, k, note, device=0):
    """Roofline of a secondary workload: its pair rate x k flops per pair against the FP32 CUDA-core
    peak (the headline's denominator), over the whole run it reports."""
    import torch
    props = torch.cuda.get_device_properties(device)
    peaks, src = _peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = _fp32_peak_tflops(props.multi_processor_count, f_max)
    achieved = k * rate / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "peak_note": f"FP32 CUDA-core peak at {f_max:.0f} MHz ({src}); k={k} flops per pair: {note}"}


def _time_oracle_sample(p, k_i, seed):
    import oracle
    il = _subset(p.n, k_i, seed)
    t0 = time.perf_counter()
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    dt = time.perf_counter() - t0
    return il, ref, dt, oracle.num_threads()


def _subset(n, k, seed):
    from paper_0707_0438_gb300 import workloads
    return workloads.i_subset(n, k, seed)


def _calibrated_oracle_size(p, target_s):
    """i-subset size for about target_s seconds of oracle time on this host."""
    k0 = min(p.n, 256)
    _, _, dt, _ = _time_oracle_sample(p, k0, 99)
    per_i = max(dt / k0, 1e-7)
    return int(max(64, min(p.n, target_s / per_i)))


def _host_cpu() -> dict:
    """The host CPU the oracle timing ran on: model (from /proc/cpuinfo) and the cores this process may use."""
    model = platform.machine()
    parts = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1"}
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name":
                model = line.split(":", 1)[1].strip()
                break
            if key == "cpu part":
                part = line.split(":", 1)[1].strip()
                model = f"{platform.machine()} {parts.get(part, 'CPU part ' + part)}"
                break
    except OSError:
        pass
    try:
        affinity = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        affinity = os.cpu_count()
    return {"cpu": model, "affinity_cores": affinity}


def run_reference(args):
    """The CPU oracle on the host cores (the reference arm), bounded sample per step."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from paper_0707_0438_gb300 import workloads
    n = args.n
    p = workloads.config_large(n)
    per_step_s = max(1.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    k_i = _calibrated_oracle_size(p, per_step_s)
    for w in range(args.warmup):
        _time_oracle_sample(p, max(16, k_i // 8), 1000 + w)
    times = []
    threads = 1
    for s in range(args.steps):
        _, _, dt, threads = _time_oracle_sample(p, k_i, 2000 + s)
        times.append(dt)
    total = sum(times)
    value = k_i * n * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(n, "oracle"),
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                              "sample": f"{k_i} i x {n} j per step (FP64 CPU oracle, OpenMP over i)"}, **_host_cpu()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(n, precision):
    return {"workload": f"plummer N={n} lognormal masses (sigma 0.5), eps=4/N, seed 1003: one full "
                        f"acc+jerk+pot evaluation of all i vs all j",
            "n": n, "eps": 4.0 / n, "precision": precision, "global_batch": n, "parallelism": "replicas",
            "l2": "256 MiB buffer written between timed steps (flushes L2)"}


def run_native(args):
    import torch

    from paper_0707_0438_gb300 import abi, metrics, workloads

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n = args.n
    p = workloads.config_large(n)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    m_d = torch.tensor(p.m, device=dev)
    x_d = torch.tensor(p.x, device=dev)
    v_d = torch.tensor(p.v, device=dev)
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev)
    jerk = torch.empty_like(acc)
    pot = torch.empty(n, dtype=torch.float64, device=dev)

    k = abi.Kirin(n, p.eps, precision="mixed", device=local, stream=sp)
    k.set_j_particles_dev(m_d, x_d, v_d)
    k.sync()
    from paper_0707_0438_gb300 import autotune
    tuned = autotune.install(k, n, torch.cuda.get_device_name(dev), "mixed")
    if args.launch:  # a fixed launch shape (profiling the bench's shape at another size)
        k.set_launch(*args.launch)
        tuned = False
    # --parallel jsplit: the ranks share one evaluation, each summing its part of the j tiles; the partial
    # sums are all-gathered over NCCL and added in part order (every rank holds the result)
    jsplit_mode = world > 1 and args.parallel == "jsplit"
    if jsplit_mode:
        from paper_0707_0438_gb300 import jsplit
        k.set_j_partition(rank, world, jsplit.TorchAllGather(device=dev))
    groups, n_split = k.get_launch(n)
    launches_per_step = 2 + (1 if n_split > 1 else 0)  # predictor/pack, force, split reduction

    def step(kk):
        kk.predict(0.0)  # rebuild the j images from the FP64 state on the device
        kk.compute_forces_dev(None, acc, jerk, pot)

    def timed(kk, steps, warmup, dn=None):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step(kk)
            kk.sync()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize(dev)
            for s in range(steps):
                flush.zero_()  # on `stream`, outside the events
                evs[s][0].record(stream)
                step(kk)
                evs[s][1].record(stream)
            kk.sync()
            torch.cuda.synchronize(dev)
        per_step.clear()
        per_step.extend(a.elapsed_time(b) for a, b in evs)
        return sum(per_step) / 1e3

    # ---- headline: mixed precision, full evaluation ----
    per_step = []
    with ClockSampler(local) as clk:
        t_mixed = timed(k, args.steps, args.warmup)
    step_ms = {"best": min(per_step), "median": float(np.median(per_step)), "worst": max(per_step)}
    clocks = clk.summary()
    pairs_per_step = float(n) * float(n)
    value, t_max = replica_rate(t_mixed, pairs_per_step, args.steps, world, dist, dev)
    if jsplit_mode:  # one shared evaluation per step, not one per rank
        value /= world
    ms_per_step = 1e3 * t_max / args.steps
    res_mixed = (acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy())

    if rank != 0 and not jsplit_mode:
        k.close()
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    extra = {}
    # ---- eps = 0 with the r_min = 1e-6 guard (Sect. 3.3.1) ----
    k.set_params(0.0, 1.0, 1e-6, "mixed")
    t_g = timed(k, max(1, args.steps // 2), 1)
    extra["eps0_rmin_guard"] = {"value": pairs_per_step * max(1, args.steps // 2) / t_g, "unit": UNIT,
                                "ms_per_step": 1e3 * t_g / max(1, args.steps // 2)}
    k.set_params(p.eps, 1.0, 0.0, "mixed")

    # ---- FP64 GPU path on an i-subset (all j) ----
    n_sub = min(n, 16384)
    il_sub = torch.tensor(workloads.i_subset(n, n_sub, 17), device=dev)
    acc_s = torch.empty((n_sub, 3), dtype=torch.float64, device=dev)
    jerk_s, pot_s = torch.empty_like(acc_s), torch.empty(n_sub, dtype=torch.float64, device=dev)
    k.set_params(p.eps, 1.0, 0.0, "fp64")
    with torch.cuda.stream(stream):
        k.compute_forces_dev(il_sub, acc_s, jerk_s, pot_s)  # warm-up
        k.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 2
        for _ in range(reps):
            k.compute_forces_dev(il_sub, acc_s, jerk_s, pot_s)
        e1.record(stream)
        k.sync()
    t64 = e0.elapsed_time(e1) / 1e3 / reps
    fp64_rate = n_sub * float(n) / t64
    fp64_res = (acc_s.cpu().numpy(), jerk_s.cpu().numpy(), pot_s.cpu().numpy())
    sub_idx = il_sub.cpu().numpy()
    mixed_vs_fp64 = {q: metrics.summary(f(a[sub_idx], b)) for q, f, a, b in (
        ("acc", metrics.rel_err_vec, res_mixed[0], fp64_res[0]),
        ("jerk", metrics.rel_err_vec, res_mixed[1], fp64_res[1]),
        ("pot", metrics.rel_err_scalar, res_mixed[2], fp64_res[2]))}
    extra["fp64"] = {"value": fp64_rate, "unit": UNIT, "sample": f"{n_sub} i x {n} j",
                     "mixed_speedup": value / world / fp64_rate, "mixed_vs_fp64_rel_err": mixed_vs_fp64}
    k.set_params(p.eps, 1.0, 0.0, "mixed")

    # ---- end to end through the host-pointer C ABI ----
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    hm, hx, hv = pin((n,)), pin((n, 3)), pin((n, 3))
    hm[:], hx[:], hv[:] = p.m, p.x, p.v
    ha, hj, hp = pin((n, 3)), pin((n, 3)), pin((n,))
    import ctypes
    L = k.lib
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def e2e_step():
        rc = L.kirin_set_j_particles(k.ctx, 0, n, dp(hm), dp(hx), dp(hv), None, None, None)
        rc = rc or L.kirin_compute_forces(k.ctx, 0, None)
        rc = rc or L.kirin_get_acc_jerk_pot(k.ctx, dp(ha), dp(hj), dp(hp))
        if rc:
            raise abi.KirinError(rc, "e2e step")

    e2e_step()
    e_steps = max(1, args.steps // 2)
    t_e2e = 0.0
    for _ in range(e_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        t_e2e += time.perf_counter() - t0
    e2e = {"value": pairs_per_step * e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(hm.nbytes + hx.nbytes + hv.nbytes),
           "d2h_bytes_per_step": int(ha.nbytes + hj.nbytes + hp.nbytes),
           "ms_per_step": 1e3 * t_e2e / e_steps}
    k.close()
    if rank != 0:  # jsplit: the other ranks took part in every exchanging call above
        dist.barrier()
        dist.destroy_process_group()
        return

    # ---- CPU oracle on a bounded sample; also the error of the mixed results ----
    cpu = None
    if not args.no_cpu:
        k_i = _calibrated_oracle_size(p, args.cpu_seconds)
        il, ref, dt, threads = _time_oracle_sample(p, k_i, 3)
        errs = {q: metrics.summary(f(a[il], b)) for q, f, a, b in (
            ("acc", metrics.rel_err_vec, res_mixed[0], ref[0]),
            ("jerk", metrics.rel_err_vec, res_mixed[1], ref[1]),
            ("pot", metrics.rel_err_scalar, res_mixed[2], ref[2]))}
        cpu = dict({"value": k_i * float(n) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                    "sample": f"{k_i} random i x all {n} j, FP64 CPU oracle (OpenMP over i), {dt:.1f} s"},
                   **_host_cpu())
        extra["mixed_vs_oracle_rel_err"] = errs

    # ---- roofline of the force kernel (FP32 CUDA-core pipe) ----
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = _peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = _fp32_peak_tflops(props.multi_processor_count, f_max)
    achieved = 60.0 * pairs_per_step / (t_mixed / args.steps) / 1e12  # Eq. 3, k = 60
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            tr = json.load(f).get("k_force_mixed", {})
        # the counters hold for the captured source, size and launch shape only
        if (tr.get("source_sha") == _kernel_source_sha() and tr.get("n") == n
                and tr.get("launch") == [groups, n_split]):
            traffic = tr.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "peak_note": f"FP32 CUDA-core peak {props.multi_processor_count} SMs x 128 x 2 x {f_max:.0f} MHz "
                         f"(max SM clock, {peak_src}); achieved counts k=60 flops per pair (Eq. 3)"}
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / _fp32_peak_tflops(props.multi_processor_count, clocks["sm_mhz"])
    # measured FMA rates of this GPU (independent FMA chains on every SM), for context
    try:
        fma = {kind: abi.measure_fma_rate(kind, local) / 1e12 for kind in ("fp32", "fp32x2", "fp64")}
        roof["measured_fma_tflops"] = fma
        roof["frac_of_measured_fp32x2"] = achieved / fma["fp32x2"]
        # the FP64 kernel: ~40 FP64 flops per interaction (30 arithmetic + the library rsqrt)
        extra["fp64"]["frac_of_measured_fp64_at_40_flops"] = 40.0 * fp64_rate / (fma["fp64"] * 1e12)
    except abi.KirinError:
        pass

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "step_ms_rank0": step_ms, "higher_is_better": True,
        "scaling": "strong" if jsplit_mode else "weak",
        "vs_baseline": None, "dtype": "f32 pair math, double-single positions, f64 results", "data": "synthetic",
        "config": dict(_config(n, "mixed"), launch={"groups": groups, "n_split": n_split,
                                                     "from": "fixed (--launch)" if args.launch else
                                                     "tuned table" if tuned else "cost model"},
                       parallelism=f"j partition over {world} GPUs (NCCL all-gather of the partial sums)"
                       if jsplit_mode else "replicas"),
        "gflops_k60": 60.0 * value / 1e9, "gflops_k38_equiv": 38.0 * value / 1e9,
        "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
        "roofline": roof, "cpu_baseline": cpu,
    }
    line.update(extra)
    if world == 1 and not args.no_sub:
        line.update(secondary_workloads(local))
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def secondary_workloads(device=0):
    """The other workloads, each with its own clock sample and oracle parity summary, as sub-records of
    the default line: small (1 + 10 shared Hermite steps, N = 1024), block (block-step Hermite, N = 65536,
    to t = 1/8, mixed and FP64), ensemble (512 clusters, 64 leapfrog steps) and adjoint (forward +
    backward of the 64-step differentiable leapfrog).  A workload that fails records its error."""
    out = {}
    for name, fn in (("small", lambda: measure_small(20, 3, device)),
                     ("block", lambda: measure_block(65536, 0.125, 0.125, True, 0.125, device)),
                     ("ensemble", lambda: measure_ensemble(3, True, device)),
                     ("adjoint", lambda: measure_adjoint(3, 1, device))):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # keep the headline line; say what failed
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def _line(metric, value, unit, steps, warmup, seconds, workload, extra, higher=True, dtype="f32 pair math"):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * seconds / max(steps, 1), "higher_is_better": higher, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": {"workload": workload}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _errs(got, ref):
    """Per-particle relative errors (median, max) of (acc, jerk, pot) or (acc, pot) against the oracle."""
    from paper_0707_0438_gb300 import metrics
    names = ("acc", "jerk", "pot") if len(got) == 3 else ("acc", "pot")
    out = {}
    for name, g, r in zip(names, got, ref):
        f = metrics.rel_err_scalar if name == "pot" else metrics.rel_err_vec
        e = metrics.summary(f(g, r))
        out[name] = {"median": float(f"{e['median']:.3g}"), "max": float(f"{e['max']:.3g}")}
    return out


def _rel_diff(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


SMALL_WORKLOAD = "plummer N=1024 eps=1/256 seed 1001: 1 + 10 shared Hermite steps dt=1/1024 (11 acc+jerk+pot evaluations)"


def measure_small(steps, warmup, device=0):
    """N = 1024, eps = 1/256: one full evaluation and 10 shared Hermite steps dt = 1/1024, mixed and FP64.
    Parity: the first evaluation (all i) and the state after the 10 steps against the oracle's."""
    import torch

    import oracle
    from oracle import hermite
    from paper_0707_0438_gb300 import abi, workloads
    p = workloads.config_small(1024)
    ref0 = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps)
    x_ref, v_ref, _, _, _ = hermite.shared_steps(p.m, p.x, p.v, p.eps, 1.0 / 1024, 10)
    res = {}
    for precision in ("mixed", "fp64"):
        with abi.Kirin(p.n, p.eps, precision=precision, device=device) as k:
            k.set_j_particles(p.m, p.x, p.v)
            first = k.forces()
            for _ in range(warmup):
                k.hermite_init(0.0)
                k.hermite_shared_run(1.0 / 1024, 10)
            torch.cuda.synchronize()
            runs = 0
            with ClockSampler(device) as clk:
                t0 = time.perf_counter()
                while runs < steps or time.perf_counter() - t0 < 0.5:  # at least half a second of runs
                    k.hermite_init(0.0)
                    k.hermite_shared_run(1.0 / 1024, 10)  # enqueued back to back, one synchronisation
                    runs += 1
                dt = time.perf_counter() - t0
            # every timed run went on from where the last one ended: the parity run starts afresh
            k.set_j_particles(p.m, p.x, p.v)
            k.hermite_init(0.0)
            k.hermite_shared_run(1.0 / 1024, 10)
            st = k.get_state()
        res[precision] = {"value": 11 * p.n * p.n * runs / dt, "ms_per_run": 1e3 * dt / runs, "runs": runs,
                          "clocks": clk.summary(),
                          "parity": {"first_evaluation_vs_oracle": _errs(first, ref0),
                                     "x_after_10_steps_rel_diff": _rel_diff(st["x"], x_ref),
                                     "v_after_10_steps_rel_diff": _rel_diff(st["v"], v_ref)}}
    m = res["mixed"]
    roof = _sub_roofline(m["value"], 60, "acc+jerk+pot (Eq. 3), init and steps included", device)
    return dict(m, unit=UNIT, workload=SMALL_WORKLOAD, fp64=res["fp64"], roofline=roof)


def run_small(args):
    r = measure_small(args.steps, args.warmup)
    _line("pair interactions/s, 1 evaluation + 10 shared Hermite steps", r["value"], UNIT, r["runs"],
          args.warmup, r["ms_per_run"] * r["runs"] / 1e3, SMALL_WORKLOAD,
          {k: v for k, v in r.items() if k not in ("value", "unit", "workload")})


def _block_workload(n, t_end):
    return f"plummer N={n} eps=1e-3 seed 1002, Hermite block steps eta=0.01, levels 2^-20..2^-3, to t={t_end:g}"


def measure_block(n=65536, t_end=0.125, fp64_t_end=0.125, host_loop=True, histogram_t_end=0.125, device=0):
    """N = 65536, eps = 1e-3, block-step Hermite (eta 0.01, levels 2^-20..2^-3) to t = 1/8, mixed (the
    device-driven loop, and the host-driven one for comparison) and FP64.  Value: (initial N^2 +
    every block's n_i N) / wall time of hermite_init + hermite_run.  Parity: the start evaluation of
    256 sampled i against the oracle, mixed against FP64 final positions, ΔE/E of each run, and
    how far the device- and host-driven loops end apart."""
    import torch

    import oracle
    from paper_0707_0438_gb300 import abi, autotune, metrics, workloads
    p = workloads.config_block(n)
    gpu = torch.cuda.get_device_name(device)
    il = workloads.i_subset(n, 256, seed=9)
    out, final, start = {}, {}, None
    runs = [("mixed", "mixed", t_end, True)]
    if host_loop:
        runs.append(("mixed_host_loop", "mixed", t_end, False))
    if fp64_t_end:
        runs.append(("fp64", "fp64", fp64_t_end, True))
    for name, precision, te, device_loop in runs:
        with abi.Kirin(n, p.eps, precision=precision, device=device) as k:
            k.set_j_particles(p.m, p.x, p.v)
            if precision == "mixed":
                autotune.install(k, n, gpu, "mixed")
                if start is None:
                    start = k.forces(il)
            k.set_device_loop(device_loop)
            kin0, pot0 = k.energy()
            torch.cuda.synchronize()
            with ClockSampler(device) as clk:
                t0 = time.perf_counter()
                k.hermite_init(0.0)
                steps, pairs = k.hermite_run(te)
                dt = time.perf_counter() - t0
            kin1, pot1 = k.energy()
            final[name] = k.get_state()
        out[name] = {"t_end": te, "block_steps": steps, "pairs": pairs + float(n) * n, "seconds": dt,
                     "value": (pairs + float(n) * n) / dt, "unit": UNIT, "device_loop": device_loop,
                     "dE_E": metrics.energy_error(kin0 + pot0, kin1 + pot1), "clocks": clk.summary()}
    ref = oracle.acc_jerk_pot(p.m, p.x, p.v, p.eps, i_idx=il)
    parity = {"start_evaluation_256_i_vs_oracle": _errs(start, ref)}
    if "fp64" in final and fp64_t_end == t_end:
        parity["x_final_mixed_vs_fp64_rel_diff"] = _rel_diff(final["mixed"]["x"], final["fp64"]["x"])
    if "mixed_host_loop" in final:
        # the two loops give the same bits under one fixed launch shape (the GPU tests check that); here
        # each takes its shapes from the launch table, the device loop per block-size class and the host
        # loop per block, so they sum in different orders and agree to rounding
        parity["x_final_device_vs_host_loop_rel_diff"] = _rel_diff(final["mixed"]["x"], final["mixed_host_loop"]["x"])
        parity["same_block_steps_device_and_host_loop"] = bool(out["mixed"]["block_steps"] ==
                                                              out["mixed_host_loop"]["block_steps"])
    res = dict(out["mixed"], workload=_block_workload(n, t_end), parity=parity)
    for name in ("mixed_host_loop", "fp64"):
        if name in out:
            res[name] = out[name]
    if "fp64" in out:
        res["mixed_vs_fp64_speedup"] = out["mixed"]["value"] / out["fp64"]["value"]
    if histogram_t_end:
        # active-block sizes of the mixed run, stepped from the host (the same launch table as the
        # host-driven timed run): blocks per power-of-two size bucket and their share of the pairs
        hist = {}
        with abi.Kirin(n, p.eps, precision="mixed", device=device) as k:
            k.set_j_particles(p.m, p.x, p.v)
            autotune.install(k, n, gpu, "mixed")
            k.hermite_init(0.0)
            while True:
                _, n_act = k.hermite_block_step(histogram_t_end)
                if n_act == 0:
                    break
                h = hist.setdefault(1 << int(math.log2(n_act)), [0, 0.0])
                h[0] += 1
                h[1] += n_act * float(n)
        total = sum(h[1] for h in hist.values())
        res["n_active_histogram"] = {str(b): {"steps": h[0], "pair_share": round(h[1] / total, 4)}
                                     for b, h in sorted(hist.items())}
    res["roofline"] = _sub_roofline(res["value"], 60, "acc+jerk+pot (Eq. 3), over the whole run with its "
                                    "predictor, scheduler and corrector", device)
    return res


def run_block(args):
    n = 65536 if args.n == N_DEFAULT else args.n
    r = measure_block(n, 0.125, args.fp64_t_end)
    _line("pair interactions/s over a block-step Hermite run (acc+jerk+pot, incl. predictor/corrector/scheduler)",
          r["value"], UNIT, r["block_steps"], 0, r["seconds"], r["workload"],
          {k: v for k, v in r.items() if k not in ("value", "unit", "workload")})


ENSEMBLE_WORKLOAD = ("512 Plummer clusters N_c=floor(256*64^U) seed 1004, eps=1/N_c, leapfrog dt=1/256 x 64 steps, "
                     "one persistent launch per force, CUDA graph")


def measure_ensemble(runs=3, no_graph=True, device=0):
    """512 clusters, N_c log-uniform in [256, 16384), eps = 1/N_c, leapfrog dt = 1/256, 64 steps.  Value:
    sum_c N_c^2 x 64 / t.  Parity: the accelerations of the largest, the smallest and a middle cluster
    against the oracle, and the smallest cluster's positions after the 64 steps against the oracle's
    leapfrog."""
    import torch

    import oracle
    from oracle import leapfrog as olf
    from paper_0707_0438_gb300 import abi, autotune, metrics, workloads
    clusters, sizes = workloads.ensemble()
    off = np.concatenate([[0], np.cumsum(sizes)])
    m = np.concatenate([c.m for c in clusters])
    x = np.concatenate([c.x for c in clusters])
    v = np.concatenate([c.v for c in clusters])
    pairs_per_step = float(np.sum(sizes.astype(np.float64) ** 2))
    res = {}
    b = abi.KirinBatch(off, [c.eps for c in clusters], device=device)
    tuned = autotune.tune_batch(b, m, x, v)  # before and outside the timed runs
    b.close()
    parity = {}
    for use_graph in ((True, False) if no_graph else (True,)):
        b = abi.KirinBatch(off, [c.eps for c in clusters], device=device)
        b.set_launch(tuned[0], tuned[1])
        if use_graph:
            b.set_state(m, x, v)
            acc = b.accel()
            order = np.argsort(sizes)
            for c in (int(order[-1]), int(order[0]), int(order[len(order) // 2])):
                ra, _ = oracle.acc_pot(clusters[c].m, clusters[c].x, clusters[c].eps)
                e = metrics.summary(metrics.rel_err_vec(acc[off[c]:off[c + 1]], ra))
                parity[f"acc_cluster_{c}_N{int(sizes[c])}_vs_oracle"] = {q: float(f"{e[q]:.3g}") for q in e}
        b.set_state(m, x, v)
        b.leapfrog(1.0 / 256, 64, use_graph=use_graph)  # warm-up (and graph build)
        b.sync()
        if use_graph:
            xg, _ = b.get_state()
            c = int(np.argmin(sizes))
            xs, _ = olf.trajectory(clusters[c].m, clusters[c].x, clusters[c].v, clusters[c].eps, 1.0 / 256, 64)
            parity[f"x_after_64_steps_cluster_{c}_N{int(sizes[c])}_rel_diff"] = _rel_diff(xg[off[c]:off[c + 1]],
                                                                                         xs[-1])
        times = []
        with ClockSampler(device) as clk:
            for _ in range(max(1, runs)):
                b.set_state(m, x, v)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b.leapfrog(1.0 / 256, 64, use_graph=use_graph)
                b.sync()
                times.append(time.perf_counter() - t0)
        b.close()
        t = float(np.median(times))
        res["graph" if use_graph else "no_graph"] = {"seconds_per_64_steps": t, "value": pairs_per_step * 64 / t,
                                                     "clocks": clk.summary()}
    g = res["graph"]
    out = {"value": g["value"], "unit": UNIT, "seconds_per_64_steps": g["seconds_per_64_steps"],
           "clocks": g["clocks"], "workload": ENSEMBLE_WORKLOAD, "sum_Nc2": pairs_per_step,
           "gflops_k38": 38 * g["value"] / 1e9, "n_total": int(off[-1]), "parity": parity,
           "launch": {"groups": tuned[0], "i_per_item": 512 // tuned[0], "j_tiles": tuned[1],
                      "from": "tune_batch (timed before the runs)",
                      "timed_ms_per_step": {f"{e[0]}x{e[1]}": round(1e3 * e[2], 3) for e in tuned[2]}}}
    if "no_graph" in res:
        out["no_graph"] = res["no_graph"]
    out["roofline"] = _sub_roofline(g["value"], 38, "acc+pot (Eq. 3 without the jerk)", device)
    return out


def run_ensemble(args):
    r = measure_ensemble(max(1, args.steps))
    _line("pair interactions/s, batched leapfrog (sum_c N_c^2 x 64 / t)", r["value"], UNIT, 64, 1,
          r["seconds_per_64_steps"], r["workload"] + f", sum N_c^2={r['sum_Nc2']:.4g}",
          {k: v for k, v in r.items() if k not in ("value", "unit", "workload", "seconds_per_64_steps")})


ADJOINT_WORKLOAD = "plummer N=16384 eps=0.01 seed 1005, 64 KDK steps dt=1/128, checkpoints every 8 steps"


def measure_adjoint(steps, warmup, device=0):
    """N = 16384, eps = 0.01, 64 leapfrog steps dt = 1/128, checkpoint every 8; forward + backward, timed
    with CUDA events.  Parity: the two force calls of the run (acc + pot and the adjoint) at the initial
    state against the oracle, every particle."""
    import torch

    import oracle
    from paper_0707_0438_gb300 import abi, autotune, metrics, workloads
    from paper_0707_0438_gb300 import autograd as kag
    dev = torch.device("cuda", device)
    n, n_steps, dt = 16384, 64, 1.0 / 128
    p = workloads.config_adjoint(n)
    q = workloads.perturb(p, 1e-3)
    stream = torch.cuda.current_stream(dev).cuda_stream
    k = abi.Kirin(n, p.eps, precision="mixed", device=device, stream=stream)
    autotune.install(k, n, torch.cuda.get_device_name(dev), "mixed")  # acc+pot and adjoint tables, if stored
    T = lambda a, g=False: torch.tensor(a, dtype=torch.float64, device=dev, requires_grad=g)
    with torch.no_grad():
        tgt, _ = kag.leapfrog(T(q.x), T(q.v), T(q.m), k, dt, n_steps)

    def run():
        x, v, mm = T(p.x, True), T(p.v, True), T(p.m, True)
        xf, _ = kag.leapfrog(x, v, mm, k, dt, n_steps, every=8)
        loss = ((xf - tgt) ** 2).sum(dim=1).mean()
        loss.backward()
        return loss

    t0 = time.perf_counter()
    for _ in range(max(1, warmup)):
        run()
    torch.cuda.synchronize()
    t_run = (time.perf_counter() - t0) / max(1, warmup)
    steps = max(steps, int(math.ceil(0.5 / max(t_run, 1e-4))))  # at least half a second of runs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(device) as clk:
        e0.record()
        for _ in range(steps):
            loss = run()
        e1.record()
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / steps
    # parity of the run's two force calls at the initial state
    g = np.random.default_rng(21).standard_normal((n, 3))
    m_d, x_d, g_d = T(p.m), T(p.x), T(g)
    acc, gx = torch.empty_like(x_d), torch.empty_like(x_d)
    pot, gm = torch.empty_like(m_d), torch.empty_like(m_d)
    k.accel_dev(m_d, x_d, acc, pot)
    k.accel_adjoint_dev(m_d, x_d, g_d, gx, gm)
    k.sync()
    k.close()
    ra, rp = oracle.acc_pot(p.m, p.x, p.eps)
    rgx, rgm = oracle.force_adjoint(p.m, p.x, g, p.eps)
    parity = {"acc_pot_vs_oracle": _errs((acc.cpu().numpy(), pot.cpu().numpy()), (ra, rp))}
    for name, got, ref in (("dL_dx", gx.cpu().numpy(), rgx), ("dL_dm", gm.cpu().numpy()[:, None], rgm[:, None])):
        err = np.linalg.norm(got - ref, axis=1)
        parity[f"adjoint_{name}_vs_oracle"] = {
            "median_rel": float(f"{np.median(err / np.linalg.norm(ref, axis=1)):.3g}"),
            "max_over_rms": float(f"{err.max() / np.sqrt(np.mean(np.sum(ref * ref, axis=1))):.3g}")}
    # force evaluations: 65 forward, 64 recomputed, 65 adjoint (one per distinct position)
    evals = 65 + 64 + 65
    rate = evals * float(n) * n / t
    return {"value": t, "unit": "s", "ms_per_forward_backward": 1e3 * t, "runs": steps,
            "pair_evaluations_per_s": rate, "loss": float(loss.item()),
            "clocks": clk.summary(), "workload": ADJOINT_WORKLOAD, "parity": parity,
            "roofline": _sub_roofline(rate, 38, "every pair evaluation counted as acc+pot, a floor (an adjoint "
                                      "pair costs about twice a force-only one)", device)}


def run_adjoint(args):
    r = measure_adjoint(args.steps, args.warmup)
    _line("seconds per forward+backward of a 64-step differentiable leapfrog", r["value"], "s", r["runs"],
          args.warmup, r["value"] * r["runs"], r["workload"],
          {k: v for k, v in r.items() if k not in ("value", "unit", "workload")}, higher=False)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    # --particles: the same, for use under torchrun, whose own parser takes "--n" for a prefix of its options
    ap.add_argument("--n", "--particles", dest="n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", choices=["large", "small", "block", "ensemble", "adjoint"], default="large")
    ap.add_argument("--fp64-t-end", type=float, default=1.0 / 8)
    ap.add_argument("--no-sub", action="store_true", help="skip the secondary workloads on the default line")
    ap.add_argument("--launch", type=lambda t: tuple(int(v) for v in t.split(",")), default=None,
                    help="fixed launch shape GROUPS,SPLITS of the large-workload force calls")
    ap.add_argument("--parallel", choices=["replicas", "jsplit"], default="replicas",
                    help="N > 1: independent replicas (weak scaling) or one evaluation over a j partition (strong)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "large":
        run_native(args)
    else:
        {"small": run_small, "block": run_block, "ensemble": run_ensemble, "adjoint": run_adjoint}[args.workload](args)


if __name__ == "__main__":
    main()
