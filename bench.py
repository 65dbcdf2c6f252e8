"""Throughput benchmark of the coherent-dedispersion path on one or more GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cdd|reference]
    python bench.py --path lsb_hann|dual|precision|band_sum|batch|fullband|serving

A step dedisperses one block of the 32 MHz / 512-channel / DM 50 / N 8192 / x16
workload (GMRT GSB real-time shape): 76 overlap-save segments per channel, i.e.
617,728 complex int8 samples per channel (9.88 s of data), through one
cdd_execute call.  Inputs are seeded synthetic voltages resident in HBM
(632 MB per step, larger than the 126 MB L2, so no flush is needed).

Prints one JSON line (rank 0).  Under torchrun each rank runs its own plan on
its own channels' data (channels are independent: replicas, weak scaling); the
only communication is the barrier and the max-over-ranks of the timed region.
`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dedispersed Msamples/s, ×real-time, % HBM roofline; block p99 latency"
WORKLOAD = "gsb"
SAMPLE_CHANNELS = 512            # CPU baseline: the whole block, threads over channels
KERNEL_SOURCES = ("paper_1509_00186_b300/csrc/cdd_kernels.cu", "paper_1509_00186_b300/csrc/cdd_fft.cuh",
                  "paper_1509_00186_b300/csrc/cdd_passes.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ols_kernel_gsb_traffic.json")


def _code_only(text: str) -> str:
    """C++ source without comments and blank or trailing space: what the compiler sees."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(root: str = ROOT) -> str:
    """Hash of the fused kernel's code (comments ignored): the key of the
    committed DRAM-traffic capture, which reads null once the code changes."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(root, f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0, "_source": "fallback"}


def workload_info(n_chan=None):
    """The benchmark workload; ``n_chan`` keeps only the lowest channels (same
    channel width, N, overlap and integration), for small profiling captures."""
    import dataclasses
    from synth import WORKLOADS
    w = WORKLOADS[WORKLOAD]
    if n_chan is not None and n_chan != w.n_chan:
        f_lo0 = w.f_center_mhz - w.bandwidth_mhz / 2
        bw = w.chan_bw_mhz * n_chan
        w = dataclasses.replace(w, n_chan=n_chan, bandwidth_mhz=bw, f_center_mhz=f_lo0 + bw / 2)
    hop = w.n_fft - 64          # overlap of this shape (n_d = 54.9 -> 64), checked below
    q = w.n_samp // hop
    return w, q


def make_input(w, n_rows, seed):
    """Seeded voltages: noise sigma=20 plus a pulse train (period 33 ms, 3% duty)
    arriving in each channel at its cold-plasma delay, taken from the plan."""
    import numpy as np
    from synth import PulseTrain, complex_int8_voltages
    from paper_1509_00186_b300.cdd import Plan
    with Plan(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg) as p:
        shifts = np.array(p.shifts(), dtype=np.float64)
    offsets = -shifts * w.n_avg                  # channel k leads channel 0 by r_k*n_avg samples
    pulses = PulseTrain(3000.0, w.period_samples, w.width_samples, w.pulse_sigma, offsets)
    return complex_int8_voltages(seed, n_rows, w.n_chan, w.sigma, pulses)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", f"-lms={period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
                power.append(float(row[3]))
            except ValueError:
                continue
            for name, val in zip(names, row[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed glue

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity at world size 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- CPU oracle

def oracle_threads() -> int:
    """Host threads for the oracle: numpy's FFT and element-wise loops release
    the GIL, so channels dedisperse in parallel threads (no copies)."""
    return max(1, min(os.cpu_count() or 1, 64))


def oracle_channels(vin, geo, channels, threads: int, taper: str = "none"):
    """The oracle as it stands, over `channels` split round-robin across threads."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    chans = list(channels)
    parts = [chans[i::threads] for i in range(threads) if chans[i::threads]]
    with ThreadPoolExecutor(len(parts)) as ex:
        list(ex.map(lambda c: O.dedisperse(vin, geo, taper, channels=c), parts))


def cpu_oracle_rate(w, vin, n_channels: int) -> dict:
    """The FP64 oracle as it stands on the first n_channels channels of the
    block, threads over channels: Msamples/s and what it ran on."""
    import oracle as O
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    threads = oracle_threads()
    t0 = time.perf_counter()
    oracle_channels(vin, geo, range(n_channels), threads)
    dt = time.perf_counter() - t0
    samples = n_channels * (vin.shape[0] // geo.hop) * geo.hop
    return {"value": samples / dt / 1e6, "unit": "Msamples/s", "cores": threads, "kind": "oracle",
            "seconds": dt,
            "sample": f"{n_channels} of {w.n_chan} channels x {vin.shape[0]} samples "
                      f"(one block), numpy FP64, {threads} threads over channels"}


# ---------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    w, q = workload_info()
    from synth import PulseTrain, complex_int8_voltages  # noqa: F401
    import oracle as O
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    rows = q * geo.hop
    from synth import complex_int8_voltages as gen
    vin = gen(w.seed, rows, w.n_chan, w.sigma)
    threads = oracle_threads()
    per_step = min(w.n_chan, 2 * threads)        # channels per step: well under a second of wall time
    for _ in range(args.warmup):
        oracle_channels(vin, geo, range(per_step), threads)
    times = []
    for s in range(args.steps):
        ch = [(s * per_step + i) % w.n_chan for i in range(per_step)]
        t0 = time.perf_counter()
        oracle_channels(vin, geo, ch, threads)
        times.append(time.perf_counter() - t0)
    samples = per_step * rows
    total = sum(times)
    value = samples * len(times) / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Msamples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(w, q, geo.hop),
        "cpu_baseline": {"value": value, "unit": "Msamples/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} channels of one {rows}-sample block per step, "
                                   f"{threads} threads over channels"},
        "e2e": {"value": value, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# the arithmetic the block computes in, by --precision
DTYPE_OF = {"fp32": "f32", "fp16x2": "f16x2 (hi+lo f16 tensor-core products, f32 accumulate)",
            "bf16x2": "bf16x2 (hi+lo bf16 tensor-core products, f32 accumulate)",
            "fp16": "f16 (tensor-core products, f32 accumulate)",
            "bf16": "bf16 (tensor-core products, f32 accumulate)"}
PRECISION_CODE = {"fp32": 0, "fp16": 1, "fp16x2": 2, "bf16x2": 3, "bf16": 4}


def config_dict(w, q, hop):
    return {"workload": f"gsb-{w.bandwidth_mhz:g}MHz@{w.f_center_mhz:g}MHz-{w.n_chan}ch-DM{w.dm:g}"
                        f"-N{w.n_fft}-x{w.n_avg}",
            "f_center_mhz": w.f_center_mhz, "bandwidth_mhz": w.bandwidth_mhz, "n_chan": w.n_chan,
            "dm": w.dm, "n_fft": w.n_fft, "n_avg": w.n_avg, "segments_per_block": q,
            "block_samples_per_channel": q * hop,
            "l2": "inputs larger than L2 (632 MB int8 per step vs 126 MB), no flush"}


# ---------------------------------------------------------------- GPU arm

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1509_00186_b300.cdd import Plan
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device for --impl cdd")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w, q = workload_info(args.channels)
    plan = Plan(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg,
                segments_per_block=q, stage_timing=True, precision=args.precision)
    hop = plan.get("hop")
    assert hop * q == plan.block_samples and q == w.n_samp // hop
    rows, n_out, C = plan.block_samples, plan.n_out, w.n_chan
    vin_np = make_input(w, rows, w.seed + rank)
    vin = torch.from_numpy(vin_np).to(dev)
    out = torch.empty((C, n_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # ---- device-resident timing
    for _ in range(max(args.warmup, 3)):
        plan.execute(vin, out)
    launches_per_step = plan.get("kernel_launches")
    torch.cuda.synchronize(dev)
    stage0 = {k: plan.get(k) for k in ("timed_blocks", "corner_turn_ns", "ols_ns")}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        time.sleep(0.3)                        # let nvidia-smi start sampling
    barrier(world)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for i in range(args.steps):
        plan.execute(vin, out)
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clock_info = clocks.stop() if clocks else None
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    # per-stage device time, from the events the library records on the launching stream
    stage = {k: plan.get(k) - v for k, v in stage0.items()}
    assert stage["timed_blocks"] == args.steps, stage
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms_max = max_over_ranks(total_ms, world, dev)
    samples_rank = float(C) * rows * args.steps
    samples_all = sum_over_ranks(samples_rank, world, dev)
    value = samples_all / (total_ms_max * 1e-3) / 1e6

    # ---- end to end: pinned host buffers through cdd_execute_host
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    hin = torch.from_numpy(vin_np).pin_memory()
    hout = torch.empty((C, n_out), dtype=torch.float32).pin_memory()
    for _ in range(2):
        plan.execute_host(hin, hout)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.execute_host(hin, hout)
        _ = float(hout[0, -1])                 # the result is on the host
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    barrier(world)
    e2e_value = sum_over_ranks(float(C) * rows * e2e_steps, world, dev) / e2e_s / 1e6

    if rank != 0:
        plan.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    # ---- roofline of the fused kernel (one launch per step)
    peaks = measured_peaks()
    n_fft = w.n_fft
    kernel_ms = stage["ols_ns"] / args.steps / 1e6          # fused kernel, mean per launch
    corner_ms = stage["corner_turn_ns"] / args.steps / 1e6
    segs = C * q
    flops = segs * (10.0 * n_fft * math.log2(n_fft) + 9.0 * n_fft)     # fwd+inv FFT, chirp, detect
    comp_bytes = C * rows * 2 + C * plan.get("n_ov") * 2 + C * n_out * 4
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    fp32_peak_tflops = sm_count * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    achieved_tflops = flops / (kernel_ms * 1e-3) / 1e12
    achieved_gbs = comp_bytes / (kernel_ms * 1e-3) / 1e9
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as fh:
            tr = json.load(fh)
        if tr.get("kernel_source_hash") == kernel_source_hash():
            traffic = tr.get("dram_bytes_per_launch")
    rt_rate = C * w.chan_bw_mhz * 1e6                  # complex samples per second, real time
    block_s = rows / (w.chan_bw_mhz * 1e6)
    line = {
        "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_OF[args.precision],
        "data": "synthetic: seeded complex int8 N(0,20) noise plus a pulse train "
                "(period 33 ms, 3% duty) at each channel's dispersion delay",
        "config": {**config_dict(w, q, hop), **({"precision": args.precision} if args.precision != "fp32" else {})},
        "parallelism": f"replicas x{world} (channels independent)",
        "x_realtime": value * 1e6 / (rt_rate * world),
        "hbm_roofline_frac": achieved_gbs / peaks["hbm_gbs"],
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": float(np.percentile(step_ms, 99)),
                       "deadline": block_s * 1e3},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved_tflops / fp32_peak_tflops,
                     "traffic": traffic,
                     "peak_source": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x "
                                    f"{peaks['sm_max_mhz']:.0f} MHz ({peaks['_source']} max clock)",
                     "kernel": (f"ols_tc_kernel<{PRECISION_CODE[args.precision]}>"
                                if args.precision != "fp32" else
                                f"ols_persistent_kernel<{int(math.log2(n_fft))}>"
                                if n_fft in (4096, 8192) else f"ols_kernel<{int(math.log2(n_fft))}>"),
                     "kernel_ms": kernel_ms,
                     "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
                     "flops_per_launch": flops, "algorithmic_bytes_per_launch": comp_bytes},
        "e2e": {"value": e2e_value, "unit": "Msamples/s",
                "h2d_bytes_per_step": int(hin.numel()), "d2h_bytes_per_step": int(hout.numel() * 4)},
        "stages": {"corner_turn": {"ms": corner_ms, "gbs": 4.0 * C * rows / (corner_ms * 1e-3) / 1e9,
                                   "hbm_frac": 4.0 * C * rows / (corner_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                   "ols": {"ms": kernel_ms}},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clock_info,
        "paper_gflops": flops / (kernel_ms * 1e-3) / 1e9,
    }
    plan.close()
    del out
    if not args.no_rows and args.precision == "fp32":
        line["rows"] = collect_rows(args, dev, peaks, vin, w, q)
    del vin
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(w, vin_np, min(SAMPLE_CHANNELS, C))
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other rows
#
# `--path P` measures one more row of the path on one GPU and prints its own
# JSON line (rank 0; other ranks exit).  Each line carries the roofline of its
# dominant kernel or of the whole step (said in "roofline.kernel") and the FP64
# oracle timed on a bounded sample of the same workload.

def _timed(fn, steps, warmup, dev):
    """W warm-up calls, then K calls bracketed by CUDA events on the current
    stream, with nvidia-smi clock samples during the timed region."""
    import torch
    for _ in range(max(warmup, 3)):
        fn()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clocks = ClockSampler(dev.index or 0)
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for i in range(steps):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    clock_info = clocks.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]), step_ms, clock_info


def _fp32_peak(dev, peaks):
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12, \
        f"{sms} SMs x 128 FP32 lanes x 2 flop x {peaks['sm_max_mhz']:.0f} MHz ({peaks['_source']} max clock)"


def _cpu_time(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def _line(path, args, metric, value, unit, ms, steps_ms, config, roofline, cpu, clocks, launches,
          dtype="f32", higher=True, **extra):
    line = {"path": path, "metric": metric, "value": value, "unit": unit, "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic: seeded complex int8 N(0,20) noise", "config": config,
            "latency_ms": {"p50": statistics.median(steps_ms),
                           "p99": float(sorted(steps_ms)[min(len(steps_ms) - 1, int(0.99 * len(steps_ms)))])},
            "roofline": roofline, "gpu_launches": launches, "clocks": clocks}
    line.update(extra)
    if cpu is not None:
        line["cpu_baseline"] = cpu
    return line


def _alu_roofline(kernel, flops, kernel_ms, dev, peaks):
    peak, src = _fp32_peak(dev, peaks)
    ach = flops / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "peak_source": src, "kernel": kernel, "kernel_ms": kernel_ms,
            "flops_per_launch": flops}


def _hbm_roofline(kernel, nbytes, kernel_ms, peaks):
    ach = nbytes / (kernel_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": None,
            "peak_source": f"hbm_gbs ({peaks['_source']})", "kernel": kernel, "kernel_ms": kernel_ms,
            "algorithmic_bytes_per_launch": nbytes}


def _ols_flops(n_fft, segments):
    return segments * (10.0 * n_fft * math.log2(n_fft) + 9.0 * n_fft)


def device_voltages(rows, n_chan, seed, dev, sigma=20.0):
    """Seeded complex int8 noise N(0, sigma) drawn on the device: the inputs of
    the rows under "rows" (their throughput does not depend on the data;
    the headline line's input comes from synth)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.empty((rows, n_chan, 2), dtype=torch.int8, device=dev)
    chunk = max(1, (1 << 27) // (2 * n_chan))
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        v = torch.randn((r1 - r0, n_chan, 2), device=dev, generator=g).mul_(sigma)
        x[r0:r1] = v.round_().clamp_(-127, 127).to(torch.int8)
    return x


def tc_tensor_flops(segments, precision):
    """Tensor-core flops one launch of the tensor-core kernel executes: per
    segment, radix-32 passes (2 tiles of 128 groups, K = 64) and radix-16
    passes (4 tiles, K = 32), N = 4R with the hi + lo DFT matrix (2R
    without), plus the lo operand's product (N = 2R) in every split pass
    but the exact first one."""
    split = precision.endswith("x2")
    def pass_flops(R, tiles, lo):
        n = 4 * R if split else 2 * R
        f = tiles * (2 * R // 16) * 2 * 128 * n * 16
        if split and lo:
            f += tiles * (2 * R // 16) * 2 * 128 * (2 * R) * 16
        return f
    per = pass_flops(32, 2, False) + 4 * pass_flops(16, 4, True) + pass_flops(32, 2, True)
    return segments * per


def row_tc(args, dev, peaks, precision, vin, w, q):
    """The 512-channel N 8192 block with the radix passes on the tensor cores
    (tcgen05 DFT products, FP32 accumulation), on the headline's input."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    plan = Plan(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg,
                segments_per_block=q, stage_timing=True, precision=precision)
    C, rows, n_out = w.n_chan, plan.block_samples, plan.n_out
    out = torch.empty((C, n_out), dtype=torch.float32, device=dev)
    fn = lambda: plan.execute(vin, out)
    for _ in range(max(args.warmup, 3)):
        fn()
    torch.cuda.synchronize(dev)
    st0 = {k: plan.get(k) for k in ("timed_blocks", "ols_ns", "corner_turn_ns")}
    total, steps_ms, clocks = _timed(fn, args.steps, 0, dev)
    st = {k: plan.get(k) - v for k, v in st0.items()}
    launches = plan.get("kernel_launches")
    errors = plan.get("device_errors")
    plan.close()
    kernel_ms = st["ols_ns"] / st["timed_blocks"] / 1e6
    segs = C * q
    tflops = tc_tensor_flops(segs, precision)
    ach = tflops / (kernel_ms * 1e-3) / 1e12
    peak = peaks["bf16_tflops"]
    roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None,
            "peak_source": f"bf16_tflops ({peaks['_source']}; dense f16 runs at the bf16 rate)",
            "kernel": f"ols_tc_kernel<{PRECISION_CODE[precision]}>", "kernel_ms": kernel_ms,
            "tensor_flops_per_launch": tflops,
            "fp32_equivalent": _alu_roofline("same kernel, radix-2 flop count", _ols_flops(w.n_fft, segs),
                                             kernel_ms, dev, peaks)["frac"],
            "corner_turn_ms": st["corner_turn_ns"] / st["timed_blocks"] / 1e6}
    value = float(C) * rows * args.steps / (total * 1e-3) / 1e6
    config = {"workload": f"tc:{config_dict(w, q, rows // q)['workload']}", "precision": precision}
    return _line(f"tc_{precision}", args, "dedispersed Msamples/s", value, "Msamples/s",
                 total / args.steps, steps_ms, config, roof, None, clocks, launches * args.steps,
                 dtype=DTYPE_OF[precision], x_realtime=value * 1e6 / (C * w.chan_bw_mhz * 1e6),
                 device_errors=errors)


def _compact(line):
    keep = ("metric", "value", "unit", "ms_per_step", "x_realtime", "dtype", "latency_ms", "gpu_launches",
            "clocks", "missed_deadlines", "deadline_ms", "device_errors")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line.get("config", {}).get("workload")
    for k in ("launch_form", "tuning_ms"):
        if k in line.get("config", {}):
            out[k] = line["config"][k]
    r = line.get("roofline")
    if r:
        out["roofline"] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "kernel_ms",
                                              "fp32_equivalent", "frac_of_min_bytes") if k in r}
    return out


def collect_rows(args, dev, peaks, vin, w, q):
    """The other rows of the path, each timed briefly (args.row_steps steps
    after 3 warm-up steps) on one GPU: the tensor-core forms of the headline
    block, the N = 65536 shape, the batched form, the full-band mode and the
    serving pool.  A row that fails reports its error instead."""
    import copy
    import torch
    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.no_cpu_baseline, sub.channels, sub.dm = args.row_steps, 3, True, None, None
    rows = {}
    jobs = [("tc_fp16x2", lambda: row_tc(sub, dev, peaks, "fp16x2", vin, w, q)),
            ("tc_fp16", lambda: row_tc(sub, dev, peaks, "fp16", vin, w, q)),
            ("precision_n65536", lambda: row_plan_variant(sub, dev, peaks, "precision", device_input=True)),
            ("batch", lambda: row_batch(sub, dev, peaks, device_input=True)),
            ("fullband", lambda: row_fullband(sub, dev, peaks)),
            ("serving", lambda: row_serving(sub, dev, peaks))]
    for name, fn in jobs:
        try:
            rows[name] = _compact(fn())
        except Exception as e:                      # report, do not lose the headline
            rows[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
    return rows


def row_plan_variant(args, dev, peaks, path, device_input=False):
    """lsb_hann: the GSB block as a lower-sideband band with the Hann taper.
    dual: the GSB block for two polarisations summed after detection.
    precision: 150 MHz / DM 100 / N 65536 (a cluster of eight CTAs per segment)."""
    import numpy as np
    import torch
    import oracle as O
    from synth import WORKLOADS, complex_int8_voltages
    from paper_1509_00186_b300.cdd import Plan
    w = WORKLOADS["precision" if path == "precision" else "gsb"]
    if args.channels is not None and args.channels != w.n_chan:
        # the lowest channels only (same channel width, so the same N, overlap and hop)
        import dataclasses
        f_lo0 = w.f_center_mhz - w.bandwidth_mhz / 2
        cut = w.chan_bw_mhz * args.channels
        w = dataclasses.replace(w, n_chan=args.channels, bandwidth_mhz=cut, f_center_mhz=f_lo0 + cut / 2)
    bw = -w.bandwidth_mhz if path == "lsb_hann" else w.bandwidth_mhz
    taper = "hann" if path == "lsb_hann" else "none"
    geo = O.plan_geometry(w.f_center_mhz, bw, w.n_chan, w.dm, w.n_fft, w.n_avg)
    q = w.n_samp // geo.hop
    pols = 2 if path == "dual" else 1
    plan = Plan(w.f_center_mhz, bw, w.n_chan, w.dm, w.n_fft, w.n_avg, segments_per_block=q,
                taper=taper, polarisations=pols, stage_timing=True)
    rows, C, n_out = plan.block_samples, w.n_chan, plan.n_out
    if device_input:
        va = vb = None
        xa = device_voltages(rows, C, w.seed, dev, w.sigma)
        xb = device_voltages(rows, C, w.seed + 100, dev, w.sigma) if pols == 2 else None
    else:
        va = complex_int8_voltages(w.seed, rows, C, w.sigma)
        vb = complex_int8_voltages(w.seed + 100, rows, C, w.sigma) if pols == 2 else None
        xa = torch.from_numpy(va).to(dev)
        xb = torch.from_numpy(vb).to(dev) if pols == 2 else None
    out = torch.empty((C, n_out), dtype=torch.float32, device=dev)
    fn = (lambda: plan.execute_dual(xa, xb, out)) if pols == 2 else (lambda: plan.execute(xa, out))
    for _ in range(max(args.warmup, 3)):
        fn()
    torch.cuda.synchronize(dev)
    st0 = {k: plan.get(k) for k in ("timed_blocks", "ols_ns", "corner_turn_ns")}
    total, steps_ms, clocks = _timed(fn, args.steps, 0, dev)
    st = {k: plan.get(k) - v for k, v in st0.items()}
    launches = plan.get("kernel_launches")
    plan.close()
    kernel_ms = st["ols_ns"] / st["timed_blocks"] / 1e6
    samples = float(C) * rows * pols
    value = samples * args.steps / (total * 1e-3) / 1e6
    logn = int(math.log2(geo.n_fft))
    kname = {"precision": "ols_cluster_kernel<13,8>"}.get(path, f"ols_persistent_kernel<{logn}>")
    roof = _alu_roofline(kname, _ols_flops(geo.n_fft, C * q), kernel_ms, dev, peaks)
    roof["corner_turn_ms"] = st["corner_turn_ns"] / st["timed_blocks"] / 1e6
    cpu = None
    if not args.no_cpu_baseline and va is not None:
        threads = oracle_threads()
        n_cpu = min(C, {"precision": 4, "dual": 4}.get(path, 8) * threads)
        dt = _cpu_time(lambda: [oracle_channels(v, geo, range(n_cpu), threads, taper)
                                for v in ((va, vb) if pols == 2 else (va,))])
        cpu = {"value": n_cpu * q * geo.hop * pols / dt / 1e6, "unit": "Msamples/s", "cores": threads,
               "kind": "oracle", "seconds": dt,
               "sample": f"{n_cpu} of {C} channels x {q * geo.hop} samples x {pols} polarisation(s), "
                         f"{threads} threads over channels"}
    wl = f"{w.f_center_mhz:g}MHz-{abs(bw):g}MHz-{'LSB' if bw < 0 else 'USB'}-{C}ch-DM{w.dm:g}-N{geo.n_fft}-x{w.n_avg}"
    config = {"workload": f"{path}:{wl}", "taper": taper, "polarisations": pols,
              "segments_per_block": q, "block_samples_per_channel": rows}
    rt = C * w.chan_bw_mhz * 1e6 * pols
    return _line(path, args, "dedispersed Msamples/s", value, "Msamples/s", total / args.steps,
                 steps_ms, config, roof, cpu, clocks, launches * args.steps,
                 x_realtime=value * 1e6 / rt)


def row_band_sum(args, dev, peaks):
    """Band sum of aligned intensities [planes][C][n_out] -> [planes][n_out] on
    the batched form's output shape: 64 DM-trial planes of 2048 channels x
    23808 outputs (12.5 GB, far larger than L2), giving the DM-trial time
    series.  HBM bound."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1509_00186_b300.cdd import band_sum
    planes, C, n_out = 64, 2048, 23808
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    out = torch.rand((planes, C, n_out), dtype=torch.float32, device=dev, generator=g)
    res = torch.empty((planes, n_out), dtype=torch.float32, device=dev)
    from paper_1509_00186_b300 import cdd as _c
    stream = torch.cuda.current_stream(dev).cuda_stream
    fn = lambda: _c.cdd_band_sum(out.data_ptr(), planes, C, n_out, res.data_ptr(), stream)
    total, steps_ms, clocks = _timed(fn, args.steps, args.warmup, dev)
    ms = total / args.steps
    nbytes = planes * C * n_out * 4 + planes * n_out * 4
    value = planes * C * n_out / (ms * 1e-3) / 1e6
    roof = _hbm_roofline("band_sum_kernel<4>", nbytes, ms, peaks)
    cpu = None
    if not args.no_cpu_baseline:
        host = out[0].cpu().numpy()
        dt = _cpu_time(lambda: O.band_sum(host))
        cpu = {"value": host.size / dt / 1e6, "unit": "Mintensities/s", "cores": 1, "kind": "oracle",
               "seconds": dt, "sample": f"one plane ({C} x {n_out}) of the {planes}, numpy"}
    # the library's band sum against a float64 sum of the same plane
    check = float(np.abs(res[0].cpu().numpy() - out[0].double().sum(0).cpu().numpy()).max()
                  / out[0].double().sum(0).abs().max().item())
    config = {"workload": f"band_sum:{planes}x{C}x{n_out}-float32 (DM-trial planes)",
              "bytes_in": planes * C * n_out * 4, "l2": "input 12.5 GB, larger than L2"}
    return _line("band_sum", args, "band-summed intensities per second", value, "Mintensities/s", ms,
                 steps_ms, config, roof, cpu, clocks, args.steps, max_rel_err_plane0=check)


def row_batch(args, dev, peaks, device_input=False):
    """Batched form: 650 MHz / 200 MHz / 2048 channels / 64 DM trials 20.0..51.5,
    tiers N = 16384, 8192, 4096, 2048 (lowest frequencies first), x16, a block
    of 24 longest hops (3.9 s)."""
    import numpy as np
    import torch
    import oracle as O
    from synth import complex_int8_voltages
    from paper_1509_00186_b300.cdd import Batch
    dms = [20.0 + 0.5 * i for i in range(64)]
    tiers = (16384, 8192, 4096, 2048)
    C, n_avg = 2048, 16
    f_c, bw = 650.0, 200.0
    if args.channels is not None and args.channels != C:
        # the lowest channels only (same channel width and lowest edge), for profiling captures
        if args.channels % 4:
            raise SystemExit("--path batch: --channels must be a multiple of the 4 tiers")
        C, bw = args.channels, bw * args.channels / C
        f_c = 650.0 - 100.0 + bw / 2
    b = Batch(f_c, bw, C, dms, tiers, n_avg, segments_per_block=24)
    bs, n_out = b.block_samples, b.n_out
    if device_input:
        vin, x = None, device_voltages(bs, C, 4, dev)
    else:
        vin = complex_int8_voltages(4, bs, C, 20.0)
        x = torch.from_numpy(vin).to(dev)
    out = torch.empty((len(dms), C, n_out), dtype=torch.float32, device=dev)
    total, steps_ms, clocks = _timed(lambda: b.execute(x, out), args.steps, args.warmup, dev)
    launches = b.get("kernel_launches")
    form = {0: "tiers", 1: "tiers_np", 2: "multi"}.get(b.get("batch_form"), "?")
    tune_ms = {"tiers": b.get("tune_ns_tiers") / 1e6, "multi": b.get("tune_ns_multi") / 1e6}
    flops = 0.0
    for t in range(len(tiers)):
        n, nov, _, ct = b.tier(t)
        segs = ct * (bs // (n - nov))
        flops += segs * (5.0 * n * math.log2(n) + len(dms) * (5.0 * n * math.log2(n) + 9.0 * n))
    b.close()
    ms = total / args.steps
    value = C * bs / (ms * 1e-3) / 1e6
    roof = _alu_roofline("whole step (forward spectra + per-DM chirp/inverse/detect/integrate)",
                         flops, ms, dev, peaks)
    roof["output_bytes_per_step"] = out.numel() * 4
    cpu = None
    if not args.no_cpu_baseline and vin is not None:
        geo = O.batch_geometry(f_c, bw, C, dms, tiers, n_avg)
        threads = oracle_threads()
        per_tier = max(1, threads // 4)
        chans = [t * (C // 4) + i for t in range(4) for i in range(min(per_tier, C // 4))]
        from concurrent.futures import ThreadPoolExecutor
        parts = [chans[i::threads] for i in range(threads) if chans[i::threads]]

        def run_parts():
            with ThreadPoolExecutor(len(parts)) as ex:
                list(ex.map(lambda c: O.dedisperse_batch(vin, geo, channels=c), parts))
        dt = _cpu_time(run_parts)
        cpu = {"value": len(chans) * bs / dt / 1e6, "unit": "Msamples/s", "cores": threads, "kind": "oracle",
               "seconds": dt, "sample": f"{len(chans)} channels ({per_tier} per tier) x {bs} samples x "
                                        f"{len(dms)} DMs, {threads} threads over channels"}
    config = {"workload": f"batch:{f_c:g}MHz-{bw:g}MHz-{C}ch-{len(dms)}DM-N16384/8192/4096/2048-x{n_avg}",
              "block_samples_per_channel": bs, "dm_trials": len(dms),
              "launch_form": form, "tuning_ms": tune_ms}
    return _line("batch", args, "input Msamples/s through all DM trials", value, "Msamples/s", ms,
                 steps_ms, config, roof, cpu, clocks, launches * args.steps,
                 x_realtime=value * 1e6 / (bw * 1e6))


def row_fullband(args, dev, peaks):
    """Full-band mode (the paper's design): 325 MHz / 32 MHz / 512-channel
    frames / DM 50: N = 2^26 real points over the whole band, one segment per
    block (h real samples, 0.65 s)."""
    import numpy as np
    import torch
    import oracle as O
    from synth import complex_int8_voltages
    from paper_1509_00186_b300.cdd import Fullband
    a = (325.0, 32.0, 512, 50.0 if args.dm is None else args.dm, 0, 16)
    f = Fullband(*a, segments_per_block=1)
    n, nov, h = f.get("n_fft"), f.get("n_ov"), f.get("hop")
    frames = f.frames
    vin = complex_int8_voltages(13, frames, 512, 20.0)
    x = torch.from_numpy(vin).to(dev)
    out = torch.empty((f.n_out,), dtype=torch.float32, device=dev)
    total, steps_ms, clocks = _timed(lambda: f.execute(x, out), args.steps, args.warmup, dev)
    launches = f.get("kernel_launches")
    pp = f.get("pass_plan")
    f.close()
    ms = total / args.steps
    logn = int(math.log2(n))
    # the library's pass plan: the shared-memory transform and the outer radices
    logs = pp & 0xFF
    radices, sh = [], 8
    while (pp >> sh) & 0xF:
        radices.append(1 << ((pp >> sh) & 0xF))
        sh += 4
    outer = len(radices)
    # per pass: the edge passes 12 bytes per point (real series in, or Re(y)^2 out),
    # the inner ones 16, the middle 24 (the transform both ways and the chirp)
    pass_bytes = (24 * n + 2 * (12 * n + 16 * n * (outer - 1))) if outer else 16 * n
    extra = 9.25 * h + 8 * nov                     # inverse channelisation and the carried overlap
    nbytes = pass_bytes + extra
    # the method's minimum: one outer pass each way around the middle (three round trips)
    min_bytes = (24 * n + 2 * 12 * n if outer else 16 * n) + extra
    value = h / (ms * 1e-3) / 1e6
    roof = _hbm_roofline(f"whole step ({outer} outer HBM passes each way, radix "
                         f"{'x'.join(map(str, radices)) or '-'}, around {1 << logs}-point shared-memory "
                         "sub-transforms)", nbytes, ms, peaks)
    roof["flops_per_launch"] = 10.0 * n * logn + 9.0 * n
    roof["min_bytes_per_launch"] = min_bytes
    roof["frac_of_min_bytes"] = min_bytes / (ms * 1e-3) / 1e9 / roof["peak"]
    cpu = None
    if not args.no_cpu_baseline:
        geo = O.fullband_geometry(*a)
        dt = _cpu_time(lambda: O.dedisperse_fullband(vin, geo))
        cpu = {"value": h / dt / 1e6, "unit": "Msamples/s", "cores": 1, "kind": "oracle", "seconds": dt,
               "sample": f"one segment (N = 2^{logn}, {h} real samples), numpy FP64"}
    config = {"workload": f"fullband:325MHz-32MHz-512ch-frames-DM{a[3]:g}-N2^{logn}-x16", "n_fft": n,
              "n_ov": nov, "hop": h, "frames_per_block": frames}
    return _line("fullband", args, "dedispersed real Msamples/s", value, "Msamples/s", ms, steps_ms,
                 config, roof, cpu, clocks, launches * args.steps, x_realtime=value / 64.0)


def row_serving(args, dev, peaks):
    """Serving pool: 8 mixed streams (GSB 16/32 MHz at 325/610 MHz, upgraded-GMRT
    200 MHz / 2048 channels at 650 MHz; DM 5..150), 8 blocks of 0.5 s each,
    ingested from pinned host memory (copy-in, dedispersion, copy-out inside
    each block's latency, counted from the block's arrival).  Three runs:
    - paced: arrivals at 20x real time, every stream admitted on arrival; the
      latency and missed deadlines (block duration / 20) of this run are the
      row's latency;
    - queued: the same pacing with an HBM budget of about half the streams'
      needs, so later streams wait in the pool's queue and enter mid-run (their
      blocks' latency includes that wait);
    - unpaced: every block at once (batched library calls), for the aggregate
      rate, which is the row's value."""
    from paper_1509_00186_b300 import cdd, serving
    specs = serving.mixed_scenario(8)
    needs = []
    for sp in specs:
        n = sp.n_fft()
        with cdd.Plan(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, n, sp.n_avg,
                      segments_per_block=sp.segments_per_block(n)) as p:
            needs.append(p.get("bytes_needed") + p.get("host_staging_bytes"))
    need = sum(needs)
    budget = max(need // 2, max(needs))
    clocks = ClockSampler(dev.index or 0)
    time.sleep(0.3)
    paced, _ = serving.run_mix(specs, 8, speedup=20.0, budget_bytes=64 << 30)
    queued, _ = serving.run_mix(specs, 8, speedup=20.0, budget_bytes=budget)
    full, _ = serving.run_mix(specs, 8, speedup=1e9, budget_bytes=64 << 30)
    clock_info = clocks.stop()
    cfg = {"workload": "serving:8-mixed-streams-x8-blocks-0.5s-host-ingest",
           "streams": [s.__dict__ for s in specs], "queued_budget_bytes": budget,
           "streams_total_need_bytes": need}
    line = {"path": "serving", "metric": "served Msamples/s (8 streams from host buffers)",
            "value": full["msamples_per_s"], "unit": "Msamples/s", "n_gpus": 1,
            "steps": full["blocks"], "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "x_realtime": full["x_realtime"],
            "latency_ms": paced["latency_ms"], "deadline_ms": paced["deadline_ms"],
            "missed_deadlines": paced["missed_deadlines"],
            "paced_run": paced, "queued_run": queued, "unpaced_run": full,
            "roofline": None, "roofline_note": "the same per-channel kernels as the block path; "
                                               "this row measures ingest, admission and latency",
            "clocks": clock_info, "gpu_launches": None}
    return line


ROWS = ("block", "lsb_hann", "dual", "precision", "band_sum", "batch", "fullband", "serving")


def run_row(args, world, rank, local):
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measured_peaks()
    if args.path in ("lsb_hann", "dual", "precision"):
        line = row_plan_variant(args, dev, peaks, args.path)
    else:
        line = {"band_sum": row_band_sum, "batch": row_batch, "fullband": row_fullband,
                "serving": row_serving}[args.path](args, dev, peaks)
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--impl", choices=("cdd", "reference"), default="cdd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true",
                    help="headline line only (without the other rows of the path under \"rows\")")
    ap.add_argument("--row-steps", type=int, default=10, help="timed steps of each row under \"rows\"")
    ap.add_argument("--precision", choices=("fp32", "fp16x2", "bf16x2", "fp16", "bf16"), default="fp32",
                    help="arithmetic of the block's transforms: fp32 on the CUDA cores, the others as "
                         "tensor-core (tcgen05) DFT products with FP32 accumulation")
    ap.add_argument("--path", choices=ROWS, default="block",
                    help="block: the headline line; others: one more row of the path (one GPU)")
    ap.add_argument("--dm", type=float, default=None,
                    help="--path fullband: another DM (sets N; smaller cases for profiling captures)")
    ap.add_argument("--channels", type=int, default=None,
                    help="keep only the lowest C channels (profiling captures; not a bench line)")
    args = ap.parse_args(argv)
    world, rank, local = dist_env()
    if args.gpus != world and world != 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.path != "block":
        return run_row(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
