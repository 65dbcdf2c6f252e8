"""Throughput benchmark of the coherent-dedispersion path on one or more GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cdd|reference]

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
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dedispersed Msamples/s, ×real-time, % HBM roofline; block p99 latency"
WORKLOAD = "gsb"
SAMPLE_CHANNELS = 192            # CPU baseline: channels of the full block (~10-20 s)
KERNEL_SOURCES = ("paper_1509_00186_b300/csrc/cdd_kernels.cu", "paper_1509_00186_b300/csrc/cdd_fft.cuh",
                  "paper_1509_00186_b300/csrc/cdd_passes.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ols_kernel_gsb_traffic.json")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
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

def cpu_oracle_rate(w, vin, n_channels: int) -> dict:
    """The FP64 oracle as it stands, on the first n_channels channels of the
    block: Msamples/s and what it ran on."""
    import oracle as O
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    t0 = time.perf_counter()
    O.dedisperse(vin, geo, channels=range(n_channels))
    dt = time.perf_counter() - t0
    samples = n_channels * (vin.shape[0] // geo.hop) * geo.hop
    return {"value": samples / dt / 1e6, "unit": "Msamples/s", "cores": 1, "kind": "oracle",
            "seconds": dt,
            "sample": f"{n_channels} of {w.n_chan} channels x {vin.shape[0]} samples "
                      f"(one block), numpy FP64, single thread"}


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
    per_step = 8                                 # channels per step: ~0.5 s of CPU work
    for _ in range(args.warmup):
        O.dedisperse(vin, geo, channels=range(per_step))
    times = []
    for s in range(args.steps):
        ch = [(s * per_step + i) % w.n_chan for i in range(per_step)]
        t0 = time.perf_counter()
        O.dedisperse(vin, geo, channels=ch)
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
        "cpu_baseline": {"value": value, "unit": "Msamples/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} channels of one {rows}-sample block per step"},
        "e2e": {"value": value, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


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
                segments_per_block=q, pipeline_chunks=4, stage_timing=True)
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
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded complex int8 N(0,20) noise plus a pulse train "
                "(period 33 ms, 3% duty) at each channel's dispersion delay",
        "config": {**config_dict(w, q, hop), "parallelism": f"replicas x{world} (channels independent)"},
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
                     "kernel": (f"ols_persistent_kernel<{int(math.log2(n_fft))}>"
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
    del vin, out
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(w, vin_np, min(SAMPLE_CHANNELS, C))
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--impl", choices=("cdd", "reference"), default="cdd")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--channels", type=int, default=None,
                    help="keep only the lowest C channels (profiling captures; not a bench line)")
    args = ap.parse_args(argv)
    world, rank, local = dist_env()
    if args.gpus != world and world != 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
