"""Real-time serving of many concurrent observation streams on one GPU.

A thin driver around the library's serving pool (cdd_pool_* in include/cdd.h):
streams are admitted against an HBM budget, each keeps its overlap tail,
alignment ring and integration state on the device, and blocks that arrive
while others are running are launched at once on the stream's own CUDA stream,
so their work overlaps on the GPU.  Arrivals are paced in virtual time (a block
of duration T arrives every T / speedup seconds of wall time); each block's
latency is measured by the library from its submit call to the completion of
its kernels.

    python -m paper_1509_00186_b300.serving [--blocks 8] [--speedup 50]

prints one JSON line: aggregate Msamples/s, x real time, p50/p99 block latency
against the block duration (the deadline), and admission results.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import cdd

D_S_MHZ2 = 4.148808e3       # s MHz^2 cm^3 / pc, for choosing N per stream


@dataclass(frozen=True)
class StreamSpec:
    f_center_mhz: float
    bandwidth_mhz: float
    n_chan: int
    dm: float
    n_avg: int = 16
    block_seconds: float = 0.5
    seed: int = 0

    @property
    def chan_bw(self) -> float:
        return self.bandwidth_mhz / self.n_chan

    def n_fft(self) -> int:
        """A power of two at least 4x the lowest channel's smear, and >= 2048."""
        f = self.f_center_mhz - self.bandwidth_mhz / 2
        n_d = D_S_MHZ2 * self.dm * (f ** -2 - (f + self.chan_bw) ** -2) * self.chan_bw * 1e6
        n = 2048
        while n < 4 * n_d:
            n *= 2
        return n


def mixed_scenario(n_streams: int = 8, seed: int = 7):
    """Streams drawn from the GSB and upgraded-GMRT shapes: 16 MHz / 256 and
    32 MHz / 512 channels at 325 and 610 MHz, 200 MHz / 2048 at 650 MHz, with
    DM uniform in [5, 150]."""
    shapes = [(325.0, 16.0, 256), (610.0, 16.0, 256), (325.0, 32.0, 512), (610.0, 32.0, 512),
              (650.0, 200.0, 2048)]
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_streams):
        f, bw, c = shapes[i % len(shapes)]
        specs.append(StreamSpec(f, bw, c, float(np.round(rng.uniform(5.0, 150.0), 2)), seed=100 + i))
    return specs


class Pool:
    """Owning wrapper of a serving pool."""

    def __init__(self, hbm_budget_bytes: int, max_streams: int = 64):
        self.handle = cdd.cdd_pool_create(hbm_budget_bytes, max_streams)

    def admit(self, spec: StreamSpec, n_fft=None):
        n_fft = n_fft or spec.n_fft()
        probe = cdd.Plan(spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n_fft,
                         spec.n_avg)
        hop = probe.get("hop")
        probe.close()
        rate = spec.chan_bw * 1e6
        q = max(1, int(spec.block_seconds * rate) // hop)
        sid = cdd.cdd_pool_admit(self.handle, spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan,
                                 spec.dm, n_fft, spec.n_avg, q, 0)
        return sid

    def get(self, sid, attr):
        return cdd.cdd_pool_stream_get(self.handle, sid, attr)

    def submit(self, sid, seq, vin, out):
        return cdd.cdd_pool_submit(self.handle, sid, seq, vin.data_ptr(), out.data_ptr())

    def wait(self, ticket) -> float:
        return cdd.cdd_pool_wait(self.handle, ticket)

    def release(self, sid):
        cdd.cdd_pool_release(self.handle, sid)

    def export_stream(self, sid):
        """(state, next sequence number) of a stream after its submitted blocks."""
        return cdd.cdd_pool_stream_export(self.handle, sid)

    def import_stream(self, sid, state, next_seq):
        """Continue an exported stream in the admitted stream `sid`."""
        cdd.cdd_pool_stream_import(self.handle, sid, state, next_seq)

    def used_bytes(self) -> int:
        return cdd.cdd_pool_get(self.handle, "used_bytes")

    def close(self):
        if self.handle:
            cdd.cdd_pool_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def make_block_inputs(spec: StreamSpec, block_samples: int, n_blocks: int):
    from synth import complex_int8_voltages
    return complex_int8_voltages(spec.seed, block_samples * n_blocks, spec.n_chan, 20.0)


def run_mix(specs, n_blocks: int, speedup: float = 1e9, budget_bytes: int = 64 << 30,
            stagger_blocks: float = 0.5, keep_outputs: bool = False, warm_first: bool = True):
    """Serve every stream for n_blocks blocks.  Stream i starts after
    i * stagger_blocks block durations; arrivals are paced at speedup x real
    time (1e9: as fast as possible).  warm_first: each stream's first block is
    served before the timed region (its plan commits there: device memory and
    tables), and the summary covers the other blocks.  Returns a summary dict
    (and the outputs of every block)."""
    import torch
    with Pool(budget_bytes, max_streams=max(1, len(specs))) as pool:
        admitted, refused = [], []
        for i, sp in enumerate(specs):
            try:
                admitted.append((i, sp, pool.admit(sp)))
            except cdd.CddError as e:
                if e.code != cdd.CDD_EBUSY:
                    raise
                refused.append(i)
        data, outs, events = {}, {}, []
        for i, sp, sid in admitted:
            bs = pool.get(sid, "block_samples")
            n_out = pool.get(sid, "n_out_per_block")
            x = torch.from_numpy(make_block_inputs(sp, bs, n_blocks)).cuda()
            data[sid] = (x, bs)
            outs[sid] = torch.empty((n_blocks, sp.n_chan, n_out), dtype=torch.float32, device="cuda")
            dur = bs / (sp.chan_bw * 1e6)
            for b in range(1 if warm_first else 0, n_blocks):
                events.append(((i * stagger_blocks + b + 1) * dur, sid, b, dur))
        events.sort()
        if warm_first:
            for i, sp, sid in admitted:
                x, bs = data[sid]
                pool.wait(pool.submit(sid, 0, x[:bs], outs[sid][0]))
        torch.cuda.synchronize()
        lat, futures = [], []
        with ThreadPoolExecutor(max_workers=8) as waiters:
            t0 = time.perf_counter()
            for t_arr, sid, b, dur in events:
                delay = t_arr / speedup - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                x, bs = data[sid]
                ticket = pool.submit(sid, b, x[b * bs:(b + 1) * bs], outs[sid][b])
                futures.append((sid, dur, waiters.submit(pool.wait, ticket)))
            results = [(sid, dur, f.result()) for sid, dur, f in futures]
            wall = time.perf_counter() - t0
        torch.cuda.synchronize()
        timed = n_blocks - (1 if warm_first else 0)
        samples = sum(data[sid][1] * specs[i].n_chan * timed for i, _, sid in admitted)
        rt = sum(specs[i].bandwidth_mhz * 1e6 for i, _, _ in admitted)
        lat = np.array([r[2] for r in results])
        deadline = np.array([r[1] * 1e3 for r in results])
        summary = {
            "streams_admitted": len(admitted), "streams_refused": refused,
            "blocks": len(results), "msamples_per_s": samples / wall / 1e6,
            "x_realtime": samples / wall / rt,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "deadline_ms": {"min": float(deadline.min()), "max": float(deadline.max())},
            "missed_deadlines": int((lat > deadline).sum()),
            "seq_gaps": sum(pool.get(sid, "seq_gaps") for _, _, sid in admitted),
            "hbm_used_bytes": pool.used_bytes(),
            "speedup": speedup,
        }
        result_outs = {i: outs[sid].cpu().numpy() for i, _, sid in admitted} if keep_outputs else None
        return summary, result_outs


def run_alone(spec: StreamSpec, n_blocks: int):
    """The same stream through a plain plan, block after block."""
    import torch
    n_fft = spec.n_fft()
    probe = cdd.Plan(spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n_fft, spec.n_avg)
    q = max(1, int(spec.block_seconds * spec.chan_bw * 1e6) // probe.get("hop"))
    probe.close()
    with cdd.Plan(spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n_fft, spec.n_avg,
                  segments_per_block=q) as p:
        bs = p.block_samples
        x = torch.from_numpy(make_block_inputs(spec, bs, n_blocks)).cuda()
        out = torch.stack([p.execute(x[b * bs:(b + 1) * bs]) for b in range(n_blocks)])
        torch.cuda.synchronize()
        return out.cpu().numpy()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--blocks", type=int, default=8)
    ap.add_argument("--speedup", type=float, default=50.0,
                    help="arrival pacing relative to real time (1e9 = as fast as possible)")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    args = ap.parse_args(argv)
    summary, _ = run_mix(mixed_scenario(args.streams), args.blocks, args.speedup,
                         int(args.budget_gb * (1 << 30)))
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
