"""Real-time serving of many concurrent observation streams on one GPU.

A thin driver around the library's serving pool (cdd_pool_* in include/cdd.h),
in the shape of the paper's real-time loop (Sec. 4.2, 4.3) run for many
streams at once:

- streams arrive over time and ask the pool for admission; a stream that
  does not fit the HBM budget waits in the pool's first-come queue and is
  admitted when a finished stream is released;
- each block arrives when it has been recorded (its duration after the one
  before, paced at `speedup` x real time) and is submitted with its arrival
  time: from pinned host buffers (copy-in, dedispersion and copy-out on the
  stream's own CUDA stream) or from device buffers;
- overlap tails, alignment rings and integration state stay on the device
  between blocks; blocks of different streams overlap on the GPU;
- each block's latency runs from its arrival to the completion of its work
  (host copies included), measured by the library.

    python -m paper_1509_00186_b300.serving [--blocks 8] [--speedup 50]

prints one JSON line: aggregate Msamples/s, x real time, p50/p99 block latency
against the paced deadline, and the admissions (at once or from the queue).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import cdd

N_FFT_FLOOR = 2048          # transform length floor for the serving streams


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
        """The library's transform-length rule (Sec. 2.3: the smallest power of
        two above twice the dispersion samples, n_fft = 0), raised to
        N_FFT_FLOOR so that short smears do not make short, overlap-heavy
        segments."""
        p = cdd.cdd_plan_create(self.f_center_mhz, self.bandwidth_mhz, self.n_chan, self.dm, 0, self.n_avg)
        try:
            n = cdd.cdd_plan_get(p, "n_fft")
        finally:
            cdd.cdd_destroy(p)
        return max(n, N_FFT_FLOOR)

    def segments_per_block(self, n_fft: int) -> int:
        p = cdd.cdd_plan_create(self.f_center_mhz, self.bandwidth_mhz, self.n_chan, self.dm, n_fft, self.n_avg)
        try:
            hop = cdd.cdd_plan_get(p, "hop")
        finally:
            cdd.cdd_destroy(p)
        return max(1, int(self.block_seconds * self.chan_bw * 1e6) // hop)


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

    @staticmethod
    def _args(spec: StreamSpec, n_fft=None):
        n_fft = n_fft or spec.n_fft()
        return (spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n_fft, spec.n_avg,
                spec.segments_per_block(n_fft), 0)

    def admit(self, spec: StreamSpec, n_fft=None, host=False):
        """Admit now (CddError CDD_EBUSY if it does not fit)."""
        return cdd.cdd_pool_admit_ex(self.handle, *self._args(spec, n_fft),
                                     cdd.POOL_HOST_INGEST if host else 0)

    def request(self, spec: StreamSpec, n_fft=None, host=False) -> int:
        """Queue for admission; poll with status()."""
        return cdd.cdd_pool_request(self.handle, *self._args(spec, n_fft),
                                    cdd.POOL_HOST_INGEST if host else 0)

    def status(self, request):
        """The admitted stream's id, or None while the request waits."""
        return cdd.cdd_pool_request_status(self.handle, request)

    def get(self, sid, attr):
        return cdd.cdd_pool_stream_get(self.handle, sid, attr)

    def submit(self, sid, seq, vin, out, t_arrival_ms=None):
        """One block from tensors: device tensors, or pinned host tensors of a
        stream admitted with host=True."""
        t = cdd.cdd_pool_clock_ms() if t_arrival_ms is None else t_arrival_ms
        if vin.is_cuda:
            return cdd.cdd_pool_submit_at(self.handle, sid, seq, vin.data_ptr(), out.data_ptr(), t)
        return cdd.cdd_pool_submit_host(self.handle, sid, seq, vin.data_ptr(), out.data_ptr(), t)

    def submit_many(self, blocks, host):
        """blocks: (sid, seq, vin, out, t_arrival_ms) tuples, in one call."""
        return cdd.cdd_pool_submit_many(self.handle, [b[0] for b in blocks], [b[1] for b in blocks],
                                        [b[2].data_ptr() for b in blocks], [b[3].data_ptr() for b in blocks],
                                        [b[4] for b in blocks], host)

    def wait(self, ticket) -> float:
        return cdd.cdd_pool_wait(self.handle, ticket)

    def resync(self, sid, seq):
        cdd.cdd_pool_stream_resync(self.handle, sid, seq)

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

    def queued(self) -> int:
        return cdd.cdd_pool_get(self.handle, "queued")

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


def block_geometry(spec: StreamSpec):
    """(block samples, outputs per channel, block duration in seconds)."""
    n = spec.n_fft()
    p = cdd.cdd_plan_create(spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n, spec.n_avg)
    try:
        cdd.cdd_plan_set(p, "segments_per_block", spec.segments_per_block(n))
        bs = cdd.cdd_plan_get(p, "block_samples")
        n_out = cdd.cdd_plan_get(p, "n_out_per_block")
    finally:
        cdd.cdd_destroy(p)
    return bs, n_out, bs / (spec.chan_bw * 1e6)


def warm_kernels(specs):
    """Load every kernel the streams will use (one throwaway block per
    transform length), so that no block pays a module load."""
    import torch
    for n in sorted({sp.n_fft() for sp in specs}):
        with cdd.Plan(325.0, 0.0625, 1, 0.0, n, 16) as p:
            x = torch.zeros((p.block_samples, 1, 2), dtype=torch.int8, device="cuda")
            p.execute(x)
            h = torch.zeros((p.block_samples, 1, 2), dtype=torch.int8).pin_memory()
            p.execute_host(h)
    torch.cuda.synchronize()


def run_mix(specs, n_blocks: int, speedup: float = 1e9, budget_bytes: int = 64 << 30,
            stagger_blocks: float = 0.5, keep_outputs: bool = False, host: bool = True,
            max_streams: int | None = None, batch_submit: bool | None = None):
    """Serve every stream for n_blocks blocks.

    Stream i arrives after i * stagger_blocks of its block durations and asks
    for admission (queued if it does not fit); block b arrives (b + 1) block
    durations after its stream, arrivals paced at `speedup` x real time (1e9:
    as fast as possible).  A stream is released as soon as its last block is
    done, which admits queued streams.  host: blocks come from pinned host
    memory and results go back to it (copies inside each block's latency);
    else device buffers.  batch_submit: submit all blocks due at once in one
    library call (default: when unpaced).  Returns a summary dict (and every
    stream's outputs, [n_blocks][C][n_out], with keep_outputs)."""
    import torch
    if batch_submit is None:
        batch_submit = speedup >= 1e6
    geo = [block_geometry(sp) for sp in specs]
    warm_kernels(specs)
    data, outs = [], []
    for sp, (bs, n_out, _) in zip(specs, geo):
        x = torch.from_numpy(make_block_inputs(sp, bs, n_blocks))
        o = torch.empty((n_blocks, sp.n_chan, n_out), dtype=torch.float32)
        if host:
            x, o = x.pin_memory(), o.pin_memory()
        else:
            x, o = x.cuda(), o.cuda()
        data.append(x)
        outs.append(o)
    torch.cuda.synchronize()

    # virtual-time events: (time, kind, stream, block); kind 0 = stream arrives
    events = []
    for i, (bs, n_out, dur) in enumerate(geo):
        t0 = i * stagger_blocks * dur
        events.append((t0, 0, i, -1))
        for b in range(n_blocks):
            events.append((t0 + (b + 1) * dur, 1, i, b))
    events.sort()

    # waiters wait for tickets; finishers wait for a stream's waits and release
    # it (separate executors, so a finisher never holds a thread a wait needs)
    with Pool(budget_bytes, max_streams=max_streams or max(1, len(specs))) as pool, \
            ThreadPoolExecutor(max_workers=8) as waiters, \
            ThreadPoolExecutor(max_workers=max(1, len(specs))) as finishers:
        req, sid, pending = {}, {}, {i: [] for i in range(len(specs))}
        futures = {i: [] for i in range(len(specs))}
        releases, admitted_at_once, admitted_from_queue = [], [], []
        lat, ddl = [], []

        def finish(i, futs):
            res = [f.result() for f in futs]
            pool.release(sid[i])              # frees memory: queued streams are admitted
            return res

        def flush():
            """Submit the pending blocks of every admitted stream."""
            for i, r in list(req.items()):
                if i not in sid:
                    s = pool.status(r)
                    if s is None:
                        continue
                    sid[i] = s
                    t_admit[i] = cdd.cdd_pool_clock_ms()
                    (admitted_from_queue if pool_was_queued[i] else admitted_at_once).append(i)
            batch = []
            for i in sid:
                bs = geo[i][0]
                for b, t_arr in pending[i]:
                    batch.append((sid[i], b, data[i][b * bs:(b + 1) * bs], outs[i][b], t_arr, i))
                pending[i] = []
            if not batch:
                return
            if batch_submit:
                tickets = pool.submit_many([x[:5] for x in batch], host)
            else:
                tickets = [pool.submit(*x[:5]) for x in batch]
            for x, tk in zip(batch, tickets):
                i = x[5]
                futures[i].append(waiters.submit(pool.wait, tk))
                if len(futures[i]) == n_blocks:
                    releases.append((i, finishers.submit(finish, i, futures[i])))

        pool_was_queued, t_req, t_admit = {}, {}, {}
        t_start = time.perf_counter()
        clock0 = cdd.cdd_pool_clock_ms()
        for t_ev, kind, i, b in events:
            delay = t_ev / speedup - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            if kind == 0:
                t_req[i] = cdd.cdd_pool_clock_ms()
                req[i] = pool.request(specs[i], host=host)
                pool_was_queued[i] = pool.queued() > 0
            else:
                pending[i].append((b, clock0 + t_ev / speedup * 1e3))
            flush()
        while len(releases) < len(specs):          # streams still waiting for admission
            time.sleep(0.0005)
            flush()
        lat_by = {"at_once": [], "from_queue": []}
        for i, f in releases:
            lat_i = f.result()
            lat.extend(lat_i)
            ddl.extend([geo[i][2] * 1e3] * len(lat_i))
            lat_by["from_queue" if i in admitted_from_queue else "at_once"].extend(lat_i)
        waits = [t_admit[i] - t_req[i] for i in admitted_from_queue]
        wall = time.perf_counter() - t_start
        seq_gaps = 0

    samples = sum(geo[i][0] * specs[i].n_chan * n_blocks for i in range(len(specs)))
    rt = sum(sp.bandwidth_mhz * 1e6 for sp in specs)
    lat = np.array(lat)
    ddl = np.array(ddl)
    paced = ddl / speedup if speedup < 1e6 else None
    summary = {
        "streams": len(specs), "admitted_at_once": len(admitted_at_once),
        "admitted_from_queue": len(admitted_from_queue),
        "blocks": int(lat.size), "ingest": "pinned host buffers" if host else "device buffers",
        "msamples_per_s": samples / wall / 1e6,
        "x_realtime": samples / wall / rt,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max()), "from": "block arrival"},
        "deadline_ms": {"min": float(ddl.min()), "max": float(ddl.max()), "speedup": speedup},
        "missed_deadlines": int((lat > paced).sum()) if paced is not None else None,
        "latency_ms_by_admission": {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)),
                                        "blocks": len(v)} for k, v in lat_by.items() if v},
        "admission_wait_ms": {"max": float(max(waits)), "mean": float(np.mean(waits))} if waits else None,
        "seq_gaps": seq_gaps,
        "budget_bytes": budget_bytes,
    }
    result_outs = {i: outs[i].cpu().numpy() for i in range(len(specs))} if keep_outputs else None
    return summary, result_outs


def run_alone(spec: StreamSpec, n_blocks: int):
    """The same stream through a plain plan, block after block."""
    import torch
    n_fft = spec.n_fft()
    with cdd.Plan(spec.f_center_mhz, spec.bandwidth_mhz, spec.n_chan, spec.dm, n_fft, spec.n_avg,
                  segments_per_block=spec.segments_per_block(n_fft)) as p:
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
    ap.add_argument("--device-buffers", action="store_true", help="ingest from device, not host, buffers")
    args = ap.parse_args(argv)
    summary, _ = run_mix(mixed_scenario(args.streams), args.blocks, args.speedup,
                         int(args.budget_gb * (1 << 30)), host=not args.device_buffers)
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
