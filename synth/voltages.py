"""Seeded synthetic complex-int8 channel voltages.

Shared by the tests and the benchmark as the single source of inputs.  It holds
none of the dedispersion arithmetic: it draws Gaussian noise, adds pulses at the
per-channel sample offsets the caller passes in, rounds and clips to int8.

Layout is the voltage-beam layout: int8 [T][C][2], time-major, channel fastest,
real part then imaginary part of each complex sample.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class PulseTrain:
    """A periodic train of noise-like pulses (complex Gaussian, per-component
    standard deviation ``sigma``) under a boxcar of ``width`` samples.

    ``start`` and ``period`` are in samples of channel 0; pulse p occupies
    [start + p*period + offset_k, ... + width) in channel k, where offset_k comes
    from the caller (e.g. the cold-plasma delay of channel k, rounded)."""
    start: float
    period: float
    width: int
    sigma: float
    offsets: np.ndarray = field(default_factory=lambda: np.zeros(0))


def complex_int8_voltages(seed: int, n_samp: int, n_chan: int, sigma: float = 20.0,
                          pulses: PulseTrain | None = None,
                          chunk_rows: int = 1 << 15) -> np.ndarray:
    """int8 [n_samp][n_chan][2]: i.i.d. N(0, sigma) per component, plus pulses,
    rounded to nearest and clipped to [-127, 127].  Deterministic in ``seed``."""
    out = np.empty((n_samp, n_chan, 2), dtype=np.int8)
    rng = np.random.Generator(np.random.PCG64(seed))
    for r0 in range(0, n_samp, chunk_rows):
        r1 = min(n_samp, r0 + chunk_rows)
        blk = rng.standard_normal((r1 - r0, n_chan, 2), dtype=np.float32)
        blk *= np.float32(sigma)
        if pulses is not None:
            _add_pulses(blk, r0, pulses, seed)
        np.rint(blk, out=blk)
        np.clip(blk, -127, 127, out=blk)
        out[r0:r1] = blk.astype(np.int8)
    return out


def _add_pulses(blk: np.ndarray, r0: int, pulses: PulseTrain, seed: int) -> None:
    n_rows, n_chan, _ = blk.shape
    offs = np.asarray(pulses.offsets, dtype=np.float64)
    if offs.size == 0:
        offs = np.zeros(n_chan)
    if offs.shape != (n_chan,):
        raise ValueError("pulse offsets must have one entry per channel")
    lo_off, hi_off = float(offs.min()), float(offs.max())
    # pulses that can touch rows [r0, r0 + n_rows)
    p_first = int(np.floor((r0 - pulses.width - hi_off - pulses.start) / pulses.period))
    p_last = int(np.ceil((r0 + n_rows - lo_off - pulses.start) / pulses.period))
    for p in range(max(p_first, 0), p_last + 1):
        # the pulse's own samples are drawn from a generator keyed on (seed, p),
        # so they do not depend on how the record is chunked
        prng = np.random.Generator(np.random.PCG64([seed, 1 + p]))
        amp = prng.standard_normal((pulses.width, n_chan, 2), dtype=np.float32)
        amp *= np.float32(pulses.sigma)
        t0 = np.rint(pulses.start + p * pulses.period + offs).astype(np.int64)  # [C]
        rows = t0[None, :] + np.arange(pulses.width)[:, None]                 # [W][C]
        inside = (rows >= r0) & (rows < r0 + n_rows)
        if not inside.any():
            continue
        w_idx, k_idx = np.nonzero(inside)
        blk[rows[w_idx, k_idx] - r0, k_idx, :] += amp[w_idx, k_idx, :]
