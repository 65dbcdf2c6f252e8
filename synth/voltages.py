"""Seeded synthetic complex-int8 channel voltages.

Shared by the tests and the benchmark as the single source of inputs.  It holds
none of the dedispersion arithmetic: it draws Gaussian noise, adds pulses at the
per-channel sample offsets the caller passes in -- optionally filtered by a
per-channel frequency response the caller also passes in (to disperse them
inside each channel) -- rounds and clips to int8.

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
    from the caller (e.g. the cold-plasma delay of channel k, rounded).

    ``response`` (optional): a callable L -> complex [C][L] array, the caller's
    frequency response of every channel in numpy FFT bin order.  Each pulse is
    then filtered by it before it is added: the pulse sits at the centre of a
    zero-padded window of ``window`` samples (a power of two, with room on
    both sides for the response's spread), which is transformed, multiplied
    by the response and transformed back."""
    start: float
    period: float
    width: int
    sigma: float
    offsets: np.ndarray = field(default_factory=lambda: np.zeros(0))
    response: object = None
    window: int = 0


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
    filt = pulses.response is not None
    L = int(pulses.window) if filt else 0
    if filt and (L < 2 * pulses.width or L & (L - 1)):
        raise ValueError("the filter window must be a power of two of at least twice the width")
    # rows a pulse can touch: its boxcar, or its filter window [t0 - L/2, t0 + L/2)
    before, after = (L // 2, L // 2) if filt else (0, pulses.width)
    p_first = int(np.floor((r0 - after - hi_off - pulses.start) / pulses.period))
    p_last = int(np.ceil((r0 + n_rows + before - lo_off - pulses.start) / pulses.period))
    gain = None
    for p in range(max(p_first, 0), p_last + 1):
        # the pulse's own samples are drawn from a generator keyed on (seed, p),
        # so they do not depend on how the record is chunked
        prng = np.random.Generator(np.random.PCG64([seed, 1 + p]))
        amp = prng.standard_normal((pulses.width, n_chan, 2), dtype=np.float32)
        amp *= np.float32(pulses.sigma)
        t0 = np.rint(pulses.start + p * pulses.period + offs).astype(np.int64)  # [C]
        if filt:
            if gain is None:
                gain = np.asarray(pulses.response(L), dtype=np.complex128)
                if gain.shape != (n_chan, L):
                    raise ValueError("the response must be complex [C][window]")
            if not np.any((t0 + after > r0) & (t0 - before < r0 + n_rows)):
                continue
            z = np.zeros((n_chan, L), dtype=np.complex128)
            z[:, L // 2:L // 2 + pulses.width] = (amp[..., 0] + 1j * amp[..., 1]).T
            z = np.fft.ifft(np.fft.fft(z, axis=1) * gain, axis=1)
            rows = t0[None, :] - L // 2 + np.arange(L)[:, None]              # [L][C]
            vals = np.stack([z.real.T, z.imag.T], axis=-1).astype(np.float32)   # [L][C][2]
        else:
            rows = t0[None, :] + np.arange(pulses.width)[:, None]             # [W][C]
            vals = amp
        inside = (rows >= r0) & (rows < r0 + n_rows)
        if not inside.any():
            continue
        w_idx, k_idx = np.nonzero(inside)
        blk[rows[w_idx, k_idx] - r0, k_idx, :] += vals[w_idx, k_idx, :]
