"""FP64 CPU oracle for per-channel overlap-save coherent dedispersion.

TEST INFRASTRUCTURE ONLY. This module is the slow, plain statement of what the
GPU path computes, used to check it. Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does.

It follows De & Gupta, "A Real-time Coherent Dedispersion Pipeline for the
GMRT" (arXiv:1509.00186), in the paper's order:

  Sec. 2.1, Eq. 1-3   the ISM transfer function and its dispersive (chirp) term
  Sec. 2.2            the taper ("chirp function") and overlap-save deconvolution
  Sec. 2.3            the FFT-length rule
  Sec. 3.1 / 4.3      detection (squaring) and integration of the voltages
  Sec. 1.2 / 1.3      time alignment of the coherently dedispersed sub-bands

Everything is numpy float64 / complex128. The only library primitives used as
steps are numpy's FFT (forward sign -, inverse scaled by 1/N), pinned against a
brute-force DFT in the tests.

Readings of points the paper leaves open (each is listed in the design notes):
  * the ISM multiplies a channel's spectrum by exp(+i*Phi) under a forward
    exp(-i...) DFT, so dedispersion multiplies by exp(-i*Phi) (Sec. 2.1 says the
    correction is the inverse of the third term of Eq. 2);
  * f_o of Eq. 3 is the lower edge of each channel; a channel's complex baseband
    bin j sits at f_l = fftfreq(j)*chan_bw + chan_bw/2 (the Nyquist bin at f_l=0);
  * D = 4.148808e3 s MHz^2 cm^3/pc (the paper's 4.148808e9 with Phi in MHz*us);
  * the overlap n_ov is ceil(n_d) of the lowest channel rounded up to a multiple
    of the integration length, and is discarded at the segment START (Sec. 2.2);
  * the inverse DFT carries 1/N; integration is a sum, not a mean;
  * channels are aligned to the lowest channel by r_k = rint(delay_k / t_int).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Dispersion constant of Eq. 3, in s MHz^2 cm^3 pc^-1 (frequencies in MHz give
# seconds).  The paper prints it as 4.148808e9 for a phase with f in MHz and time
# in microseconds; the two differ by the 1e6 that ``chirp_phase`` applies.
D_DISP_S_MHZ2 = 4.148808e3

TAPERS = ("none", "hann", "welch")


# --------------------------------------------------------------------------
# Geometry (Sec. 2.1, Sec. 2.3)
# --------------------------------------------------------------------------

def channel_lower_edges(f_center_mhz: float, bandwidth_mhz: float, n_chan: int):
    """Lower edge f_k of every channel and the channel width (Sec. 2.1: f_o is the
    lower edge of the band).  Upper sideband (bandwidth > 0): channel 0 is the
    lowest.  Lower sideband (bandwidth < 0): channel 0 is the highest, so
    f_k = f_center + |B|/2 - (k + 1) * chan_bw."""
    chan_bw = abs(bandwidth_mhz) / n_chan
    k = np.arange(n_chan, dtype=np.float64)
    if bandwidth_mhz > 0:
        f_lo = f_center_mhz - bandwidth_mhz / 2.0 + chan_bw * k
    else:
        f_lo = f_center_mhz + abs(bandwidth_mhz) / 2.0 - chan_bw * (k + 1.0)
    return f_lo, chan_bw


def dispersion_delay_s(f_mhz, f_ref_mhz, dm: float):
    """Cold-plasma arrival delay of frequency f relative to f_ref, in seconds
    (positive when f is below f_ref).  Sec. 1.2: the delay grows as 1/f^2."""
    f = np.asarray(f_mhz, dtype=np.float64)
    return D_DISP_S_MHZ2 * dm * (f ** -2 - float(f_ref_mhz) ** -2)


def dispersion_samples(f_lo_mhz: float, chan_bw_mhz: float, dm: float) -> float:
    """Dispersion time across one channel [f_lo, f_lo + chan_bw], in complex
    samples of that channel (sample rate chan_bw MHz).  Sec. 2.2: this is the
    length of the impulse response that has to be deconvolved."""
    t = dispersion_delay_s(f_lo_mhz, f_lo_mhz + chan_bw_mhz, dm)
    return float(t * chan_bw_mhz * 1e6)


def _next_pow2_above(x: float) -> int:
    n = 1
    while n <= x:
        n *= 2
    return n


@dataclass(frozen=True)
class Geometry:
    n_chan: int
    chan_bw_mhz: float
    f_lo_mhz: np.ndarray      # [C] lower channel edges
    dm: float
    n_fft: int                # N
    n_ov: int                 # samples discarded per segment (overlap)
    hop: int                  # h = N - n_ov, new samples per segment
    n_avg: int                # integration length
    n_disp: float             # dispersion samples of the lowest channel
    shift: np.ndarray         # [C] int64 alignment shift r_k in integrated samples
    sideband: int = 1         # +1 upper, -1 lower


def plan_geometry(f_center_mhz: float, bandwidth_mhz: float, n_chan: int, dm: float,
                  n_fft: int = 0, n_avg: int = 1) -> Geometry:
    """Segment geometry of the per-channel overlap-save.

    * n_d: dispersion samples of the lowest channel (longest smear), Sec. 2.2.
    * n_ov = ceil(n_d) rounded up to a multiple of n_avg (so every integration
      window stays inside one segment).
    * N: given, or (n_fft == 0) the Sec. 2.3 rule -- the smallest power of two
      greater than twice n_d -- raised if needed so that N > n_ov, N >= 2*n_avg
      and N >= 64 (the smallest transform the GPU path runs).
    * r_k = rint(delay of f_k relative to f_0, in integrated samples), Sec. 1.2.
    """
    if n_chan <= 0 or n_avg <= 0 or bandwidth_mhz == 0 or dm < 0:
        raise ValueError("n_chan, n_avg must be positive, bandwidth non-zero and DM >= 0")
    f_lo, chan_bw = channel_lower_edges(f_center_mhz, bandwidth_mhz, n_chan)
    n_d = dispersion_samples(float(f_lo.min()), chan_bw, dm)
    n_ov = int(math.ceil(n_d))
    n_ov = -(-n_ov // n_avg) * n_avg
    if n_fft == 0:
        n_fft = max(_next_pow2_above(2.0 * n_d), _next_pow2_above(n_ov), 64)
        while n_fft < 2 * n_avg:
            n_fft *= 2
    if n_fft & (n_fft - 1) or n_fft <= n_ov:
        raise ValueError(f"N={n_fft} must be a power of two larger than n_ov={n_ov}")
    hop = n_fft - n_ov
    if hop % n_avg:
        raise ValueError(f"hop {hop} is not a multiple of n_avg {n_avg}")
    delay = dispersion_delay_s(f_lo, f_lo.min(), dm)         # <= 0: higher channels lead
    shift = np.rint(-delay * chan_bw * 1e6 / n_avg).astype(np.int64)
    return Geometry(n_chan, chan_bw, f_lo, float(dm), int(n_fft), int(n_ov), int(hop),
                    int(n_avg), float(n_d), shift, 1 if bandwidth_mhz > 0 else -1)


# --------------------------------------------------------------------------
# The chirp (Sec. 2.1, Eq. 3) and taper (Sec. 2.2)
# --------------------------------------------------------------------------

def bin_offsets(n_fft: int, chan_bw_mhz: float) -> np.ndarray:
    """f_l (MHz above the channel's lower edge) of each DFT bin j of a complex
    baseband channel: numpy's fftfreq order plus half a channel, so f_l is in
    [0, chan_bw) and the Nyquist bin j = N/2 lands on f_l = 0."""
    return np.fft.fftfreq(n_fft, d=1.0 / chan_bw_mhz) + chan_bw_mhz / 2.0


def chirp_phase(f_lo_mhz, f_l_mhz, dm: float):
    """Phase (radians) of Eq. 3, the dispersive term of the ISM transfer function:
    Phi = 2*pi * D * DM * f_l^2 / ((f_l + f_o) * f_o^2), frequencies in MHz."""
    f_lo = np.asarray(f_lo_mhz, dtype=np.float64)
    f_l = np.asarray(f_l_mhz, dtype=np.float64)
    return 2.0 * np.pi * D_DISP_S_MHZ2 * 1e6 * dm * f_l ** 2 / ((f_l + f_lo) * f_lo ** 2)


def taper(f_l_mhz, chan_bw_mhz: float, kind: str = "none"):
    """Frequency-domain window of Sec. 2.2 (the paper names Hann and Welch but
    prints neither): Hann sin^2(pi x), Welch 1 - (2x - 1)^2, x = f_l / chan_bw."""
    x = np.asarray(f_l_mhz, dtype=np.float64) / chan_bw_mhz
    if kind == "none":
        return np.ones_like(x)
    if kind == "hann":
        return np.sin(np.pi * x) ** 2
    if kind == "welch":
        return 1.0 - (2.0 * x - 1.0) ** 2
    raise ValueError(f"unknown taper {kind!r}")


def dedispersion_filter(f_lo_mhz: float, chan_bw_mhz: float, dm: float, n_fft: int,
                        taper_kind: str = "none", sideband: int = 1) -> np.ndarray:
    """The "chirp function" of Sec. 2.2 for one channel on an N-point grid: the
    taper times the inverse of Eq. 3's term, conj(H) = exp(-i*Phi).

    A lower-sideband channel carries the conjugate of the upper-sideband
    baseband of the same sky band (frequency runs downward), so its bin j sits
    where the upper-sideband bin -j (mod N) does -- f_l = chan_bw/2 - nu_j, with
    the Nyquist bin its own mirror at f_l = 0 -- and the correction is the
    conjugate: exp(+i*Phi)."""
    f_l = bin_offsets(n_fft, chan_bw_mhz)
    if sideband > 0:
        return np.conj(np.exp(1j * chirp_phase(f_lo_mhz, f_l, dm))) * taper(f_l, chan_bw_mhz, taper_kind)
    f_l = f_l[(-np.arange(n_fft)) % n_fft]
    return np.exp(1j * chirp_phase(f_lo_mhz, f_l, dm)) * taper(f_l, chan_bw_mhz, taper_kind)


# --------------------------------------------------------------------------
# Overlap-save deconvolution (Sec. 2.2, Sec. 4.3)
# --------------------------------------------------------------------------

def dft(x: np.ndarray) -> np.ndarray:
    """Forward DFT X[j] = sum_n x[n] exp(-2 pi i j n / N) along the last axis."""
    return np.fft.fft(x, axis=-1)


def idft(X: np.ndarray) -> np.ndarray:
    """Inverse DFT x[n] = (1/N) sum_j X[j] exp(+2 pi i j n / N) along the last axis."""
    return np.fft.ifft(X, axis=-1)


def overlap_save(x: np.ndarray, filt: np.ndarray, n_ov: int,
                 history: np.ndarray | None = None) -> np.ndarray:
    """Overlap-save convolution of one channel's complex series with the N-point
    filter spectrum ``filt`` (Sec. 2.2).

    Segment s takes N consecutive inputs starting n_ov samples before s*h
    (h = N - n_ov), so consecutive segments overlap by n_ov.  After the forward
    DFT, the product with the filter and the inverse DFT, the first n_ov outputs
    are discarded and the remaining h are kept.  The samples before the start of
    the stream are ``history`` (the last n_ov samples of earlier data), or zeros
    (Sec. 4.3: the lost samples are prefixed to the next block).
    Only whole segments are processed: len(x) // h of them.
    """
    n_fft = filt.shape[-1]
    hop = n_fft - n_ov
    n_seg = x.shape[-1] // hop
    if history is None:
        history = np.zeros(n_ov, dtype=np.complex128)
    xp = np.concatenate([np.asarray(history, dtype=np.complex128),
                         np.asarray(x, dtype=np.complex128)])
    out = np.empty(n_seg * hop, dtype=np.complex128)
    if n_seg == 0:
        return out
    segs = np.lib.stride_tricks.sliding_window_view(xp, n_fft)[::hop][:n_seg]
    y = idft(dft(segs) * filt)
    out[:] = y[:, n_ov:].reshape(-1)
    return out


# --------------------------------------------------------------------------
# Detection, integration and alignment (Sec. 3.1, Sec. 4.3, Sec. 1.2)
# --------------------------------------------------------------------------

def detect(v: np.ndarray) -> np.ndarray:
    """Square the dedispersed voltage: |v|^2 (Sec. 3.1 "squares it")."""
    return v.real ** 2 + v.imag ** 2


def integrate(p: np.ndarray, n_avg: int) -> np.ndarray:
    """Sum n_avg consecutive detected samples (Sec. 3.1 "integrates it to a given
    number of samples"); trailing samples that do not fill a window are dropped."""
    n = (p.shape[-1] // n_avg) * n_avg
    return p[..., :n].reshape(*p.shape[:-1], -1, n_avg).sum(axis=-1)


def align(intensity: np.ndarray, shift: int) -> np.ndarray:
    """Delay one channel's integrated series by ``shift`` samples (Sec. 1.2: the
    sub-bands are aligned in time by applying their dispersion delays);
    Out[m] = I[m - shift], zero before the series starts."""
    out = np.zeros_like(intensity)
    if shift < intensity.shape[-1]:
        out[shift:] = intensity[: intensity.shape[-1] - shift]
    return out


# --------------------------------------------------------------------------
# Whole path
# --------------------------------------------------------------------------

def unpack(vin: np.ndarray, k: int) -> np.ndarray:
    """Channel k of int8 [T][C][2] (re, im; two's complement, Sec. 2.3 "8-bit
    integers") as complex128 [T]."""
    if vin.dtype != np.int8 or vin.ndim != 3 or vin.shape[2] != 2:
        raise ValueError("input must be int8 [T][C][2]")
    return vin[:, k, 0].astype(np.float64) + 1j * vin[:, k, 1].astype(np.float64)


def dedisperse(vin: np.ndarray, geo: Geometry, taper_kind: str = "none",
               return_voltages: bool = False, channels=None):
    """The whole hot path on one record, from the start of the stream.

    vin: int8 [T][C][2].  Returns Out float64 [C'][n_out] with
    n_out = (T // h) * h / n_avg, and, if asked, the dedispersed voltages
    complex128 [C'][(T // h) * h].  ``channels`` restricts the work to a subset
    (C' of them) for bounded timing runs.
    """
    chans = range(geo.n_chan) if channels is None else list(channels)
    outs, volts = [], []
    for k in chans:
        filt = dedispersion_filter(float(geo.f_lo_mhz[k]), geo.chan_bw_mhz, geo.dm,
                                   geo.n_fft, taper_kind, geo.sideband)
        v = overlap_save(unpack(vin, k), filt, geo.n_ov)
        i_k = integrate(detect(v), geo.n_avg)
        outs.append(align(i_k, int(geo.shift[k])))
        if return_voltages:
            volts.append(v)
    out = np.stack(outs) if outs else np.zeros((0, 0))
    if return_voltages:
        return out, np.stack(volts)
    return out


def rel_rms(a: np.ndarray, b: np.ndarray) -> float:
    """sqrt(sum |a-b|^2 / sum |b|^2): the error measure stated per output array."""
    a = np.asarray(a)
    b = np.asarray(b)
    den = float(np.sum(np.abs(b) ** 2))
    num = float(np.sum(np.abs(a - b) ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return math.sqrt(num / den)


# --------------------------------------------------------------------------
# Batched form: many DM trials over a band whose channel groups (tiers) use
# different transform lengths
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class BatchGeometry:
    n_chan: int
    chan_bw_mhz: float
    f_lo_mhz: np.ndarray      # [C]
    dms: np.ndarray           # [D]
    tier_nfft: tuple          # N of each tier, lowest-frequency tier first
    tier_nov: tuple           # overlap of each tier
    n_avg: int
    tier_of: np.ndarray       # [C] tier index of each channel
    shift: np.ndarray         # [D][C] alignment shifts, integrated samples
    sideband: int = 1         # +1 upper, -1 lower (channel 0 highest)

    def hop(self, t: int) -> int:
        return self.tier_nfft[t] - self.tier_nov[t]


def batch_geometry(f_center_mhz: float, bandwidth_mhz: float, n_chan: int, dms, tier_nfft,
                   n_avg: int) -> BatchGeometry:
    """Geometry of the batched form.

    The band is cut into len(tier_nfft) equal groups of channels, lowest
    frequencies first (for a lower sideband, bandwidth < 0, channel 0 is the
    highest, so tier 0 holds the last channels); tier t coherently dedisperses
    with N_t points.  Its overlap is N_t/32, raised if needed to the dispersion
    samples of the tier's lowest channel at the largest DM (Sec. 2.2: at least
    the impulse response) and rounded up to a multiple of n_avg.  Shifts follow
    the single-DM rule for every DM (Sec. 1.2), relative to the band's lowest
    channel."""
    dms = np.asarray(dms, dtype=np.float64)
    n_t = len(tier_nfft)
    if n_chan % n_t or np.any(dms < 0) or dms.size == 0 or bandwidth_mhz == 0:
        raise ValueError("channels must split evenly into tiers; DMs >= 0; bandwidth non-zero")
    f_lo, chan_bw = channel_lower_edges(f_center_mhz, bandwidth_mhz, n_chan)
    per = n_chan // n_t
    k = np.arange(n_chan)
    tier_of = k // per if bandwidth_mhz > 0 else (n_chan - 1 - k) // per
    nov = []
    for t, n in enumerate(tier_nfft):
        n_d = dispersion_samples(float(f_lo[tier_of == t].min()), chan_bw, float(dms.max()))
        ov = max(n // 32, int(math.ceil(n_d)))
        ov = -(-ov // n_avg) * n_avg
        if n & (n - 1) or n <= ov or (n - ov) % n_avg:
            raise ValueError(f"tier {t}: N={n} does not fit overlap {ov} and n_avg {n_avg}")
        nov.append(ov)
    shift = np.stack([np.rint(-dispersion_delay_s(f_lo, f_lo.min(), dm) * chan_bw * 1e6 / n_avg)
                      for dm in dms]).astype(np.int64)
    return BatchGeometry(n_chan, chan_bw, f_lo, dms, tuple(int(n) for n in tier_nfft),
                         tuple(nov), int(n_avg), tier_of, shift, 1 if bandwidth_mhz > 0 else -1)


def dedisperse_batch(vin: np.ndarray, geo: BatchGeometry, channels=None, dm_index=None,
                     taper_kind: str = "none"):
    """Out[d][k][m] for every DM trial d: channel k runs the single-DM steps
    (overlap-save with its tier's N and overlap, the chirp with the taper,
    detection, integration, alignment) once per DM.  All channels are cut to
    the same number of outputs: whole segments of the longest hop."""
    chans = range(geo.n_chan) if channels is None else list(channels)
    dsel = range(len(geo.dms)) if dm_index is None else list(dm_index)
    h_max = max(geo.hop(t) for t in range(len(geo.tier_nfft)))
    n_samp = (vin.shape[0] // h_max) * h_max
    out = np.zeros((len(dsel), len(chans), n_samp // geo.n_avg))
    for ci, k in enumerate(chans):
        t = int(geo.tier_of[k])
        x = unpack(vin[:n_samp], k)
        for di, d in enumerate(dsel):
            filt = dedispersion_filter(float(geo.f_lo_mhz[k]), geo.chan_bw_mhz, float(geo.dms[d]),
                                       geo.tier_nfft[t], taper_kind, geo.sideband)
            v = overlap_save(x, filt, geo.tier_nov[t])
            out[di, ci] = align(integrate(detect(v), geo.n_avg), int(geo.shift[d, k]))
    return out


# --------------------------------------------------------------------------
# Band sum and polarisation sum (Sec. 1.2 incoherent addition; Sec. 4.3 two
# polarisations combined after detection)
# --------------------------------------------------------------------------

def band_sum(out: np.ndarray) -> np.ndarray:
    """Add the aligned channels: [..., C, n_out] -> [..., n_out] (Sec. 1.2: the
    aligned sub-bands are added to give the dedispersed time series)."""
    return np.asarray(out).sum(axis=-2)


def dedisperse_dual(vin_a: np.ndarray, vin_b: np.ndarray, geo: Geometry, taper_kind: str = "none"):
    """Two polarisations of one beam, each dedispersed and detected, summed
    after detection (Sec. 4.3 combines the polarisations after detection)."""
    return dedisperse(vin_a, geo, taper_kind) + dedisperse(vin_b, geo, taper_kind)


# --------------------------------------------------------------------------
# Full-band mode: the paper's own design (Sec. 2.3, Sec. 3.1, Sec. 4.3)
# --------------------------------------------------------------------------
#
# The voltage beam holds, for every frame t, the C complex outputs of a 2C-point
# FFT of the real, Nyquist-sampled voltage (Sec. 2.3, Sec. 3.1).  The
# inverse transform of each frame gives back 2C real samples; the frames in
# series are the continuous real time series at 2B samples per second.  One
# long real FFT over the whole band, the chirp on its N/2 bins, the inverse FFT
# and overlap-save then dedisperse it coherently without sub-banding
# (Sec. 2.3, Sec. 4.3), and the result is squared and integrated (Sec. 3.1).

@dataclass(frozen=True)
class FullbandGeometry:
    f_lo_mhz: float           # lower edge of the band
    bandwidth_mhz: float
    n_chan: int               # C: complex outputs per frame
    frame: int                # 2C real samples per frame
    fs_mhz: float             # real sample rate 2B
    dm: float
    n_fft: int                # N (real points)
    n_ov: int
    hop: int
    n_avg: int
    n_disp: float             # dispersion samples across the whole band
    sideband: int = 1         # +1 upper; -1 lower: the series is the band inverted


def fullband_geometry(f_center_mhz: float, bandwidth_mhz: float, n_chan: int, dm: float,
                      n_fft: int = 0, n_avg: int = 1) -> FullbandGeometry:
    """Sec. 2.3: N is the smallest power of two greater than twice the
    dispersion samples across the band (real samples at 2B).  The overlap is
    the dispersion samples rounded up to a whole number of frames and of
    integration windows, so segments and blocks stay on frame boundaries."""
    if n_chan <= 0 or n_avg <= 0 or bandwidth_mhz == 0 or dm < 0:
        raise ValueError("n_chan, n_avg must be positive, bandwidth non-zero and DM >= 0")
    sideband = 1 if bandwidth_mhz > 0 else -1
    bandwidth_mhz = abs(bandwidth_mhz)
    f_lo = f_center_mhz - bandwidth_mhz / 2.0
    fs = 2.0 * bandwidth_mhz
    n_d = float(dispersion_delay_s(f_lo, f_lo + bandwidth_mhz, dm) * fs * 1e6)
    frame = 2 * n_chan
    unit = max(frame, n_avg)
    if unit % frame or unit % n_avg:
        raise ValueError("frame and n_avg must be powers of two")
    n_ov = -(-int(math.ceil(n_d)) // unit) * unit
    if n_fft == 0:
        n_fft = max(_next_pow2_above(2.0 * n_d), _next_pow2_above(n_ov), 2 * unit)
    if n_fft & (n_fft - 1) or n_fft <= n_ov or (n_fft - n_ov) % unit:
        raise ValueError(f"N={n_fft} does not fit overlap {n_ov}")
    return FullbandGeometry(f_lo, bandwidth_mhz, n_chan, frame, fs, float(dm), int(n_fft),
                            int(n_ov), int(n_fft - n_ov), int(n_avg), n_d, sideband)


def inverse_channelise(vin: np.ndarray) -> np.ndarray:
    """int8 [T][C][2] spectra -> real float64 [T * 2C]: the inverse real FFT of
    every frame (bins 0..C-1 from the data, the Nyquist bin C zero; numpy's
    inverse real FFT keeps only the real part of bin 0), frames in series."""
    spec = vin[..., 0].astype(np.float64) + 1j * vin[..., 1].astype(np.float64)   # [T][C]
    full = np.concatenate([spec, np.zeros((spec.shape[0], 1))], axis=1)           # + Nyquist
    return np.fft.irfft(full, n=2 * spec.shape[1], axis=1).reshape(-1)


def fullband_filter(geo: FullbandGeometry, taper_kind: str = "none") -> np.ndarray:
    """The chirp function on the N/2 + 1 bins of the long real FFT (Sec. 4.3):
    bin j sits f_l = j * fs / N above the band's lower edge f_o (Eq. 3 with f_o
    the band edge, Sec. 2.1).  A lower-sideband series is the band inverted
    (bin j at B - j * fs / N above f_o, with the conjugate phase), so its
    correction is the conjugate of the upper-sideband one at that offset."""
    f_bb = np.arange(geo.n_fft // 2 + 1) * (geo.fs_mhz / geo.n_fft)
    f_l = f_bb if geo.sideband > 0 else geo.bandwidth_mhz - f_bb
    h = np.exp(1j * chirp_phase(geo.f_lo_mhz, f_l, geo.dm))
    corr = np.conj(h) if geo.sideband > 0 else h
    return corr * taper(f_l, geo.bandwidth_mhz, taper_kind)


def dedisperse_fullband(vin: np.ndarray, geo: FullbandGeometry, return_voltages: bool = False):
    """Inverse channelisation, then overlap-save with the long real FFT, the
    chirp and the inverse real FFT, then squaring and integration (zero history
    before the record).  Returns the intensity series float64 [n_seg*h/n_avg]."""
    x = inverse_channelise(vin)
    filt = fullband_filter(geo)
    n_seg = x.size // geo.hop
    xp = np.concatenate([np.zeros(geo.n_ov), x])
    v = np.empty(n_seg * geo.hop)
    for s in range(n_seg):
        u = xp[s * geo.hop: s * geo.hop + geo.n_fft]
        y = np.fft.irfft(np.fft.rfft(u) * filt, n=geo.n_fft)
        v[s * geo.hop:(s + 1) * geo.hop] = y[geo.n_ov:]
    out = integrate(v * v, geo.n_avg)
    return (out, v) if return_voltages else out
