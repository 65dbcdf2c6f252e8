"""Recovery of injected pulses against their truth (GPU).

The inputs carry pulse trains dispersed as the interstellar medium disperses
them: delayed across channels by the cold-plasma law and chirped inside each
channel by exp(+i Phi), Phi the Eq. 3 phase (the response is taken from the
oracle and handed to synth).  The library dedisperses, aligns and band-sums
the channels; each pulse must then appear at its truth time (the centre of
its excess power within +-1 integrated sample of the truth centre) with
close to the SNR the workload states, SNR = (sigma_p^2 / sigma^2) sqrt(C W).
The boxcar that measures it is ceil(W / n_avg) + 2 outputs long: the
channels are aligned to whole outputs (up to half an output apart), and the
pulse starts anywhere inside an output, so a shorter box can miss part of
it.  A box of B outputs holding all of the pulse's power reads
SNR sqrt(W / (n_avg B)); the test asks for 0.8 to 1.15 of that.  The batched
form must also put the highest peak on the DM trial the pulse was
dispersed with.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import WORKLOADS, PulseTrain, complex_int8_voltages

pytestmark = pytest.mark.gpu


def dispersing_response(f_lo_mhz, chan_bw_mhz, dm):
    def resp(L):
        f_l = O.bin_offsets(L, chan_bw_mhz)
        return np.exp(1j * O.chirp_phase(np.asarray(f_lo_mhz)[:, None], f_l[None, :], dm))
    return resp


def dispersed_pulses(f_lo_mhz, chan_bw_mhz, dm, start, period, width, sigma_p, window=256):
    offs = O.dispersion_delay_s(f_lo_mhz, f_lo_mhz[0], dm) * chan_bw_mhz * 1e6
    return PulseTrain(start, period, width, sigma_p, offs,
                      response=dispersing_response(f_lo_mhz, chan_bw_mhz, dm), window=window)


def box_outputs(width, n_avg):
    return int(math.ceil(width / n_avg)) + 2


def expected_snr(snr, width, n_avg):
    return snr * math.sqrt(width / (n_avg * box_outputs(width, n_avg)))


def recovered(series, n_avg, width, starts, m_lo):
    """(centre offsets in integrated samples, boxcar SNRs) of the pulses that
    start at channel-0 samples `starts`, from the band-summed series."""
    nb = box_outputs(width, n_avg)
    box = np.convolve(series, np.ones(nb), "valid")          # box[m] = sum series[m:m+nb]
    off = np.ones(box.size, bool)
    off[:m_lo] = False
    for t in starts:
        m0 = int(t // n_avg)
        off[max(0, m0 - 3 * nb):m0 + 3 * nb] = False
    mu, sd = box[off].mean(), box[off].std()
    excess_level = np.median(series[m_lo:])
    centres, snrs = [], []
    for t in starts:
        m0 = int(t // n_avg)
        lo = max(0, m0 - nb - 2)
        pk = lo + int(np.argmax(box[lo:m0 + 3]))
        snrs.append((box[pk] - mu) / sd)
        seg = np.arange(max(0, m0 - 2 * nb), m0 + 3 * nb)
        ex = np.clip(series[seg] - excess_level, 0, None)
        centres.append(float((seg * ex).sum() / ex.sum()) + 0.5 - (t + width / 2) / n_avg)
    return np.array(centres), np.array(snrs)


def band_series(out):
    from paper_1509_00186_b300.cdd import band_sum
    return band_sum(out)


def test_tiny_pulses_recovered(cuda_device):
    """16 MHz / 256 channels / DM 10, 0.5 s, N 64, x4: two pulses of 1 ms at SNR 50."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    w = WORKLOADS["tiny"]
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    start = 4000.0
    pulses = dispersed_pulses(geo.f_lo_mhz, w.chan_bw_mhz, w.dm, start, w.period_samples,
                              w.width_samples, w.pulse_sigma)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)
    q = w.n_samp // geo.hop
    with Plan(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg,
              segments_per_block=q) as plan:
        out = plan.execute(torch.from_numpy(np.ascontiguousarray(vin[:q * geo.hop])).cuda())
        series = band_series(out).cpu().numpy()
    starts = [start + p * w.period_samples for p in range(2)]
    c, snr = recovered(series, w.n_avg, w.width_samples, starts, int(geo.shift.max()))
    want = expected_snr(w.pulse_snr, w.width_samples, w.n_avg)
    assert np.all(np.abs(c) <= 1.0), c
    assert np.all((snr > 0.8 * want) & (snr < 1.15 * want)), (snr, want)


@pytest.mark.slow
def test_gsb_pulse_train_recovered(cuda_device):
    """32 MHz / 512 channels / DM 50, 10 s, N 8192, x16 (one block of 76
    segments, the benchmark's launch): every pulse of the 33 ms train after the
    alignment fill-in, at its truth time and SNR."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    w = WORKLOADS["gsb"]
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    start = 3000.0
    pulses = dispersed_pulses(geo.f_lo_mhz, w.chan_bw_mhz, w.dm, start, w.period_samples,
                              w.width_samples, w.pulse_sigma)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)
    q = w.n_samp // geo.hop
    with Plan(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg,
              segments_per_block=q) as plan:
        out = plan.execute(torch.from_numpy(np.ascontiguousarray(vin[:q * geo.hop])).cuda())
        series = band_series(out).cpu().numpy()
    m_lo = int(geo.shift.max()) + 8
    n_out = series.size
    starts = [start + p * w.period_samples for p in range(400)]
    starts = [t for t in starts if m_lo * w.n_avg <= t and (t + w.width_samples) / w.n_avg + 8 < n_out]
    assert len(starts) > 250
    c, snr = recovered(series, w.n_avg, w.width_samples, starts, m_lo)
    want = expected_snr(w.pulse_snr, w.width_samples, w.n_avg)
    assert np.all(np.abs(c) <= 1.0), np.abs(c).max()
    assert np.all((snr > 0.8 * want) & (snr < 1.15 * want)), (snr.min(), snr.max(), want)


@pytest.mark.slow
def test_upgraded_gmrt_batch_finds_the_dm_35_pulse(cuda_device):
    """200 MHz at 650 MHz, 2048 channels, 64 DM trials 20.0..51.5, 4 s, one
    pulse of 1 ms at DM 35 with SNR 50: the DM 35 plane of the band-summed
    batch output holds the highest peak, at the pulse's truth time and close
    to its SNR."""
    import torch
    from paper_1509_00186_b300.cdd import Batch
    dms = list(20.0 + 0.5 * np.arange(64))
    args = (650.0, 200.0, 2048, dms, (16384, 8192, 4096, 2048), 16)
    g = O.batch_geometry(*args)
    C, n_avg, sigma, snr_want = 2048, 16, 20.0, 50.0
    rate = g.chan_bw_mhz * 1e6
    width = int(round(1e-3 * rate))
    sigma_p = sigma * math.sqrt(snr_want / math.sqrt(C * width))
    start = 1.2 * rate                                # 1.2 s into the record at channel 0
    pulses = dispersed_pulses(g.f_lo_mhz, g.chan_bw_mhz, 35.0, start, 1e12, width, sigma_p)
    n_samp = int(round(4.0 * 200e6 / 2048))
    q = n_samp // g.hop(0)
    vin = complex_int8_voltages(41, q * g.hop(0), C, sigma, pulses)
    with Batch(*args, segments_per_block=q) as b:
        out = b.execute(torch.from_numpy(vin).cuda())
        series = band_series(out).cpu().numpy()           # [64][n_out]
    m_lo = int(g.shift.max()) + 8
    peaks = []
    for d in range(len(dms)):
        _, snr = recovered(series[d], n_avg, width, [start], m_lo)
        peaks.append(snr[0])
    peaks = np.array(peaks)
    d35 = dms.index(35.0)
    assert int(np.argmax(peaks)) == d35, peaks
    c, snr = recovered(series[d35], n_avg, width, [start], m_lo)
    want = expected_snr(snr_want, width, n_avg)
    assert abs(c[0]) <= 1.0, c
    assert 0.8 * want < snr[0] < 1.15 * want, (snr, want)
    assert peaks[d35 - 1] < 0.8 * peaks[d35] and peaks[d35 + 1] < 0.8 * peaks[d35]
