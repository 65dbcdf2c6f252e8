"""Pulses dispersed inside each channel (CPU).

synth takes the dispersing response from its caller; here the caller is the
test and the response is exp(+i Phi) of the oracle's Eq. 3 phase (the
interstellar medium's own transfer function, whose inverse the method
applies).  Checks: an identity response changes nothing; a pure delay moves
the pulse by whole samples; and the oracle's dedispersion of a noise-free
dispersed pulse puts its power back inside the pulse's own samples."""
import numpy as np

import oracle as O
from synth import PulseTrain, complex_int8_voltages


def dispersing_response(geo, dm):
    def resp(L):
        f_l = O.bin_offsets(L, geo.chan_bw_mhz)
        return np.exp(1j * O.chirp_phase(geo.f_lo_mhz[:, None], f_l[None, :], dm))
    return resp


def test_identity_response_changes_nothing():
    plain = complex_int8_voltages(3, 6000, 8, 20.0, PulseTrain(1000, 2500, 50, 15.0, np.zeros(8)))
    ident = complex_int8_voltages(3, 6000, 8, 20.0,
                                  PulseTrain(1000, 2500, 50, 15.0, np.zeros(8),
                                             response=lambda L: np.ones((8, L)), window=256),
                                  chunk_rows=777)
    assert np.array_equal(plain, ident)


def test_delay_response_moves_the_pulse():
    d = 7
    delay = lambda L: np.exp(-2j * np.pi * np.fft.fftfreq(L)[None, :] * d).repeat(4, 0)
    a = complex_int8_voltages(0, 4000, 4, 0.0, PulseTrain(500, 3000, 40, 30.0, np.zeros(4)))
    b = complex_int8_voltages(0, 4000, 4, 0.0, PulseTrain(500, 3000, 40, 30.0, np.zeros(4),
                                                          response=delay, window=256))
    assert np.array_equal(np.roll(a, d, axis=0), b)


def test_dedispersion_recovers_a_dispersed_pulse():
    """16 channels of 62.5 kHz at 317 MHz, DM 40 (a smear of about 50
    samples), one pulse of 62 samples, no noise: after dispersion inside each
    channel the pulse is smeared; after the oracle's dedispersion (N 256,
    before integration) at least 99.9% of each channel's power is back inside
    the pulse's samples."""
    args = (325.0 - 8.0 + 0.5, 1.0, 16, 40.0, 256, 1)
    geo = O.plan_geometry(*args)
    t0, W = 3000, 62
    pulses = PulseTrain(t0, 1e9, W, 40.0, np.zeros(16), response=dispersing_response(geo, 40.0),
                        window=512)
    vin = complex_int8_voltages(5, 10 * geo.hop * 8, 16, 0.0, pulses)
    raw = vin[..., 0].astype(float) ** 2 + vin[..., 1].astype(float) ** 2
    spread = 1 - raw[t0:t0 + W].sum(0) / raw.sum(0)
    assert np.all(spread > 0.2)                   # really smeared by the dispersion
    _, v = O.dedisperse(vin, geo, return_voltages=True)
    p = np.abs(v) ** 2                            # [C][T]
    inside = p[:, t0:t0 + W].sum(1) / p.sum(1)
    assert np.all(inside > 0.98), inside.min()
    assert np.all(1 - inside < spread / 10)
