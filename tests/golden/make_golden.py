"""Writes tests/golden/tiny_oracle_digest.json from the FP64 oracle alone.

The digest freezes the oracle's output on the seeded 16 MHz / 256-channel input
so that any later change to the oracle's arithmetic shows up as a test failure.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from synth import WORKLOADS, PulseTrain, complex_int8_voltages  # noqa: E402

CHANNELS = [0, 1, 77, 128, 255]


def tiny_input():
    w = WORKLOADS["tiny"]
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    offs = O.dispersion_delay_s(geo.f_lo_mhz, geo.f_lo_mhz[0], w.dm) * w.chan_bw_mhz * 1e6
    pulses = PulseTrain(start=4000.0, period=w.period_samples, width=w.width_samples,
                        sigma=w.pulse_sigma, offsets=offs)
    return geo, complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)


def digest():
    geo, vin = tiny_input()
    out = O.dedisperse(vin, geo, channels=CHANNELS)
    return {
        "cite": "oracle output on the seeded tiny workload (Sec. 2.2 overlap-save, Sec. 3.1 "
                "detect/integrate, Sec. 1.2 alignment); written by tests/golden/make_golden.py",
        "channels": CHANNELS,
        "n_out": int(out.shape[1]),
        "input_sum": int(vin.astype(np.int64).sum()),
        "input_sq_sum": int((vin.astype(np.int64) ** 2).sum()),
        "row_sums": [float(s) for s in out.sum(axis=1)],
        "row_max": [float(s) for s in out.max(axis=1)],
        "argmax": [int(i) for i in out.argmax(axis=1)],
        "samples": {str(k): [float(v) for v in out[i, 1000:1008]] for i, k in enumerate(CHANNELS)},
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "tiny_oracle_digest.json"), "w") as fh:
        json.dump(digest(), fh, indent=1)
    print("wrote", os.path.join(HERE, "tiny_oracle_digest.json"))
