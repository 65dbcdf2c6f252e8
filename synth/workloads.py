"""Named synthetic workloads shaped like GMRT GSB / upgraded-GMRT voltage data.

Each entry states the observation (centre frequency, bandwidth, channels, DM),
the record length, the transform length and the integration, and how the pulse
train is drawn.  The numbers are inputs, not arithmetic of the method: the
pulse's per-channel arrival offsets are supplied by whoever builds the input.
"""

from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    f_center_mhz: float
    bandwidth_mhz: float
    n_chan: int
    dm: float
    seconds: float
    n_fft: int
    n_avg: int
    sigma: float = 20.0
    pulse_period_s: float = 0.25
    pulse_width_s: float = 1e-3
    pulse_snr: float = 50.0
    seed: int = 1

    @property
    def chan_bw_mhz(self) -> float:
        return self.bandwidth_mhz / self.n_chan

    @property
    def n_samp(self) -> int:
        """Complex samples per channel in the record (sample time 1/chan_bw)."""
        return int(round(self.seconds * self.chan_bw_mhz * 1e6))

    @property
    def width_samples(self) -> int:
        return max(1, int(round(self.pulse_width_s * self.chan_bw_mhz * 1e6)))

    @property
    def period_samples(self) -> float:
        return self.pulse_period_s * self.chan_bw_mhz * 1e6

    @property
    def pulse_sigma(self) -> float:
        """Per-component pulse amplitude that gives ``pulse_snr`` on the band-summed,
        aligned, width-integrated intensity: SNR = (sp^2 / s^2) * sqrt(C * W)."""
        return self.sigma * math.sqrt(self.pulse_snr / math.sqrt(self.n_chan * self.width_samples))


WORKLOADS = {
    # 16 MHz at 325 MHz, 256 x 62.5 kHz channels, DM 10, 0.5 s; N = 64 (>= 4x the
    # smear), integration x4; pulses every 0.25 s, 1 ms wide, SNR 50.
    "tiny": Workload("tiny", 325.0, 16.0, 256, 10.0, 0.5, 64, 4),
    # GSB real-time shape: 32 MHz at 325 MHz, 512 x 62.5 kHz, DM 50, 10 s,
    # N = 8192, x16; pulse train with period 33 ms and 3% duty cycle.
    "gsb": Workload("gsb", 325.0, 32.0, 512, 50.0, 10.0, 8192, 16,
                    pulse_period_s=33e-3, pulse_width_s=0.03 * 33e-3),
    # long-chirp shape: 32 MHz at 150 MHz, 512 channels, DM 100, N = 65536, x16.
    "precision": Workload("precision", 150.0, 32.0, 512, 100.0, 10.0, 65536, 16,
                          pulse_period_s=0.5, pulse_width_s=1e-3),
}
