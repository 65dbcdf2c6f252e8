"""Full-band mode (the paper's own design) on the GPU against the FP64 oracle:
inverse channelisation, one long transform over the band, chirp, overlap-save,
squaring and integration.  Relative RMS <= 1e-5 on the intensity series."""
import numpy as np
import pytest

import oracle as O
from synth import complex_int8_voltages

pytestmark = pytest.mark.gpu
TOL = 1e-5


def run_fullband(vin, args, q, n_blocks):
    import torch
    from paper_1509_00186_b300.cdd import Fullband
    with Fullband(*args, segments_per_block=q) as f:
        fr = f.frames
        x = torch.from_numpy(np.ascontiguousarray(vin[: fr * n_blocks])).cuda()
        outs = [f.execute(x[b * fr:(b + 1) * fr]) for b in range(n_blocks)]
        torch.cuda.synchronize()
        return torch.cat(outs).cpu().numpy()


@pytest.mark.parametrize("args", [
    (610.0, 1.0, 32, 20.0, 0, 4),            # N = 2^14: the shared-memory transform only
    (325.0, 2.0, 64, 5.0, 1 << 20, 8),       # N = 2^20: 8192-point middle, one radix-128 tile pass, lanes sum 8
    (325.0, 2.0, 64, 5.0, 1 << 20, 1),       # N = 2^20: radix 128, n_avg 1
    (325.0, 2.0, 64, 5.0, 1 << 20, 32),      # N = 2^20: radix 128, 32-sample windows over two lane groups
    (325.0, 2.0, 64, 5.0, 1 << 20, 64),      # N = 2^20: radix 128, n_avg 64 > 32 keeps the integration kernel
    (325.0, 2.0, 64, 5.0, 1 << 15, 8),       # N = 2^15: one radix-2 outer pass, integration kernel
    (325.0, 2.0, 64, 5.0, 1 << 18, 1),       # N = 2^18: one radix-16 pass, integrated across lanes (n_avg 1)
    (325.0, 4.0, 128, 40.0, 0, 16),          # N = 2^20: radix 128, 16-sample windows across lanes
    (325.0, 8.0, 256, 30.0, 0, 32),          # N = 2^21: radix 64 then 4, 32-sample windows across lanes
    (325.0, 2.0, 64, 5.0, 1 << 21, 64),      # N = 2^21: radix 64, n_avg 64 > 32 keeps the integration kernel
    (325.0, 2.0, 64, 5.0, 1 << 24, 4),       # N = 2^24: radix 128 then 16
    pytest.param((325.0, 2.0, 64, 5.0, 1 << 25, 16), marks=pytest.mark.slow),   # N = 2^25: radix 64 then 64
    (610.0, -1.0, 32, 20.0, 0, 4),           # lower sideband, the shared-memory transform only
    (325.0, -2.0, 64, 5.0, 1 << 18, 1),      # lower sideband through the outer passes
    (325.0, -2.0, 64, 5.0, 1 << 20, 2),      # lower sideband through a radix-128 pass
    (610.0, 1.0, 32, 0.0, 1 << 14, 4),       # DM 0: no overlap, the correction is 1
    (325.0, 2.0, 64, 0.0, 1 << 18, 1),       # DM 0 through the outer passes
])
def test_fullband_matches_oracle(cuda_device, args):
    g = O.fullband_geometry(*args)
    frames_per_seg = g.hop // g.frame
    vin = complex_int8_voltages(11, frames_per_seg * 4, args[2], 20.0)
    want = O.dedisperse_fullband(vin, g)
    got = run_fullband(vin, args, 2, 2)
    assert got.shape == want.shape
    assert O.rel_rms(got, want) <= TOL


def test_fullband_block_split_is_bit_identical(cuda_device):
    args = (610.0, 1.0, 32, 20.0, 0, 4)
    g = O.fullband_geometry(*args)
    vin = complex_int8_voltages(12, g.hop // g.frame * 6, 32, 20.0)
    a = run_fullband(vin, args, 6, 1)
    b = run_fullband(vin, args, 2, 3)
    c = run_fullband(vin, args, 1, 6)
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.slow
def test_fullband_gsb_32mhz_mode(cuda_device):
    """The paper's 32 MHz mode at 325 MHz with DM 50: N = 2^26 over the whole
    band (a radix-64 and a radix-128 pass through HBM each way around
    8192-point sub-transforms); two segments against the oracle."""
    args = (325.0, 32.0, 512, 50.0, 0, 16)
    g = O.fullband_geometry(*args)
    assert g.n_fft == 2 ** 26
    vin = complex_int8_voltages(13, g.hop // g.frame * 2, 512, 20.0)
    want = O.dedisperse_fullband(vin, g)
    got = run_fullband(vin, args, 1, 2)
    assert O.rel_rms(got, want) <= TOL


@pytest.mark.slow
def test_fullband_largest_transform(cuda_device):
    """N = 2^27, the largest transform the full-band mode takes: two radix-128
    tile passes each way around 8192-point sub-transforms; one segment against
    the oracle."""
    args = (325.0, 2.0, 64, 5.0, 1 << 27, 16)
    g = O.fullband_geometry(*args)
    assert g.n_fft == 2 ** 27
    vin = complex_int8_voltages(14, g.hop // g.frame, 64, 20.0)
    want = O.dedisperse_fullband(vin, g)
    got = run_fullband(vin, args, 1, 1)
    assert got.shape == want.shape
    assert O.rel_rms(got, want) <= TOL
