"""Tensor-core (tcgen05) forms of the N = 8192 fused kernel against the FP64
oracle, through the C ABI (CDD_ATTR_PRECISION).

Tolerances, relative RMS per output array (voltages and intensities):
- FP16X2 (hi + lo FP16 operands, three products per pass): 1e-5, the bound
  stated for the split-precision form (its rounding model gives about 1e-6);
- BF16X2: 2e-5 (16 significant bits per operand: about 2^-17 per rounding
  over five rounded operand stages gives 1e-5 to 2e-5);
- FP16 alone: 2e-3, the bound stated for plain FP16 (11 bits: about 6e-4);
- BF16 alone: 1.5e-2 (8 bits: about 5e-3).
Every form must also report no device error (no wait gave up).
"""
import numpy as np
import pytest

import oracle as O
from synth import WORKLOADS, PulseTrain, complex_int8_voltages

pytestmark = pytest.mark.gpu
TOL = {"fp16x2": 1e-5, "bf16x2": 2e-5, "fp16": 2e-3, "bf16": 1.5e-2}


def rel_rms_rows(a, b):
    return np.array([O.rel_rms(a[i], b[i]) for i in range(a.shape[0])])


def gpu_run(vin, args, q, n_blocks, precision, taper="none", volt=True):
    import torch
    from paper_1509_00186_b300.cdd import Plan
    with Plan(*args, segments_per_block=q, taper=taper, precision=precision) as plan:
        assert plan.get("precision") != 0
        bs, n_out, C = plan.block_samples, plan.n_out, plan.n_chan
        x = torch.from_numpy(np.ascontiguousarray(vin[: bs * n_blocks])).cuda()
        outs, volts = [], []
        for b in range(n_blocks):
            o = torch.empty((C, n_out), dtype=torch.float32, device="cuda")
            v = torch.empty((C, bs, 2), dtype=torch.float32, device="cuda") if volt else None
            plan.execute(x[b * bs:(b + 1) * bs], o, v)
            outs.append(o)
            if volt:
                volts.append(v)
        torch.cuda.synchronize()
        assert plan.get("device_errors") == 0
        out = torch.cat(outs, 1).cpu().numpy()
        if volt:
            vv = torch.cat(volts, 1).cpu().numpy()
            return out, vv[..., 0] + 1j * vv[..., 1]
        return out, None


def oracle_run(vin, args, n_samples, taper="none", channels=None):
    geo = O.plan_geometry(*args)
    return O.dedisperse(vin[:n_samples], geo, taper, return_voltages=True, channels=channels)


@pytest.mark.parametrize("precision", ["fp16x2", "bf16x2", "fp16", "bf16"])
def test_forms_match_oracle(cuda_device, precision):
    """16 channels of 62.5 kHz at 309.5 MHz, DM 50, x16, two blocks of four
    segments: the shape of the benchmark block, cut down."""
    args = (309.5, 1.0, 16, 50.0, 8192, 16)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(31, 8 * geo.hop, 16, 20.0)
    out_o, v_o = oracle_run(vin, args, 8 * geo.hop)
    out_g, v_g = gpu_run(vin, args, 4, 2, precision)
    tol = TOL[precision]
    assert np.all(rel_rms_rows(v_g, v_o) <= tol), rel_rms_rows(v_g, v_o).max()
    assert np.all(rel_rms_rows(out_g, out_o) <= tol), rel_rms_rows(out_g, out_o).max()


def test_fp16x2_is_far_closer_than_fp16(cuda_device):
    """The split form recovers the precision the single rounding loses."""
    args = (309.5, 1.0, 8, 50.0, 8192, 16)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(32, 3 * geo.hop, 8, 20.0)
    out_o, _ = oracle_run(vin, args, 3 * geo.hop)
    e2 = O.rel_rms(gpu_run(vin, args, 3, 1, "fp16x2", volt=False)[0], out_o)
    e1 = O.rel_rms(gpu_run(vin, args, 3, 1, "fp16", volt=False)[0], out_o)
    assert e2 * 20 < e1


@pytest.mark.parametrize("n_avg", [1, 32, 64, 256])
def test_fp16x2_integration_lengths(cuda_device, n_avg):
    """n_avg 1 and 32 integrate across lanes, 64 and 256 through the operand
    region in shared memory; two blocks split or whole are bit-identical."""
    args = (313.0, 2.0, 32, 50.0, 8192, n_avg)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(25, 6 * geo.hop, 32, 20.0)
    out_o, _ = oracle_run(vin, args, 6 * geo.hop)
    whole, _ = gpu_run(vin, args, 6, 1, "fp16x2", volt=False)
    split, _ = gpu_run(vin, args, 3, 2, "fp16x2", volt=False)
    assert np.array_equal(split, whole)
    assert np.all(rel_rms_rows(whole, out_o) <= TOL["fp16x2"])


@pytest.mark.parametrize("taper", ["hann", "welch"])
def test_fp16x2_lower_sideband_and_tapers(cuda_device, taper):
    args = (330.0, -1.0, 16, 50.0, 8192, 16)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(33, 4 * geo.hop, 16, 20.0)
    out_o, v_o = oracle_run(vin, args, 4 * geo.hop, taper=taper)
    out_g, v_g = gpu_run(vin, args, 2, 2, "fp16x2", taper=taper)
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL["fp16x2"])
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL["fp16x2"])


def test_fp16x2_dm_zero_and_ragged_work(cuda_device):
    """DM 0 (no overlap: every segment starts on a block row) on 5 channels x
    3 segments: an odd number of work items over the two pipelines of a CTA."""
    args = (325.0, 0.3125, 5, 0.0, 8192, 4)
    geo = O.plan_geometry(*args)
    assert geo.n_ov == 0
    vin = complex_int8_voltages(34, 6 * geo.hop, 5, 20.0)
    vin[5, 0] = (-128, 127)
    out_o, v_o = oracle_run(vin, args, 6 * geo.hop)
    out_g, v_g = gpu_run(vin, args, 3, 2, "fp16x2")
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL["fp16x2"])
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL["fp16x2"])


def test_fp16x2_single_channel_single_segment(cuda_device):
    args = (325.0, 0.0625, 1, 30.0, 8192, 16)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(35, 2 * geo.hop, 1, 20.0)
    out_o, v_o = oracle_run(vin, args, 2 * geo.hop)
    out_g, v_g = gpu_run(vin, args, 1, 2, "fp16x2")
    assert O.rel_rms(v_g, v_o) <= TOL["fp16x2"] and O.rel_rms(out_g, out_o) <= TOL["fp16x2"]


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp16x2", "fp16"])
def test_gsb_full_size_sampled_channels(cuda_device, precision):
    """The 32 MHz / 512-channel / DM 50 / N 8192 block at its full 10 s size in
    the benchmark's launch configuration (76 segments, one block), sampled
    channels recomputed by the oracle one by one."""
    w = WORKLOADS["gsb"]
    args = (w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    geo = O.plan_geometry(*args)
    offs = O.dispersion_delay_s(geo.f_lo_mhz, geo.f_lo_mhz[0], w.dm) * w.chan_bw_mhz * 1e6
    pulses = PulseTrain(3000.0, w.period_samples, w.width_samples, w.pulse_sigma, offs)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)
    q = w.n_samp // geo.hop
    out_g, _ = gpu_run(vin, args, q, 1, precision, volt=False)
    chans = [0, 1, 255, 256, 510, 511]
    out_o, _ = oracle_run(vin, args, q * geo.hop, channels=chans)
    assert np.all(rel_rms_rows(out_g[chans], out_o) <= TOL[precision])
    assert np.all(np.isfinite(out_g))
