"""GPU path (libcdd.so through its C ABI) against the FP64 oracle.

Tolerance: relative RMS error <= 1e-5 per output array (dedispersed voltages
and aligned intensities), the bound stated for the FP32 form.  The FP32 path's
expected error is ~1e-6 (log2(N) radix stages of float rounding on an
exactly represented int8 input, a chirp rounded once from FP64), so 1e-5
leaves an order of magnitude of margin while still catching any wrong bin,
sign, twiddle or index (those give errors of order 1).
Integer decisions (geometry, shifts) are compared exactly on the CPU side.
"""
import numpy as np
import pytest

import oracle as O
from synth import WORKLOADS, PulseTrain, complex_int8_voltages

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_rms_rows(a, b):
    return np.array([O.rel_rms(a[i], b[i]) for i in range(a.shape[0])])


def gpu_run(vin, geo_args, q, n_blocks, taper="none", volt=True, pinned_host=False):
    import torch
    from paper_1509_00186_b300.cdd import Plan
    plan = Plan(*geo_args, segments_per_block=q, taper=taper)
    try:
        bs, n_out, C = plan.block_samples, plan.n_out, plan.n_chan
        outs, volts = [], []
        if pinned_host:
            x = torch.from_numpy(np.ascontiguousarray(vin[: bs * n_blocks])).pin_memory()
            for b in range(n_blocks):
                o = torch.empty((C, n_out), dtype=torch.float32).pin_memory()
                plan.execute_host(x[b * bs:(b + 1) * bs], o)
                outs.append(o.clone())
            return torch.cat(outs, 1).numpy(), None
        x = torch.from_numpy(np.ascontiguousarray(vin[: bs * n_blocks])).cuda()
        for b in range(n_blocks):
            o = torch.empty((C, n_out), dtype=torch.float32, device="cuda")
            v = torch.empty((C, bs, 2), dtype=torch.float32, device="cuda") if volt else None
            plan.execute(x[b * bs:(b + 1) * bs], o, v)
            outs.append(o)
            if volt:
                volts.append(v)
        torch.cuda.synchronize()
        out = torch.cat(outs, 1).cpu().numpy()
        if volt:
            vv = torch.cat(volts, 1).cpu().numpy()
            return out, vv[..., 0] + 1j * vv[..., 1]
        return out, None
    finally:
        plan.close()


def oracle_run(vin, geo_args, n_samples, taper="none", channels=None):
    geo = O.plan_geometry(*geo_args)
    return O.dedisperse(vin[:n_samples], geo, taper, return_voltages=True, channels=channels)


def tiny_input():
    w = WORKLOADS["tiny"]
    geo = O.plan_geometry(w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    offs = O.dispersion_delay_s(geo.f_lo_mhz, geo.f_lo_mhz[0], w.dm) * w.chan_bw_mhz * 1e6
    pulses = PulseTrain(4000.0, w.period_samples, w.width_samples, w.pulse_sigma, offs)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)
    args = (w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    return vin, args, geo


@pytest.fixture(scope="module")
def tiny(cuda_device):
    vin, args, geo = tiny_input()
    q = vin.shape[0] // geo.hop                   # 600 segments, 31200 samples
    out_o, v_o = oracle_run(vin, args, q * geo.hop)
    return vin, args, geo, q, out_o, v_o


def test_tiny_whole_record_matches_oracle(tiny):
    vin, args, geo, q, out_o, v_o = tiny
    out_g, v_g = gpu_run(vin, args, q, 1)
    assert out_g.shape == out_o.shape == (256, q * geo.hop // geo.n_avg)
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL)
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL)
    assert O.rel_rms(out_g, out_o) <= TOL
    # the delayed channels start with exactly r_k zeros (no earlier data)
    for k in (1, 100, 255):
        r = int(geo.shift[k])
        assert np.all(out_g[k, :r] == 0.0) and out_g[k, r] > 0


def test_block_split_is_bit_identical(tiny):
    """Any split of the stream into blocks gives the same bits: the overlap tail
    and the alignment ring carry the state between calls."""
    vin, args, geo, q, out_o, _ = tiny
    whole, _ = gpu_run(vin, args, q, 1, volt=False)
    for qb in (100, 24, 1):
        split, _ = gpu_run(vin, args, qb, q // qb, volt=False)
        assert np.array_equal(split, whole), qb


def test_short_blocks_against_oracle(tiny):
    """Blocks much shorter than the largest alignment shift (r_max = 603 outputs,
    13 outputs per segment): every output goes through the ring."""
    vin, args, geo, q, out_o, _ = tiny
    out_g, _ = gpu_run(vin, args, 5, q // 5, volt=False)
    assert O.rel_rms(out_g, out_o) <= TOL


def test_host_buffer_path_equals_device_path(tiny):
    vin, args, geo, q, out_o, _ = tiny
    dev, _ = gpu_run(vin, args, 120, 5, volt=False)
    host, _ = gpu_run(vin, args, 120, 5, volt=False, pinned_host=True)
    assert np.array_equal(host, dev)
    assert O.rel_rms(host, out_o) <= TOL


def test_stage_timing_changes_no_bits(tiny):
    """Events around the two stages are recorded on the launching stream; the
    output is the same bits with and without them, and every block is timed."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    vin, args, geo, q, _, _ = tiny
    plain, _ = gpu_run(vin, args, 100, 3, volt=False)
    plan = Plan(*args, segments_per_block=100, stage_timing=True)
    try:
        bs = plan.block_samples
        x = torch.from_numpy(np.ascontiguousarray(vin[: 3 * bs])).cuda()
        outs = [plan.execute(x[b * bs:(b + 1) * bs]) for b in range(3)]
        timed = torch.cat(outs, 1).cpu().numpy()
        assert plan.get("timed_blocks") == 3
        ct, ols = plan.get("corner_turn_ns"), plan.get("ols_ns")
        assert 0 < ct < 1e9 and 0 < ols < 1e9
    finally:
        plan.close()
    assert np.array_equal(timed, plain)


@pytest.mark.parametrize("logn", list(range(6, 17)))
def test_every_fft_length(cuda_device, logn):
    """Each supported N on a ragged channel count (the last CTA is partly idle
    for small N), two blocks of three segments, overlap ~ N/8."""
    n = 1 << logn
    n_chan, n_avg = 5, 4
    chan_bw = 0.0625
    dm = (n / 8) / O.dispersion_samples(317.0, chan_bw, 1.0)
    args = (317.0 + n_chan * chan_bw / 2, n_chan * chan_bw, n_chan, dm, n, n_avg)
    geo = O.plan_geometry(*args)
    assert 0 < geo.n_ov < n
    rng = np.random.default_rng(logn)
    T = 6 * geo.hop
    vin = np.clip(np.rint(rng.normal(0, 20, (T, n_chan, 2))), -127, 127).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, T)
    out_g, v_g = gpu_run(vin, args, 3, 2)
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL)
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL)


@pytest.mark.parametrize("logn,taper", [(6, "none"), (10, "hann"), (13, "none"), (16, "none")])
def test_lower_sideband(cuda_device, logn, taper):
    """A lower-sideband band (negative bandwidth): channel 0 highest, bins
    mirrored, conjugate correction; checked against the oracle."""
    n = 1 << logn
    n_chan, n_avg, chan_bw = 6, 4, 0.0625
    dm = (n / 8) / O.dispersion_samples(317.0, chan_bw, 1.0)
    args = (317.0 + n_chan * chan_bw / 2, -n_chan * chan_bw, n_chan, dm, n, n_avg)
    geo = O.plan_geometry(*args)
    assert geo.sideband == -1 and geo.shift[0] == geo.shift.max()
    rng = np.random.default_rng(100 + logn)
    T = 4 * geo.hop
    vin = np.clip(np.rint(rng.normal(0, 20, (T, n_chan, 2))), -127, 127).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, T, taper=taper)
    out_g, v_g = gpu_run(vin, args, 2, 2, taper=taper)
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL)
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL)


@pytest.mark.parametrize("taper", ["hann", "welch"])
def test_tapers(cuda_device, taper):
    args = (317.0 + 1.0, 2.0, 32, 10.0, 256, 4)
    geo = O.plan_geometry(*args)
    rng = np.random.default_rng(7)
    T = 10 * geo.hop
    vin = np.clip(np.rint(rng.normal(0, 20, (T, 32, 2))), -127, 127).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, T, taper=taper)
    out_g, v_g = gpu_run(vin, args, 5, 2, taper=taper)
    assert O.rel_rms(v_g, v_o) <= TOL
    assert O.rel_rms(out_g, out_o) <= TOL


def test_dm_zero_no_overlap(cuda_device):
    args = (325.0, 16.0, 16, 0.0, 64, 4)
    rng = np.random.default_rng(9)
    vin = rng.integers(-128, 128, size=(64 * 12, 16, 2)).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, 64 * 12)
    out_g, v_g = gpu_run(vin, args, 4, 3)
    assert O.rel_rms(v_g, v_o) <= TOL
    assert O.rel_rms(out_g, out_o) <= TOL
    # extreme int8 values (-128 included) survive the unpack
    assert np.max(np.abs(v_g.real - vin[:, :, 0].T)) < 1e-3


def test_single_channel_single_segment(cuda_device):
    args = (325.0, 0.0625, 1, 10.0, 64, 4)
    geo = O.plan_geometry(*args)
    rng = np.random.default_rng(10)
    vin = np.clip(np.rint(rng.normal(0, 20, (geo.hop * 3, 1, 2))), -127, 127).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, geo.hop * 3)
    out_g, v_g = gpu_run(vin, args, 1, 3)
    assert O.rel_rms(v_g, v_o) <= TOL and O.rel_rms(out_g, out_o) <= TOL


@pytest.mark.slow
def test_gsb_full_size_sampled_channels(cuda_device):
    """The 32 MHz / 512-channel / DM 50 / N 8192 shape at its full 10 s size, in
    the benchmark's launch configuration (one block of 76 segments); the oracle
    recomputes a sample of channels one by one."""
    w = WORKLOADS["gsb"]
    args = (w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    geo = O.plan_geometry(*args)
    offs = O.dispersion_delay_s(geo.f_lo_mhz, geo.f_lo_mhz[0], w.dm) * w.chan_bw_mhz * 1e6
    pulses = PulseTrain(3000.0, w.period_samples, w.width_samples, w.pulse_sigma, offs)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma, pulses)
    q = w.n_samp // geo.hop
    assert q == 76
    out_g, _ = gpu_run(vin, args, q, 1, volt=False)
    chans = [0, 1, 255, 256, 510, 511]
    out_o, _ = oracle_run(vin, args, q * geo.hop, channels=chans)
    assert np.all(rel_rms_rows(out_g[chans], out_o) <= TOL)
    assert np.all(np.isfinite(out_g))
    # every channel, not only the sampled ones, carries the noise power:
    # mean intensity ~ n_avg * 2 * sigma^2 after the r_k leading zeros
    means = np.array([out_g[k, geo.shift[k]:].mean() for k in range(w.n_chan)])
    assert np.all(np.abs(means / (w.n_avg * 2 * w.sigma ** 2) - 1) < 0.1)


@pytest.mark.slow
def test_precision_shape_full_size_sampled_channels(cuda_device):
    """The 32 MHz / 512-channel band at 150 MHz, DM 100, N 65536 (a cluster of
    eight CTAs per segment) at its full 10 s size, one block of 9 segments;
    sampled channels against the oracle."""
    w = WORKLOADS["precision"]
    args = (w.f_center_mhz, w.bandwidth_mhz, w.n_chan, w.dm, w.n_fft, w.n_avg)
    geo = O.plan_geometry(*args)
    assert (geo.n_ov, geo.hop) == (1360, 64176)
    vin = complex_int8_voltages(w.seed, w.n_samp, w.n_chan, w.sigma)
    q = w.n_samp // geo.hop
    out_g, _ = gpu_run(vin, args, q, 1, volt=False)
    chans = [0, 7, 300, 511]
    out_o, _ = oracle_run(vin, args, q * geo.hop, channels=chans)
    assert np.all(rel_rms_rows(out_g[chans], out_o) <= TOL)
    assert np.all(np.isfinite(out_g))


def test_two_polarisations_summed_after_detection(cuda_device):
    import torch
    from paper_1509_00186_b300.cdd import Plan
    args = (318.0, 2.0, 32, 10.0, 64, 4)
    geo = O.plan_geometry(*args)
    rng = np.random.default_rng(41)
    q, blocks = 30, 3
    T = q * geo.hop * blocks
    a = np.clip(np.rint(rng.normal(0, 20, (T, 32, 2))), -127, 127).astype(np.int8)
    b = np.clip(np.rint(rng.normal(0, 15, (T, 32, 2))), -127, 127).astype(np.int8)
    want = O.dedisperse_dual(a, b, geo)
    with Plan(*args, segments_per_block=q, polarisations=2) as p:
        bs = p.block_samples
        xa, xb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        zero = torch.zeros_like(xb[:bs])
        got = torch.cat([p.execute_dual(xa[i * bs:(i + 1) * bs], xb[i * bs:(i + 1) * bs])
                         for i in range(blocks)], 1).cpu().numpy()
    assert O.rel_rms(got, want) <= TOL
    # a silent second polarisation leaves the first one's result bit for bit
    with Plan(*args, segments_per_block=q, polarisations=2) as p2, Plan(*args, segments_per_block=q) as p1:
        only = p2.execute_dual(xa[:bs], zero).cpu().numpy()
        single = p1.execute(xa[:bs]).cpu().numpy()
    assert np.array_equal(only, single)


def test_band_sum_of_plan_and_batch_outputs(cuda_device):
    import torch
    from paper_1509_00186_b300.cdd import Batch, band_sum
    vin, args, geo = tiny_input()
    q = vin.shape[0] // geo.hop
    out_g, _ = gpu_run(vin, args, q, 1, volt=False)
    want = O.band_sum(O.dedisperse(vin[: q * geo.hop], geo))
    got = band_sum(torch.from_numpy(out_g).cuda()).cpu().numpy()
    assert O.rel_rms(got, want) <= TOL
    # DM-trial time series of a small batch: one band sum per DM plane
    bargs = (650.0, 6.25, 64, [5.0, 20.0], (2048, 1024, 512, 256), 4)
    g = O.batch_geometry(*bargs)
    x = complex_int8_voltages(5, 1984 * 2, 64, 20.0)
    with Batch(*bargs, segments_per_block=2) as b:
        series = band_sum(b.execute(torch.from_numpy(x).cuda())).cpu().numpy()
    assert series.shape == (2, 1984 * 2 // 4)
    assert O.rel_rms(series, O.band_sum(O.dedisperse_batch(x, g))) <= TOL


def test_band_sum_ragged_and_misaligned(cuda_device):
    """The scalar form of the band sum (n_out not a multiple of 4, or a buffer
    that is not 16-byte aligned) and the vector form agree with a float64 sum."""
    import torch
    from paper_1509_00186_b300.cdd import band_sum
    rng = np.random.default_rng(3)
    for planes, C, n in ((3, 37, 1001), (2, 512, 4096), (1, 1, 5)):
        a = rng.random((planes, C, n)).astype(np.float32)
        got = band_sum(torch.from_numpy(a).cuda()).cpu().numpy()
        assert O.rel_rms(got, O.band_sum(a.astype(np.float64))) <= 1e-6
        raw = torch.empty(a.size + 1, dtype=torch.float32, device="cuda")
        shifted = raw[1:].view(planes, C, n)                  # 4 bytes past a 16-byte boundary
        shifted.copy_(torch.from_numpy(a))
        got2 = band_sum(shifted).cpu().numpy()
        assert np.array_equal(got2, got) or O.rel_rms(got2, got) <= 1e-6


def test_unaligned_input_pointer(cuda_device):
    """A caller's block that does not start on a 16-byte boundary (here 2
    bytes past one) takes the corner turn's element-wise path and gives the
    same bits as an aligned copy."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    args = (313.0, 8.0, 128, 50.0, 8192, 16)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(22, 4 * geo.hop, 128, 20.0)
    with Plan(*args, segments_per_block=4) as p:
        a = p.execute(torch.from_numpy(vin).cuda()).cpu().numpy()
    raw = torch.empty(vin.size + 2, dtype=torch.int8, device="cuda")
    shifted = raw[2:].view(vin.shape)
    assert shifted.data_ptr() % 16 == 2
    shifted.copy_(torch.from_numpy(vin))
    with Plan(*args, segments_per_block=4) as p:
        b = p.execute(shifted).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["tiny", "n8192", "dual"])
def test_checkpoint_resume_is_bit_identical(cuda_device, case):
    """Export a stream's state after three blocks, import it into a fresh plan of
    the same geometry: the next blocks come out bit for bit as from the
    original plan (overlap tail, alignment ring window and stream position)."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    if case == "tiny":
        vin, args, geo = tiny_input()
        q, pols = 24, 1                           # blocks far shorter than r_max: the ring matters
    else:
        args = (313.0, 8.0, 128, 50.0, 8192, 16)
        geo = O.plan_geometry(*args)
        q, pols = 3, 2 if case == "dual" else 1
        vin = complex_int8_voltages(23, 5 * q * geo.hop, 128, 20.0)
    vin_b = complex_int8_voltages(24, vin.shape[0], args[2], 20.0)
    bs = q * geo.hop
    xa = torch.from_numpy(np.ascontiguousarray(vin[: 5 * bs])).cuda()
    xb = torch.from_numpy(np.ascontiguousarray(vin_b[: 5 * bs])).cuda()

    def run(plan, b):
        blk = slice(b * bs, (b + 1) * bs)
        if pols == 2:
            return plan.execute_dual(xa[blk], xb[blk]).cpu().numpy()
        return plan.execute(xa[blk]).cpu().numpy()

    with Plan(*args, segments_per_block=q, polarisations=pols) as a:
        for b in range(3):                        # tiny: the ring window wraps after 3 blocks
            run(a, b)
        state = a.export_state()
        want = [run(a, b) for b in (3, 4)]
    with Plan(*args, segments_per_block=q, polarisations=pols) as c:
        c.import_state(state)
        got = [run(c, b) for b in (3, 4)]
        assert c.get("blocks_done") == 5
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("logn", [8, 13, 16])
def test_overlap_longer_than_the_hop(cuda_device, logn):
    """Overlap 0.7 N: each segment discards more samples than it keeps, and the
    first segments of a block reach back into the previous block's tail.
    N = 256 (ols_kernel), 8192 (persistent) and 65536 (clusters); each block
    spans enough segments to outlast the largest shift."""
    n = 1 << logn
    n_chan, n_avg = 3, 4
    chan_bw = 0.0625
    dm = (0.7 * n) / O.dispersion_samples(317.0, chan_bw, 1.0)
    args = (317.0 + n_chan * chan_bw / 2, n_chan * chan_bw, n_chan, dm, n, n_avg)
    geo = O.plan_geometry(*args)
    assert geo.n_ov > geo.hop
    q = max(3, -(-int(geo.shift.max()) * n_avg // geo.hop))
    rng = np.random.default_rng(100 + logn)
    T = 2 * q * geo.hop
    vin = np.clip(np.rint(rng.normal(0, 20, (T, n_chan, 2))), -127, 127).astype(np.int8)
    out_o, v_o = oracle_run(vin, args, T)
    out_g, v_g = gpu_run(vin, args, q, 2)
    assert np.all(rel_rms_rows(v_g, v_o) <= TOL)
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL)


def test_cluster_window_at_the_limit(cuda_device):
    """N = 65536 runs on clusters of eight 8192-point CTAs, each holding
    1024-sample runs of the segment: n_avg = 1024 (integration through shared
    memory, windows as long as a run) still matches the oracle."""
    n, n_chan, n_avg = 65536, 3, 1024
    chan_bw = 0.0625
    dm = (n / 8) / O.dispersion_samples(317.0, chan_bw, 1.0)
    args = (317.0 + n_chan * chan_bw / 2, n_chan * chan_bw, n_chan, dm, n, n_avg)
    geo = O.plan_geometry(*args)
    rng = np.random.default_rng(5)
    T = 4 * geo.hop
    vin = np.clip(np.rint(rng.normal(0, 20, (T, n_chan, 2))), -127, 127).astype(np.int8)
    out_o, _ = oracle_run(vin, args, T)
    out_g, _ = gpu_run(vin, args, 2, 2, volt=False)
    assert np.all(rel_rms_rows(out_g, out_o) <= TOL)


@pytest.mark.parametrize("n_avg", [1, 32, 64, 256])
def test_integration_lengths_n8192(cuda_device, n_avg):
    """N = 8192 (the persistent kernel): n_avg 1 and 32 sum across lanes, 64 and
    256 go through the shared-memory buffer (and the barrier that ends each
    segment); all against the oracle over two blocks, split and whole alike."""
    args = (313.0, 2.0, 32, 50.0, 8192, n_avg)
    geo = O.plan_geometry(*args)
    vin = complex_int8_voltages(25, 6 * geo.hop, 32, 20.0)
    out_o, _ = oracle_run(vin, args, 6 * geo.hop)
    whole, _ = gpu_run(vin, args, 6, 1, volt=False)
    split, _ = gpu_run(vin, args, 3, 2, volt=False)
    assert np.array_equal(split, whole)
    assert np.all(rel_rms_rows(whole, out_o) <= TOL)


@pytest.mark.parametrize("args, q", [
    ((325.0, 4.0, 64, 10.0, 1024, 8), 5),       # 64 channels: whole tiles across, rows ragged
    ((325.0, 4.5, 72, 10.0, 1024, 8), 3),       # 72 channels: a ragged last channel tile
    ((325.0, 32.0, 512, 50.0, 8192, 16), 2),    # the 512-channel block shape
    ((325.0, 2.3125, 37, 10.0, 512, 4), 4),     # 37 channels: not a multiple of 8, the default turn
    ((150.0, 4.0, 64, 100.0, 65536, 16), 1),    # the channel-major copy of a cluster shape
])
def test_tma_corner_turn_same_bits(cuda_device, args, q):
    """The corner turn as tensor tile copies (CDD_ATTR_TURN_TMA) gives the
    same outputs, bit for bit, as the default turn, and within the bound of
    the oracle; it reports no device error."""
    import torch
    from paper_1509_00186_b300.cdd import Plan
    outs = []
    for tma in (False, True):
        with Plan(*args, segments_per_block=q, turn_tma=tma) as plan:
            bs, n_out, C = plan.block_samples, plan.n_out, plan.n_chan
            vin = complex_int8_voltages(31, bs * 2, C, 20.0)
            x = torch.from_numpy(np.ascontiguousarray(vin)).cuda()
            o = [plan.execute(x[b * bs:(b + 1) * bs]) for b in range(2)]
            torch.cuda.synchronize()
            assert plan.get("device_errors") == 0
            assert plan.get("turn_tma") == int(tma)
            outs.append(torch.cat(o, 1).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    want, _ = oracle_run(vin, args, bs * 2, channels=range(min(8, C)))
    assert rel_rms_rows(outs[1][:min(8, C)], want[:min(8, C)]).max() <= TOL
