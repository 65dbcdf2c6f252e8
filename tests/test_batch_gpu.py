"""Batched form on the GPU (many DM trials sharing each forward transform,
tiered N) against the FP64 oracle, relative RMS <= 1e-5 per DM plane."""
import numpy as np
import pytest

import oracle as O
from synth import complex_int8_voltages

pytestmark = pytest.mark.gpu
TOL = 1e-5

SMALL = (650.0, 6.25, 64, [5.0, 10.0, 15.0, 20.0], (2048, 1024, 512, 256), 4)


def run_batch(vin, args, q, n_blocks, taper="none"):
    import torch
    from paper_1509_00186_b300.cdd import Batch
    with Batch(*args, segments_per_block=q, taper=taper) as b:
        bs = b.block_samples
        x = torch.from_numpy(np.ascontiguousarray(vin[: bs * n_blocks])).cuda()
        outs = [b.execute(x[i * bs:(i + 1) * bs]) for i in range(n_blocks)]
        torch.cuda.synchronize()
        return torch.cat(outs, 2).cpu().numpy()


@pytest.fixture(scope="module")
def small(cuda_device):
    g = O.batch_geometry(*SMALL)
    vin = complex_int8_voltages(3, 1984 * 8, 64, 20.0)
    want = O.dedisperse_batch(vin, g)
    return vin, g, want


def test_small_batch_matches_oracle(small):
    vin, g, want = small
    got = run_batch(vin, SMALL, 2, 4)
    assert got.shape == want.shape == (4, 64, 1984 * 8 // 4)
    for d in range(4):
        assert O.rel_rms(got[d], want[d]) <= TOL, d
        for k in (0, 17, 40, 63):                 # one channel in each tier
            assert O.rel_rms(got[d, k], want[d, k]) <= TOL, (d, k)
    # the last tier (N = 256) and the first (N = 2048) both carry the shifts
    for d in range(4):
        r = int(g.shift[d, 63])
        assert np.all(got[d, 63, :r] == 0.0)


def test_batch_block_split_is_bit_identical(small):
    vin, g, _ = small
    a = run_batch(vin, SMALL, 8, 1)
    b = run_batch(vin, SMALL, 2, 4)
    c = run_batch(vin, SMALL, 1, 8)
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("bandwidth,taper", [(-6.25, "none"), (6.25, "hann"), (-6.25, "welch")])
def test_batch_lower_sideband_and_taper(cuda_device, bandwidth, taper):
    """A lower-sideband band (tiers by frequency: the longest transform on the
    last channels) and tapered chirps, every DM plane against the oracle."""
    args = (650.0, bandwidth, 64, [5.0, 10.0, 15.0, 20.0], (2048, 1024, 512, 256), 4)
    g = O.batch_geometry(*args)
    vin = complex_int8_voltages(28, 1984 * 4, 64, 20.0)
    want = O.dedisperse_batch(vin, g, taper_kind=taper)
    got = run_batch(vin, args, 2, 2, taper)
    assert got.shape == want.shape
    for d in range(len(args[3])):
        assert O.rel_rms(got[d], want[d]) <= TOL, d


@pytest.mark.parametrize("bandwidth", [4.0, -4.0])
def test_batch_overlap_set_by_the_smear(cuda_device, bandwidth):
    """DM 300 at 325 MHz smears 288 samples across the lowest 62.5 kHz
    channel, far above N/32 = 16: the overlap (292) comes from the smear, and
    each block spans 82 hops to outlast a 4463-sample alignment shift.  Both
    sidebands, every DM plane against the oracle."""
    args = (325.0, bandwidth, 64, [10.0, 300.0], (512,), 4)
    g = O.batch_geometry(*args)
    assert g.tier_nov == (292,)
    vin = complex_int8_voltages(29, g.hop(0) * 82 * 2, 64, 20.0)
    want = O.dedisperse_batch(vin, g)
    got = run_batch(vin, args, 82, 2)
    assert got.shape == want.shape
    for d in range(2):
        assert O.rel_rms(got[d], want[d]) <= TOL, d


def test_batch_with_a_dm_zero_trial(cuda_device):
    """A DM-0 trial beside a dispersed one: its plane is every channel's
    integrated power, unshifted; both planes against the oracle."""
    args = (650.0, 6.25, 64, [0.0, 12.5], (2048, 1024, 512, 256), 4)
    g = O.batch_geometry(*args)
    assert np.all(g.shift[0] == 0)
    vin = complex_int8_voltages(31, 1984 * 4, 64, 20.0)
    want = O.dedisperse_batch(vin, g)
    got = run_batch(vin, args, 2, 2)
    assert got.shape == want.shape
    for d in range(2):
        assert O.rel_rms(got[d], want[d]) <= TOL, d


def test_batch_checkpoint_resume_is_bit_identical(small):
    """Two blocks in one batch, its state exported; a new batch of the same
    geometry imports it and runs the next two: all four blocks equal the
    uninterrupted run bit for bit."""
    import torch
    from paper_1509_00186_b300.cdd import Batch
    vin, g, _ = small
    ref = run_batch(vin, SMALL, 2, 4)
    with Batch(*SMALL, segments_per_block=2) as b:
        bs = b.block_samples
        x = torch.from_numpy(np.ascontiguousarray(vin[: bs * 4])).cuda()
        first = [b.execute(x[i * bs:(i + 1) * bs]) for i in range(2)]
        blob = b.export_state()
        assert b.get("blocks_done") == 2
    with Batch(*SMALL, segments_per_block=2) as b2:
        b2.import_state(blob)
        assert b2.get("blocks_done") == 2
        rest = [b2.execute(x[i * bs:(i + 1) * bs]) for i in range(2, 4)]
        torch.cuda.synchronize()
    got = torch.cat(first + rest, 2).cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.slow
def test_upgraded_gmrt_batch_full_size_sampled(cuda_device):
    """200 MHz at 650 MHz, 2048 channels, 64 DM trials 20.0..51.5, tiers
    N = 16384 / 8192 / 4096 / 2048, 4 s, one block of 24 longest hops; sampled
    (DM, channel) pairs against the oracle."""
    import torch
    from paper_1509_00186_b300.cdd import Batch
    dms = list(20.0 + 0.5 * np.arange(64))
    args = (650.0, 200.0, 2048, dms, (16384, 8192, 4096, 2048), 16)
    g = O.batch_geometry(*args)
    n_samp = int(round(4.0 * 200e6 / 2048))        # 390,625
    q = n_samp // g.hop(0)
    vin = complex_int8_voltages(4, q * g.hop(0), 2048, 20.0)
    with Batch(*args, segments_per_block=q) as b:
        out = b.execute(torch.from_numpy(vin).cuda())
        pairs = [(0, 0), (63, 511), (30, 512), (5, 1500), (63, 2047), (17, 1024)]
        got = np.stack([out[d, k].cpu().numpy() for d, k in pairs])
        assert bool(torch.isfinite(out).all())
    for i, (d, k) in enumerate(pairs):
        want = O.dedisperse_batch(vin, g, channels=[k], dm_index=[d])[0, 0]
        assert O.rel_rms(got[i], want) <= TOL, (d, k)


@pytest.mark.parametrize("n_avg", [32, 64])
def test_batch_persistent_tiers(cuda_device, n_avg):
    """Tiers of 8192 points (the persistent batch kernel) and 4096 points
    (three CTAs per SM): n_avg 32 sums across lanes, 64 through shared memory;
    every DM plane against the oracle, and a block split gives the same bits."""
    args = (650.0, 1.5625, 16, [5.0, 10.0, 15.0], (8192, 4096), n_avg)
    g = O.batch_geometry(*args)
    h = g.hop(0)
    vin = complex_int8_voltages(26, h * 4, 16, 20.0)
    want = O.dedisperse_batch(vin, g)
    got = run_batch(vin, args, 2, 2)
    assert got.shape == want.shape
    for d in range(len(args[3])):
        assert O.rel_rms(got[d], want[d]) <= TOL, d
    assert np.array_equal(run_batch(vin, args, 4, 1), got)


def test_batch_two_float_phase_table(cuda_device):
    """Chirp phases up to 238 turns (150 MHz, DM 20) keep the two-float phase
    table; every DM plane against the oracle."""
    from paper_1509_00186_b300.cdd import Batch
    args = (150.0, 1.5625, 16, [15.0, 20.0], (16384,), 4)
    g = O.batch_geometry(*args)
    vin = complex_int8_voltages(27, g.hop(0) * 3, 16, 20.0)
    with Batch(*args, segments_per_block=1) as b:
        assert b.get("phase_floats") == 2
    want = O.dedisperse_batch(vin, g)
    got = run_batch(vin, args, 1, 3)
    for d in range(2):
        assert O.rel_rms(got[d], want[d]) <= TOL, d


def test_batch_one_float_phase_table(small):
    """The small band's phases (under 3 turns) use the single-float table."""
    from paper_1509_00186_b300.cdd import Batch
    with Batch(*SMALL, segments_per_block=1) as b:
        assert b.get("phase_floats") == 1


# tiers of 16384 .. 2048 points (the upgraded-GMRT tiering) on a narrow band:
# every launch form applies, the one-launch form included
FORMS = (650.0, 0.78125, 8, [20.0, 30.0, 35.0, 40.0], (16384, 8192, 4096, 2048), 16)


def run_form(vin, form, q, n_blocks):
    import torch
    from paper_1509_00186_b300.cdd import Batch
    with Batch(*FORMS, segments_per_block=q, form=form) as b:
        bs = b.block_samples
        x = torch.from_numpy(np.ascontiguousarray(vin[: bs * n_blocks])).cuda()
        outs = [b.execute(x[i * bs:(i + 1) * bs]) for i in range(n_blocks)]
        torch.cuda.synchronize()
        info = {k: b.get(k) for k in ("batch_form", "tune_ns_tiers", "tune_ns_tiers_np", "tune_ns_multi",
                                      "kernel_launches")}
        return torch.cat(outs, 2).cpu().numpy(), info


def test_batch_launch_forms_are_bit_identical_and_match_the_oracle(cuda_device):
    """Per-tier launches and the one-launch persistent form give the same
    bits over two blocks; the per-tier form without the persistent N = 8192
    kernel (first-pass twiddles formed as products) agrees within the
    tolerance; all against the oracle."""
    g = O.batch_geometry(*FORMS)
    q = 2
    vin = complex_int8_voltages(51, 2 * q * g.hop(0), 8, 20.0)
    outs = {}
    for form in ("tiers", "tiers_np", "multi"):
        outs[form], info = run_form(vin, form, q, 2)
        assert info["batch_form"] == {"tiers": 0, "tiers_np": 1, "multi": 2}[form]
    assert np.array_equal(outs["tiers"], outs["multi"])
    want = O.dedisperse_batch(vin[: 2 * q * g.hop(0)], g)
    for d in range(4):
        assert O.rel_rms(outs["multi"][d], want[d]) <= TOL, d
        assert O.rel_rms(outs["tiers_np"][d], want[d]) <= TOL, d


def test_batch_tuning_picks_a_form_and_remembers_it(cuda_device):
    """With the form left to tuning, the first execute times the per-tier and
    the one-launch forms (each time reported), keeps the faster, and gives the
    same bits as a forced form; a second batch of the same shape reuses the
    choice without timing."""
    g = O.batch_geometry(*FORMS)
    vin = complex_int8_voltages(52, 2 * g.hop(0), 8, 20.0)
    forced, _ = run_form(vin, "tiers", 2, 1)
    tuned, info = run_form(vin, "tune", 2, 1)
    assert np.array_equal(tuned, forced)
    assert info["batch_form"] in (0, 2)
    times = {0: info["tune_ns_tiers"], 2: info["tune_ns_multi"]}
    assert all(t > 0 for t in times.values()) and info["tune_ns_tiers_np"] == 0
    assert times[info["batch_form"]] == min(times.values())
    again, info2 = run_form(vin, "tune", 2, 1)
    assert np.array_equal(again, forced)
    assert info2["batch_form"] == info["batch_form"]
    assert info2["tune_ns_tiers"] == info2["tune_ns_tiers_np"] == info2["tune_ns_multi"] == 0
