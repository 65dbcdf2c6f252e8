"""C-ABI checks that need no GPU: the library loads, exports every function the
header declares, and its host-side geometry equals the oracle's exactly."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cdd():
    from paper_1509_00186_b300 import build
    build.build()
    from paper_1509_00186_b300 import cdd as mod
    return mod


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(cdd_\w+)\s*\(", src, flags=re.M)
    return names


def test_library_exports_every_declared_symbol(cdd):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(cdd._lib, n), n
    assert set(names) == set(cdd.EXPORTS)


def test_version_and_strerror(cdd):
    assert cdd.cdd_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert cdd.strerror(code) and "unknown" not in cdd.strerror(code)
    assert "unknown" in cdd.strerror(-99)


GEOMS = [
    (325.0, 16.0, 256, 10.0, 64, 4),
    (325.0, 32.0, 512, 50.0, 8192, 16),
    (150.0, 32.0, 512, 100.0, 16384, 16),
    (150.0, 32.0, 512, 100.0, 65536, 16),
    (150.0, 32.0, 512, 100.0, 32768, 16),
    (610.0, 32.0, 512, 20.0, 0, 16),
    (325.0, 32.0, 512, 50.0, 0, 16),
    (235.0, 16.0, 256, 67.99, 0, 8),
    (650.0, 200.0, 2048, 35.0, 2048, 16),
    (325.0, 0.4375, 7, 3.0, 256, 2),
    (325.0, 16.0, 8, 0.0, 64, 4),
    (1000.0, 1.0, 3, 1000.0, 0, 1),
    (325.0, 32.0, 512, 50.0, 0, 1),            # Sec. 2.3 rule binds: N = 128, n_ov = 55
    (325.0, -32.0, 512, 50.0, 0, 1),
    (325.0, -32.0, 512, 50.0, 8192, 16),       # lower sideband
    (610.0, -16.0, 256, 70.0, 0, 8),
    (150.0, -32.0, 512, 100.0, 65536, 16),
]


@pytest.mark.parametrize("geo", GEOMS)
def test_geometry_matches_oracle(cdd, geo):
    f_c, bw, n_chan, dm, n_fft, n_avg = geo
    g = O.plan_geometry(f_c, bw, n_chan, dm, n_fft, n_avg)
    p = cdd.cdd_plan_create(f_c, bw, n_chan, dm, n_fft, n_avg)
    try:
        assert cdd.cdd_plan_get(p, "n_fft") == g.n_fft
        assert cdd.cdd_plan_get(p, "n_ov") == g.n_ov
        assert cdd.cdd_plan_get(p, "hop") == g.hop
        assert cdd.cdd_plan_get(p, "r_max") == int(g.shift.max())
        assert np.array_equal(np.array(cdd.cdd_plan_shifts(p, n_chan)), g.shift)
        cdd.cdd_plan_set(p, "segments_per_block", 6)
        assert cdd.cdd_plan_get(p, "block_samples") == 6 * g.hop
        assert cdd.cdd_plan_get(p, "n_out_per_block") == 6 * g.hop // n_avg
        assert cdd.cdd_plan_get(p, "bytes_device") == 0
    finally:
        cdd.cdd_destroy(p)


def test_invalid_geometry_is_rejected(cdd):
    bad = [
        (325.0, 32.0, 512, 50.0, 48, 16),      # N not a power of two
        (325.0, 32.0, 512, 50.0, 64, 16),      # N <= n_ov
        (325.0, 0.0, 512, 50.0, 0, 16),        # no bandwidth
        (325.0, 32.0, 0, 50.0, 0, 16),         # no channels
        (325.0, 32.0, 512, -5.0, 0, 16),       # negative DM
        (325.0, 32.0, 512, 50.0, 0, 0),        # no integration
        (10.0, 32.0, 512, 50.0, 0, 16),        # band below 0 MHz
        (325.0, 32.0, 512, 50.0, 128, 48),     # hop not a multiple of n_avg
        (float("nan"), 32.0, 512, 50.0, 0, 16),  # not a frequency
        (325.0, 32.0, 512, float("inf"), 0, 16),  # not a DM
        (325.0, 32.0, 512, 50.0, -8192, 16),   # negative N
    ]
    for args in bad:
        with pytest.raises(cdd.CddError) as ei:
            cdd.cdd_plan_create(*args)
        assert ei.value.code == cdd.CDD_EINVAL, args
    with pytest.raises(cdd.CddError) as ei:
        cdd.cdd_plan_create(150.0, 32.0, 512, 100.0, 131072, 16)    # valid, not in this library
    assert ei.value.code == cdd.CDD_EUNSUPPORTED
    with pytest.raises(cdd.CddError) as ei:                         # window spans two CTAs
        cdd.cdd_plan_create(150.0, 32.0, 512, 100.0, 65536, 2048)
    assert ei.value.code in (cdd.CDD_EUNSUPPORTED, cdd.CDD_EINVAL)


def test_setters(cdd):
    p = cdd.cdd_plan_create(325.0, 32.0, 512, 50.0, 8192, 16)
    try:
        for attr, val in (("segments_per_block", 0), ("taper", 7), ("pipeline_chunks", 3),
                          ("n_fft", 1024),
                          ("segments_per_block", (1 << 24) + 1),     # beyond the per-call limit
                          ("segments_per_block", 1 << 20),           # q*h*C above 2^40 samples
                          ("polarisations", 3), ("stage_timing", 2), ("r_max", 5)):
            with pytest.raises(cdd.CddError):
                cdd.cdd_plan_set(p, attr, val)
        cdd.cdd_plan_set(p, "segments_per_block", 76)
        assert cdd.cdd_plan_get(p, "pipeline_chunks") == 19          # 19 chunks of 4 segments
        cdd.cdd_plan_set(p, "pipeline_chunks", 2)
        assert cdd.cdd_plan_get(p, "pipeline_chunks") == 2
        cdd.cdd_plan_set(p, "taper", cdd.TAPER["welch"])
        assert cdd.cdd_plan_get(p, "taper") == 2
        # precision: every form at N = 8192 (the tensor-core forms exist for it)
        for name in ("fp16", "fp16x2", "bf16x2", "bf16", "fp32"):
            cdd.cdd_plan_set(p, "precision", cdd.PRECISION[name])
            assert cdd.cdd_plan_get(p, "precision") == cdd.PRECISION[name]
        with pytest.raises(cdd.CddError) as ei:
            cdd.cdd_plan_set(p, "precision", 9)
        assert ei.value.code == cdd.CDD_EINVAL
        assert cdd.cdd_plan_get(p, "precision") == cdd.PRECISION["fp32"]
        # the corner turn's form: 0 (default) or 1 (tensor tile copies)
        assert cdd.cdd_plan_get(p, "turn_tma") == 0
        cdd.cdd_plan_set(p, "turn_tma", 1)
        assert cdd.cdd_plan_get(p, "turn_tma") == 1
        with pytest.raises(cdd.CddError) as ei:
            cdd.cdd_plan_set(p, "turn_tma", 2)
        assert ei.value.code == cdd.CDD_EINVAL
        cdd.cdd_plan_set(p, "turn_tma", 0)
        # nothing allocated yet: no error flag to read
        assert cdd.cdd_plan_get(p, "device_errors") == 0
    finally:
        cdd.cdd_destroy(p)
    # other transform lengths run FP32 only: the reduced forms are refused
    p = cdd.cdd_plan_create(325.0, 32.0, 512, 50.0, 4096, 16)
    try:
        for name in ("fp16", "fp16x2", "bf16x2", "bf16"):
            with pytest.raises(cdd.CddError) as ei:
                cdd.cdd_plan_set(p, "precision", cdd.PRECISION[name])
            assert ei.value.code == cdd.CDD_EUNSUPPORTED
        assert cdd.cdd_plan_get(p, "precision") == cdd.PRECISION["fp32"]
    finally:
        cdd.cdd_destroy(p)
    cdd.cdd_destroy(0)     # NULL is accepted


def test_stage_timing_attributes_before_commit(cdd):
    p = cdd.cdd_plan_create(325.0, 32.0, 512, 50.0, 8192, 16)
    try:
        assert cdd.cdd_plan_get(p, "stage_timing") == 0
        with pytest.raises(cdd.CddError):
            cdd.cdd_plan_set(p, "stage_timing", 2)
        cdd.cdd_plan_set(p, "stage_timing", 1)
        assert cdd.cdd_plan_get(p, "stage_timing") == 1
        for a in ("timed_blocks", "corner_turn_ns", "ols_ns"):      # nothing timed yet, no GPU call
            assert cdd.cdd_plan_get(p, a) == 0
        with pytest.raises(cdd.CddError):                           # read-only
            cdd.cdd_plan_set(p, "ols_ns", 5)
    finally:
        cdd.cdd_destroy(p)


def test_static_entry_rejects_before_touching_the_gpu(cdd):
    """cdd_execute_static checks geometry and its fixed scratch size first."""
    with pytest.raises(cdd.CddError) as ei:       # 2048 x 16384 chirp table = 256 MiB
        cdd.cdd_execute_static(650.0, 200.0, 2048, 35.0, 16384, 16, 1, 0, 1, 1)
    assert ei.value.code == cdd.CDD_ETOOBIG
    with pytest.raises(cdd.CddError) as ei:
        cdd.cdd_execute_static(325.0, 32.0, 512, 50.0, 48, 16, 1, 0, 1, 1)
    assert ei.value.code == cdd.CDD_EINVAL
    with pytest.raises(cdd.CddError) as ei:
        cdd.cdd_execute_static(325.0, 32.0, 512, 50.0, 8192, 16, 0, 0, 1, 1)
    assert ei.value.code == cdd.CDD_EINVAL


BATCH_GEOMS = [
    (650.0, 200.0, 2048, 20.0 + 0.5 * np.arange(64), (16384, 8192, 4096, 2048), 16),
    (650.0, 6.25, 64, [5.0, 10.0, 15.0, 20.0], (2048, 1024, 512, 256), 4),
    (325.0, 0.25, 4, [20.0], (256,), 4),
    (650.0, -6.25, 64, [5.0, 10.0, 15.0, 20.0], (2048, 1024, 512, 256), 4),   # lower sideband
    (325.0, -0.25, 4, [20.0], (256,), 4),
    # overlap set by the smear (above N/32) at the largest DM, both sidebands
    # (one tier: with two, these overlaps give hops that do not nest)
    (325.0, 32.0, 512, [10.0, 250.0, 600.0], (8192,), 16),
    (325.0, -32.0, 512, [10.0, 250.0, 600.0], (8192,), 16),
]


@pytest.mark.parametrize("geo", BATCH_GEOMS)
def test_batch_geometry_matches_oracle(cdd, geo):
    f_c, bw, n_chan, dms, tiers, n_avg = geo
    g = O.batch_geometry(f_c, bw, n_chan, dms, tiers, n_avg)
    b = cdd.cdd_batch_create(f_c, bw, n_chan, list(dms), tiers, n_avg)
    try:
        for t in range(len(tiers)):
            n_fft, n_ov, chan0, n_t = cdd.cdd_batch_tier(b, t)
            assert (n_fft, n_ov) == (g.tier_nfft[t], g.tier_nov[t])
            in_tier = np.flatnonzero(g.tier_of == t)              # tiers by frequency
            assert chan0 == in_tier.min() and n_t == in_tier.size == n_chan // len(tiers)
        assert np.array_equal(np.array(cdd.cdd_batch_shifts(b, len(dms), n_chan)), g.shift)
        assert cdd.cdd_batch_get(b, "r_max") == int(g.shift.max())
        n_out = cdd.cdd_batch_get(b, "n_out_per_block")
        assert n_out >= int(g.shift.max())
        assert cdd.cdd_batch_get(b, "block_samples") % max(g.hop(t) for t in range(len(tiers))) == 0
    finally:
        cdd.cdd_batch_destroy(b)


def test_batch_rejects_bad_requests(cdd):
    with pytest.raises(cdd.CddError):              # hops that do not nest
        cdd.cdd_batch_create(650.0, 6.25, 64, [51.5], (1024, 512, 256, 128), 4)
    with pytest.raises(cdd.CddError) as ei:        # tier N beyond the single-CTA shapes
        cdd.cdd_batch_create(650.0, 6.25, 64, [5.0], (32768, 16384), 4)
    assert ei.value.code == cdd.CDD_EUNSUPPORTED
    with pytest.raises(cdd.CddError):              # channels do not split into tiers
        cdd.cdd_batch_create(650.0, 6.25, 63, [5.0], (2048, 1024), 4)
    b = cdd.cdd_batch_create(650.0, 6.25, 64, [5.0, 20.0], (2048, 1024, 512, 256), 4)
    try:
        assert cdd.cdd_batch_get(b, "taper") == 0
        with pytest.raises(cdd.CddError):          # not a taper
            cdd.cdd_batch_set(b, "taper", 3)
        cdd.cdd_batch_set(b, "taper", cdd.TAPER["hann"])
        assert cdd.cdd_batch_get(b, "taper") == 1
        r_max = cdd.cdd_batch_get(b, "r_max")
        with pytest.raises(cdd.CddError):          # a block shorter than the largest delay
            cdd.cdd_batch_set(b, "segments_per_block", 1) if r_max > 1984 // 4 else \
                cdd.cdd_batch_set(b, "segments_per_block", 0)
    finally:
        cdd.cdd_batch_destroy(b)


FULLBAND = [
    (325.0, 32.0, 512, 50.0, 0, 16),        # the 32 MHz GSB mode: N = 2^26
    (325.0, -32.0, 512, 50.0, 0, 16),       # the same band as a lower sideband
    (610.0, 16.0, 256, 10.0, 0, 16),
    (610.0, 1.0, 32, 20.0, 0, 4),
    (325.0, 2.0, 64, 5.0, 1 << 20, 8),
    (610.0, 1.0, 32, 0.0, 1 << 14, 4),      # DM 0: no overlap
]


@pytest.mark.parametrize("geo", FULLBAND)
def test_fullband_geometry_matches_oracle(cdd, geo):
    f_c, bw, C, dm, n_fft, n_avg = geo
    g = O.fullband_geometry(f_c, bw, C, dm, n_fft, n_avg)
    f = cdd.cdd_fullband_create(f_c, bw, C, dm, n_fft, n_avg)
    try:
        assert cdd.cdd_fullband_get(f, "n_fft") == g.n_fft
        assert cdd.cdd_fullband_get(f, "n_ov") == g.n_ov
        assert cdd.cdd_fullband_get(f, "hop") == g.hop
        assert cdd.cdd_fullband_get(f, "block_samples") * 2 * C == g.hop
    finally:
        cdd.cdd_fullband_destroy(f)
    if geo[0] == 325.0 and geo[1] == 32.0:
        assert g.n_fft == 2 ** 26


@pytest.mark.parametrize("logn, want", [
    (14, (14, [])),                 # one shared-memory transform
    (15, (14, [1])),                # one radix-2 register pass
    (18, (14, [4])),                # one radix-16 pass
    (19, (14, [4, 1])),             # radix 16 then 2
    (20, (13, [7])),                # 8192-point transforms and one radix-128 tile pass
    (21, (13, [6, 2])),
    (24, (13, [7, 4])),
    (25, (13, [6, 6])),
    (26, (13, [6, 7])),             # the 32 MHz mode: radix 64 then 128
    (27, (13, [7, 7])),
])
def test_fullband_pass_plan(cdd, logn, want):
    """Every outer pass plan covers log2 N exactly, and the plans are those the
    full-band parity tests run (CDD_ATTR_PASS_PLAN)."""
    f = cdd.cdd_fullband_create(325.0, 2.0, 64, 5.0, 1 << logn, 4)
    try:
        pp = cdd.cdd_fullband_get(f, "pass_plan")
    finally:
        cdd.cdd_fullband_destroy(f)
    logs, lrs, sh = pp & 0xFF, [], 8
    while (pp >> sh) & 0xF:
        lrs.append((pp >> sh) & 0xF)
        sh += 4
    assert (logs, lrs) == want
    assert logs + sum(lrs) == logn


def test_fullband_rejects_bad_requests(cdd):
    for args in [(325.0, 32.0, 500, 50.0, 0, 16),          # frame not a power of two
                 (325.0, 32.0, 512, 50.0, 1 << 20, 16),    # N below the smear
                 (325.0, 0.0, 512, 50.0, 0, 16)]:          # no bandwidth
        with pytest.raises(cdd.CddError):
            cdd.cdd_fullband_create(*args)
    with pytest.raises(cdd.CddError) as ei:                 # N = 2^28: beyond this library
        cdd.cdd_fullband_create(325.0, 32.0, 512, 200.0, 0, 16)
    assert ei.value.code == cdd.CDD_EUNSUPPORTED


def test_stream_state_blob_before_any_launch(cdd):
    """The checkpoint blob: its size, the fresh-stream export (no GPU touched),
    and refusal of a blob from another geometry or of a short buffer."""
    a = cdd.cdd_plan_create(325.0, 32.0, 64, 50.0, 8192, 16)
    b = cdd.cdd_plan_create(325.0, 32.0, 64, 60.0, 8192, 16)         # another DM
    try:
        cdd.cdd_plan_set(a, "segments_per_block", 4)
        cdd.cdd_plan_set(b, "segments_per_block", 4)
        n = cdd.cdd_plan_state_bytes(a)
        r_max, n_ov = cdd.cdd_plan_get(a, "r_max"), cdd.cdd_plan_get(a, "n_ov")
        assert n > 64 * (2 * n_ov + 4 * r_max)
        blob = cdd.cdd_plan_export_state(a)
        assert len(blob) == n and blob[:4] == b"SDDC"
        assert not any(blob[120:])                                  # zero history
        for target, data in ((b, blob), (a, blob[:-1])):
            with pytest.raises(cdd.CddError) as ei:
                cdd.cdd_plan_import_state(target, data)
            assert ei.value.code == cdd.CDD_EINVAL
    finally:
        cdd.cdd_destroy(a)
        cdd.cdd_destroy(b)



def test_batch_state_blob_before_any_launch(cdd):
    """The batch checkpoint blob: size, fresh-stream export (no GPU touched),
    refusal of another geometry (DM list, segments per block) or a short
    buffer."""
    tiers = (2048, 1024, 512, 256)
    a = cdd.cdd_batch_create(650.0, 6.25, 64, [5.0, 10.0, 15.0, 20.0], tiers, 4)
    b = cdd.cdd_batch_create(650.0, 6.25, 64, [5.0, 10.0, 15.0, 21.0], tiers, 4)   # another DM list
    c = cdd.cdd_batch_create(650.0, 6.25, 64, [5.0, 10.0, 15.0, 20.0], tiers, 4)
    try:
        cdd.cdd_batch_set(c, "segments_per_block", cdd.cdd_batch_get(a, "segments_per_block") + 1)
        n = cdd.cdd_batch_state_bytes(a)
        r_max = cdd.cdd_batch_get(a, "r_max")
        assert n >= 88 + 64 * 2 + 4 * 64 * 4 * r_max
        blob = cdd.cdd_batch_export_state(a)
        assert len(blob) == n and blob[:4] == b"SDDB"
        assert not any(blob[88:])                                   # zero history
        for target, data in ((b, blob), (c, blob), (a, blob[:-1])):
            with pytest.raises(cdd.CddError) as ei:
                cdd.cdd_batch_import_state(target, data)
            assert ei.value.code == cdd.CDD_EINVAL
    finally:
        for h in (a, b, c):
            cdd.cdd_batch_destroy(h)


def test_batch_phase_table_form(cdd):
    """The batch keeps the DM = 1 chirp phase as single floats when no phase
    exceeds 16 turns (650 MHz, DMs to 51.5: 12.2 turns) and as two floats
    otherwise (150 MHz, DM 20: 238 turns)."""
    for args, want in (((650.0, 200.0, 2048, list(20.0 + 0.5 * np.arange(64)),
                         (16384, 8192, 4096, 2048), 16), 1),
                       ((150.0, 1.5625, 16, [15.0, 20.0], (16384,), 4), 2)):
        b = cdd.cdd_batch_create(*args)
        try:
            assert cdd.cdd_batch_get(b, "phase_floats") == want
        finally:
            cdd.cdd_batch_destroy(b)


def test_batch_form_attribute(cdd):
    """CDD_ATTR_BATCH_FORM: -1 (tune at the first execute) by default; 0..2
    settable before the first execute; anything else refused."""
    b = cdd.cdd_batch_create(650.0, 0.78125, 8, [20.0, 30.0], [16384, 8192, 4096, 2048], 16)
    try:
        assert cdd.cdd_batch_get(b, "batch_form") == -1
        for f in (0, 1, 2, -1):
            cdd.cdd_batch_set(b, "batch_form", f)
            assert cdd.cdd_batch_get(b, "batch_form") == f
        for bad in (3, -2):
            with pytest.raises(cdd.CddError) as ei:
                cdd.cdd_batch_set(b, "batch_form", bad)
            assert ei.value.code == cdd.CDD_EINVAL
        assert cdd.cdd_batch_get(b, "tune_ns_multi") == 0
    finally:
        cdd.cdd_batch_destroy(b)
