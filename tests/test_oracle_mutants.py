"""Mutation check of the oracle's pins (CPU only).

Each case plants one plausible mistake (a dropped term, a wrong sign, index or
unit, a transposed reference) in a temporary copy of the oracle and runs the
pin file against it.  Every mutant must fail at least one pin.  The frozen
digest of the oracle's output is deselected: it fails on any change at all,
so it would hide a pin that misses the mistake.  An unmutated copy runs first
as the control and must pass.
"""

import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "cdd_oracle.py")

# name: (text in the oracle, the planted mistake)
MUTANTS = {
    "chirp_not_conjugated": ("return np.conj(np.exp(1j * chirp_phase(f_lo_mhz, f_l, dm)))",
                             "return (np.exp(1j * chirp_phase(f_lo_mhz, f_l, dm)))"),
    "lsb_chirp_sign": ("    return np.exp(1j * chirp_phase(f_lo_mhz, f_l, dm)) * taper",
                       "    return np.exp(-1j * chirp_phase(f_lo_mhz, f_l, dm)) * taper"),
    "lsb_not_mirrored": ("f_l = f_l[(-np.arange(n_fft)) % n_fft]", "f_l = f_l"),
    "lsb_wrong_reference": ("dispersion_delay_s(f_lo, f_lo.min(), dm)",
                            "dispersion_delay_s(f_lo, f_lo[0], dm)"),
    "no_half_channel_offset": ("+ chan_bw_mhz / 2.0\n", "\n"),
    "discard_at_the_end": ("out[:] = y[:, n_ov:].reshape(-1)", "out[:] = y[:, :hop].reshape(-1)"),
    "shifted_reference_edge": ("((f_l + f_lo) * f_lo ** 2)", "((f_l + f_lo) * (f_lo+0.0625) ** 2)"),
    "units_1e3_for_1e6": ("D_DISP_S_MHZ2 * 1e6 * dm", "D_DISP_S_MHZ2 * 1e3 * dm"),
    "shift_sign": ("np.rint(-delay", "np.rint(delay"),
    "mean_for_sum": (".sum(axis=-1)\n", ".mean(axis=-1)\n"),
    "hop_off_by_one": ("[::hop]", "[1::hop]"),
    "f_l_for_f_l_squared": ("dm * f_l ** 2 /", "dm * f_l /"),
    "detect_drops_imaginary": ("v.real ** 2 + v.imag ** 2", "v.real ** 2"),
    "overlap_not_rounded": ("n_ov = -(-n_ov // n_avg) * n_avg", "n_ov = n_ov"),
    "fullband_chirp_sign": ("corr = np.conj(h) if geo.sideband > 0 else h",
                            "corr = h if geo.sideband > 0 else h"),
    "fullband_lsb_not_inverted": ("f_l = f_bb if geo.sideband > 0 else geo.bandwidth_mhz - f_bb",
                                  "f_l = f_bb"),
    "fullband_half_band_delay": ("dispersion_delay_s(f_lo, f_lo + bandwidth_mhz, dm)",
                                 "dispersion_delay_s(f_lo, f_lo + bandwidth_mhz / 2, dm)"),
    "fullband_rate_b_for_2b": ("fs = 2.0 * bandwidth_mhz", "fs = bandwidth_mhz"),
    "fullband_discard": ("v[s * geo.hop:(s + 1) * geo.hop] = y[geo.n_ov:]",
                         "v[s * geo.hop:(s + 1) * geo.hop] = y[:geo.hop]"),
    "fullband_nyquist": ("full = np.concatenate([spec, np.zeros((spec.shape[0], 1))], axis=1)",
                         "full = np.concatenate([spec, spec[:, -1:]], axis=1)"),
    "batch_overlap_at_min_dm": ("float(dms.max())", "float(dms.min())"),
    "batch_overlap_at_tier_top": ("f_lo[tier_of == t].min()", "f_lo[tier_of == t].max()"),
    "batch_lsb_tier_order": ("else (n_chan - 1 - k) // per", "else k // per"),
    "dual_drops_second_pol": ("+ dedisperse(vin_b, geo, taper_kind)", "+ dedisperse(vin_a, geo, taper_kind)"),
    "band_sum_wrong_axis": ("return np.asarray(out).sum(axis=-2)", "return np.asarray(out).sum(axis=-1)"),
    "welch_as_hann": ("return 1.0 - (2.0 * x - 1.0) ** 2", "return np.sin(np.pi * x) ** 2"),
    "hann_cosine": ("return np.sin(np.pi * x) ** 2", "return np.cos(np.pi * x) ** 2"),
    "lsb_edges_off_by_one": ("chan_bw * (k + 1.0)", "chan_bw * k"),
    "unpack_conjugated": ("+ 1j * vin[:, k, 1]", "- 1j * vin[:, k, 1]"),
    "unpack_re_im_swapped": ("vin[:, k, 0].astype(np.float64) + 1j * vin[:, k, 1].astype(np.float64)",
                             "vin[:, k, 1].astype(np.float64) + 1j * vin[:, k, 0].astype(np.float64)"),
    "align_advances": ("out[shift:] = intensity[: intensity.shape[-1] - shift]",
                       "out[: intensity.shape[-1] - shift] = intensity[shift:]"),
    "sec23_rule_not_doubled": ("_next_pow2_above(2.0 * n_d), _next_pow2_above(n_ov), 64)",
                               "_next_pow2_above(n_d), _next_pow2_above(n_ov), 64)"),
    "overlap_from_highest_channel": ("dispersion_samples(float(f_lo.min()), chan_bw, dm)",
                                     "dispersion_samples(float(f_lo.max()), chan_bw, dm)"),
    "delay_sign": ("(f ** -2 - float(f_ref_mhz) ** -2)", "(float(f_ref_mhz) ** -2 - f ** -2)"),
    "chirp_pi_for_2pi": ("return 2.0 * np.pi * D_DISP_S_MHZ2", "return np.pi * D_DISP_S_MHZ2"),
    "bin_offsets_reversed": ("return np.fft.fftfreq(n_fft, d=1.0 / chan_bw_mhz)",
                             "return -np.fft.fftfreq(n_fft, d=1.0 / chan_bw_mhz)"),
    "fullband_detect_magnitude": ("integrate(v * v, geo.n_avg)", "integrate(np.abs(v), geo.n_avg)"),
    "fullband_overlap_not_frames": ("n_ov = -(-int(math.ceil(n_d)) // unit) * unit", "n_ov = int(math.ceil(n_d))"),
    "history_ignored": ("xp = np.concatenate([np.asarray(history, dtype=np.complex128),",
                        "xp = np.concatenate([np.zeros(n_ov, dtype=np.complex128),"),
    "inverse_and_forward_swapped": ("y = idft(dft(segs) * filt)", "y = dft(idft(segs) * filt)"),
    "every_channel_gets_channel_0_filter": ("dedispersion_filter(float(geo.f_lo_mhz[k]), geo.chan_bw_mhz, geo.dm,",
                                            "dedispersion_filter(float(geo.f_lo_mhz[0]), geo.chan_bw_mhz, geo.dm,"),
    "every_channel_gets_channel_0_shift": ("align(i_k, int(geo.shift[k]))", "align(i_k, int(geo.shift[0]))"),
    "lsb_mirror_off_by_one": ("f_l = f_l[(-np.arange(n_fft)) % n_fft]", "f_l = f_l[::-1]"),
}


def _run_pins(source):
    """Run the pin file against an oracle with the given source; returns the
    pytest exit code."""
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        os.makedirs(os.path.join(d, "oracle"))
        with open(os.path.join(d, "oracle", "cdd_oracle.py"), "w") as fh:
            fh.write(source)
        shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(d, "oracle", "__init__.py"))
        os.makedirs(os.path.join(d, "tests"))
        for f in ("conftest.py", "test_oracle_pins.py"):
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
        shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
        env = {**os.environ, "PYTHONPATH": os.pathsep.join([d, ROOT]), "OMP_NUM_THREADS": "1"}
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            "--deselect", "tests/test_oracle_pins.py::test_oracle_digest_unchanged",
                            "tests/test_oracle_pins.py"],
                           cwd=d, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_every_planted_mistake_fails_a_pin():
    with open(ORACLE) as fh:
        src = fh.read()
    for name, (orig, _) in MUTANTS.items():
        assert src.count(orig) >= 1, f"{name}: the oracle no longer contains {orig!r}"
    assert _run_pins(src) == 0, "the unmutated oracle must pass its pins"
    sources = [src.replace(orig, bad, 1) for orig, bad in MUTANTS.values()]
    with ThreadPoolExecutor(max_workers=min(len(sources), os.cpu_count() or 1)) as ex:
        codes = list(ex.map(_run_pins, sources))
    # exit code 1 = some pin failed; anything else (2 = collection error and
    # so on) would mean the mutant broke the module rather than a result
    missed = [n for n, c in zip(MUTANTS, codes) if c != 1]
    assert not missed, f"no pin fails for: {missed} (exit codes {dict(zip(MUTANTS, codes))})"
