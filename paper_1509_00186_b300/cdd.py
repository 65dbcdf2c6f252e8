"""Thin Python binding of the C ABI in include/cdd.h (argument marshalling only).

Functions keep the C names; every computation happens in libcdd.so's CUDA
kernels.  Importing this module loads the in-tree library and fails loudly
if it is missing: there is no fallback.

``Plan`` is a small convenience wrapper that takes torch tensors (device or
pinned host) and passes their pointers and the current CUDA stream through.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcdd.so")

CDD_OK = 0
CDD_EINVAL = -1
CDD_ENOMEM = -2
CDD_ECUDA = -3
CDD_EUNSUPPORTED = -4
CDD_ESTATE = -5
CDD_ETOOBIG = -6
CDD_EBUSY = -7
STATIC_SCRATCH_BYTES = 64 * 1024 * 1024

ATTR = {
    "n_fft": 0, "n_ov": 1, "hop": 2, "n_avg": 3, "n_chan": 4, "segments_per_block": 5,
    "block_samples": 6, "n_out_per_block": 7, "r_max": 8, "bytes_device": 9, "taper": 10,
    "blocks_done": 11, "pipeline_chunks": 12, "kernel_launches": 13, "bytes_needed": 14,
    "seq_gaps": 15, "polarisations": 16, "stage_timing": 17, "timed_blocks": 18,
    "corner_turn_ns": 19, "ols_ns": 20, "phase_floats": 22, "precision": 23,
    "device_errors": 24, "host_staging_bytes": 25, "batch_form": 26, "tune_ns_tiers": 27,
    "tune_ns_tiers_np": 28, "tune_ns_multi": 29, "turn_tma": 30, "pass_plan": 31,
}
BATCH_FORM = {"tune": -1, "tiers": 0, "tiers_np": 1, "multi": 2}
POOL_ATTR = {"budget": 100, "used_bytes": 101, "streams": 102, "queued": 103}
POOL_HOST_INGEST = 1
TAPER = {"none": 0, "hann": 1, "welch": 2}
PRECISION = {"fp32": 0, "fp16": 1, "fp16x2": 2, "bf16x2": 3, "bf16": 4}

# every symbol include/cdd.h declares
EXPORTS = ("cdd_plan_create", "cdd_plan_set", "cdd_plan_get", "cdd_plan_shifts", "cdd_execute",
           "cdd_execute_voltages", "cdd_execute_host", "cdd_execute_static", "cdd_reset",
           "cdd_destroy", "cdd_strerror", "cdd_version",
           "cdd_batch_create", "cdd_batch_set", "cdd_batch_get", "cdd_batch_tier",
           "cdd_batch_shifts", "cdd_batch_execute", "cdd_batch_reset", "cdd_batch_destroy",
           "cdd_plan_commit", "cdd_execute_dual", "cdd_band_sum", "cdd_pool_create", "cdd_pool_admit", "cdd_pool_stream_get",
           "cdd_pool_submit", "cdd_pool_wait", "cdd_pool_release", "cdd_pool_get",
           "cdd_pool_destroy", "cdd_fullband_create", "cdd_fullband_set", "cdd_fullband_get",
           "cdd_fullband_execute", "cdd_fullband_reset", "cdd_fullband_destroy",
           "cdd_plan_state_bytes", "cdd_plan_export_state", "cdd_plan_import_state",
           "cdd_pool_stream_state_bytes", "cdd_pool_stream_export", "cdd_pool_stream_import",
           "cdd_batch_state_bytes", "cdd_batch_export_state", "cdd_batch_import_state",
           "cdd_execute_host_async", "cdd_plan_prepare_host", "cdd_pool_clock_ms", "cdd_pool_admit_ex",
           "cdd_pool_request", "cdd_pool_request_status", "cdd_pool_submit_at", "cdd_pool_submit_host",
           "cdd_pool_submit_many", "cdd_pool_stream_resync", "cdd_selftest_wait_limit")


class CddError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1509_00186_b300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    lib.cdd_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.cdd_plan_set.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    lib.cdd_plan_get.argtypes = [vp, ctypes.c_int, i64p]
    lib.cdd_plan_shifts.argtypes = [vp, i64p]
    lib.cdd_plan_state_bytes.argtypes = [vp, i64p]
    lib.cdd_plan_export_state.argtypes = [vp, vp, ctypes.c_int64, vp]
    lib.cdd_plan_import_state.argtypes = [vp, vp, ctypes.c_int64, vp]
    lib.cdd_pool_stream_state_bytes.argtypes = [vp, ctypes.c_int, i64p]
    lib.cdd_batch_state_bytes.argtypes = [vp, i64p]
    lib.cdd_batch_export_state.argtypes = [vp, vp, ctypes.c_int64, vp]
    lib.cdd_batch_import_state.argtypes = [vp, vp, ctypes.c_int64, vp]
    lib.cdd_pool_stream_export.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, i64p]
    lib.cdd_pool_stream_import.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int64]
    lib.cdd_execute.argtypes = [vp, vp, vp, vp]
    lib.cdd_execute_voltages.argtypes = [vp, vp, vp, vp, vp]
    lib.cdd_execute_host.argtypes = [vp, vp, vp, vp]
    lib.cdd_execute_static.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, vp, vp, vp]
    lib.cdd_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int]
    lib.cdd_batch_set.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    lib.cdd_batch_get.argtypes = [vp, ctypes.c_int, i64p]
    lib.cdd_batch_tier.argtypes = [vp, ctypes.c_int, i64p, i64p, i64p, i64p]
    lib.cdd_batch_shifts.argtypes = [vp, i64p]
    lib.cdd_batch_execute.argtypes = [vp, vp, vp, vp]
    lib.cdd_batch_reset.argtypes = [vp]
    lib.cdd_batch_destroy.argtypes = [vp]
    lib.cdd_plan_commit.argtypes = [vp]
    lib.cdd_fullband_create.argtypes = [ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_int]
    lib.cdd_fullband_set.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    lib.cdd_fullband_get.argtypes = [vp, ctypes.c_int, i64p]
    lib.cdd_fullband_execute.argtypes = [vp, vp, vp, vp]
    lib.cdd_fullband_reset.argtypes = [vp]
    lib.cdd_fullband_destroy.argtypes = [vp]
    lib.cdd_execute_dual.argtypes = [vp, vp, vp, vp, vp]
    lib.cdd_band_sum.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, vp, vp]
    lib.cdd_pool_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_int]
    lib.cdd_pool_admit.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.cdd_pool_stream_get.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64p]
    lib.cdd_pool_submit.argtypes = [vp, ctypes.c_int, ctypes.c_int64, vp, vp, i64p]
    lib.cdd_pool_wait.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    lib.cdd_pool_release.argtypes = [vp, ctypes.c_int]
    lib.cdd_pool_get.argtypes = [vp, ctypes.c_int, i64p]
    lib.cdd_pool_destroy.argtypes = [vp]
    lib.cdd_execute_host_async.argtypes = [vp, vp, vp, vp]
    lib.cdd_plan_prepare_host.argtypes = [vp]
    lib.cdd_pool_clock_ms.argtypes = []
    lib.cdd_pool_admit_ex.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.cdd_pool_request.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, i64p]
    lib.cdd_pool_request_status.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    lib.cdd_pool_submit_at.argtypes = [vp, ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_double, i64p]
    lib.cdd_pool_submit_host.argtypes = [vp, ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_double, i64p]
    lib.cdd_pool_submit_many.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p,
                                         ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int, i64p,
                                         ctypes.POINTER(ctypes.c_int)]
    lib.cdd_pool_stream_resync.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    lib.cdd_reset.argtypes = [vp]
    lib.cdd_destroy.argtypes = [vp]
    lib.cdd_strerror.argtypes = [ctypes.c_int]
    lib.cdd_strerror.restype = ctypes.c_char_p
    lib.cdd_version.argtypes = []
    lib.cdd_selftest_wait_limit.argtypes = [ctypes.POINTER(ctypes.c_int)]
    for name in EXPORTS:
        if name not in ("cdd_strerror", "cdd_pool_clock_ms"):
            getattr(lib, name).restype = ctypes.c_int
    lib.cdd_pool_clock_ms.restype = ctypes.c_double
    return lib


_lib = _load()


def _check(rc: int, where: str) -> None:
    if rc != CDD_OK:
        raise CddError(rc, where)


# ------------------------------------------------------------------ C names

def strerror(code: int) -> str:
    return _lib.cdd_strerror(int(code)).decode()


def cdd_version() -> int:
    return int(_lib.cdd_version())


def cdd_selftest_wait_limit() -> int:
    """Run the bounded-wait self-test; returns the kernel's error flag (2 expected)."""
    st = ctypes.c_int(0)
    _check(_lib.cdd_selftest_wait_limit(ctypes.byref(st)), "cdd_selftest_wait_limit")
    return int(st.value)


def cdd_plan_create(f_center_mhz: float, bandwidth_mhz: float, n_chan: int, dm: float,
                    n_fft: int = 0, n_avg: int = 1) -> int:
    h = ctypes.c_void_p()
    _check(_lib.cdd_plan_create(ctypes.byref(h), float(f_center_mhz), float(bandwidth_mhz),
                                int(n_chan), float(dm), int(n_fft), int(n_avg)), "cdd_plan_create")
    return h.value


def cdd_plan_set(plan: int, attr, value: int) -> None:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    _check(_lib.cdd_plan_set(ctypes.c_void_p(plan), a, int(value)), "cdd_plan_set")


def cdd_plan_get(plan: int, attr) -> int:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    v = ctypes.c_int64()
    _check(_lib.cdd_plan_get(ctypes.c_void_p(plan), a, ctypes.byref(v)), "cdd_plan_get")
    return int(v.value)


def cdd_plan_shifts(plan: int, n_chan: int):
    buf = (ctypes.c_int64 * n_chan)()
    _check(_lib.cdd_plan_shifts(ctypes.c_void_p(plan), buf), "cdd_plan_shifts")
    return list(buf)


def cdd_plan_state_bytes(plan: int) -> int:
    v = ctypes.c_int64()
    _check(_lib.cdd_plan_state_bytes(ctypes.c_void_p(plan), ctypes.byref(v)), "cdd_plan_state_bytes")
    return v.value


def cdd_plan_export_state(plan: int, stream: int = 0) -> bytes:
    n = cdd_plan_state_bytes(plan)
    buf = ctypes.create_string_buffer(n)
    _check(_lib.cdd_plan_export_state(ctypes.c_void_p(plan), buf, n, ctypes.c_void_p(stream)),
           "cdd_plan_export_state")
    return buf.raw


def cdd_plan_import_state(plan: int, state: bytes, stream: int = 0) -> None:
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(_lib.cdd_plan_import_state(ctypes.c_void_p(plan), buf, len(state), ctypes.c_void_p(stream)),
           "cdd_plan_import_state")


def cdd_batch_state_bytes(batch: int) -> int:
    v = ctypes.c_int64()
    _check(_lib.cdd_batch_state_bytes(ctypes.c_void_p(batch), ctypes.byref(v)), "cdd_batch_state_bytes")
    return v.value


def cdd_batch_export_state(batch: int, stream: int = 0) -> bytes:
    n = cdd_batch_state_bytes(batch)
    buf = ctypes.create_string_buffer(n)
    _check(_lib.cdd_batch_export_state(ctypes.c_void_p(batch), buf, n, ctypes.c_void_p(stream)),
           "cdd_batch_export_state")
    return buf.raw


def cdd_batch_import_state(batch: int, state: bytes, stream: int = 0) -> None:
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(_lib.cdd_batch_import_state(ctypes.c_void_p(batch), buf, len(state), ctypes.c_void_p(stream)),
           "cdd_batch_import_state")


def cdd_execute(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_execute(ctypes.c_void_p(plan), ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                            ctypes.c_void_p(stream)), "cdd_execute")


def cdd_execute_voltages(plan: int, d_in: int, d_out: int, d_volt: int, stream: int = 0) -> None:
    _check(_lib.cdd_execute_voltages(ctypes.c_void_p(plan), ctypes.c_void_p(d_in),
                                     ctypes.c_void_p(d_out), ctypes.c_void_p(d_volt),
                                     ctypes.c_void_p(stream)), "cdd_execute_voltages")


def cdd_execute_host(plan: int, h_in: int, h_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_execute_host(ctypes.c_void_p(plan), ctypes.c_void_p(h_in),
                                 ctypes.c_void_p(h_out), ctypes.c_void_p(stream)),
           "cdd_execute_host")


def cdd_execute_static(f_center_mhz: float, bandwidth_mhz: float, n_chan: int, dm: float,
                       n_fft: int, n_avg: int, n_seg: int, taper: int, d_in: int, d_out: int,
                       stream: int = 0) -> None:
    """One block from a fresh stream without any device allocation (see cdd.h)."""
    _check(_lib.cdd_execute_static(float(f_center_mhz), float(bandwidth_mhz), int(n_chan),
                                   float(dm), int(n_fft), int(n_avg), int(n_seg), int(taper),
                                   ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                   ctypes.c_void_p(stream)), "cdd_execute_static")


def cdd_reset(plan: int) -> None:
    _check(_lib.cdd_reset(ctypes.c_void_p(plan)), "cdd_reset")


def cdd_destroy(plan: int) -> None:
    _check(_lib.cdd_destroy(ctypes.c_void_p(plan)), "cdd_destroy")


def cdd_batch_create(f_center_mhz, bandwidth_mhz, n_chan, dms, tier_nfft, n_avg) -> int:
    h = ctypes.c_void_p()
    d = (ctypes.c_double * len(dms))(*[float(x) for x in dms])
    t = (ctypes.c_int * len(tier_nfft))(*[int(x) for x in tier_nfft])
    _check(_lib.cdd_batch_create(ctypes.byref(h), float(f_center_mhz), float(bandwidth_mhz),
                                 int(n_chan), d, len(dms), t, len(tier_nfft), int(n_avg)),
           "cdd_batch_create")
    return h.value


def cdd_batch_set(batch: int, attr, value: int) -> None:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    _check(_lib.cdd_batch_set(ctypes.c_void_p(batch), a, int(value)), "cdd_batch_set")


def cdd_batch_get(batch: int, attr) -> int:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    v = ctypes.c_int64()
    _check(_lib.cdd_batch_get(ctypes.c_void_p(batch), a, ctypes.byref(v)), "cdd_batch_get")
    return int(v.value)


def cdd_batch_tier(batch: int, t: int):
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(_lib.cdd_batch_tier(ctypes.c_void_p(batch), int(t), *[ctypes.byref(v) for v in vals]),
           "cdd_batch_tier")
    return tuple(int(v.value) for v in vals)


def cdd_batch_shifts(batch: int, n_dm: int, n_chan: int):
    buf = (ctypes.c_int64 * (n_dm * n_chan))()
    _check(_lib.cdd_batch_shifts(ctypes.c_void_p(batch), buf), "cdd_batch_shifts")
    return [list(buf[d * n_chan:(d + 1) * n_chan]) for d in range(n_dm)]


def cdd_batch_execute(batch: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_batch_execute(ctypes.c_void_p(batch), ctypes.c_void_p(d_in),
                                  ctypes.c_void_p(d_out), ctypes.c_void_p(stream)),
           "cdd_batch_execute")


def cdd_batch_reset(batch: int) -> None:
    _check(_lib.cdd_batch_reset(ctypes.c_void_p(batch)), "cdd_batch_reset")


def cdd_batch_destroy(batch: int) -> None:
    _check(_lib.cdd_batch_destroy(ctypes.c_void_p(batch)), "cdd_batch_destroy")


def cdd_execute_dual(plan: int, d_in_a: int, d_in_b: int, d_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_execute_dual(ctypes.c_void_p(plan), ctypes.c_void_p(d_in_a),
                                 ctypes.c_void_p(d_in_b), ctypes.c_void_p(d_out),
                                 ctypes.c_void_p(stream)), "cdd_execute_dual")


def cdd_band_sum(d_out: int, n_planes: int, n_chan: int, n_out: int, d_sum: int,
                 stream: int = 0) -> None:
    _check(_lib.cdd_band_sum(ctypes.c_void_p(d_out), int(n_planes), int(n_chan), int(n_out),
                             ctypes.c_void_p(d_sum), ctypes.c_void_p(stream)), "cdd_band_sum")


def band_sum(out):
    """Torch convenience: [..., C, n_out] device float32 -> [..., n_out] (in the library)."""
    import torch
    if out.dtype != torch.float32 or not out.is_contiguous() or out.device.type != "cuda":
        raise ValueError("band_sum needs a contiguous device float32 tensor")
    c, n = out.shape[-2], out.shape[-1]
    planes = out.numel() // (c * n)
    res = torch.empty(out.shape[:-2] + (n,), dtype=torch.float32, device=out.device)
    cdd_band_sum(out.data_ptr(), planes, c, n, res.data_ptr(),
                 torch.cuda.current_stream(out.device).cuda_stream)
    return res


def cdd_fullband_create(f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft=0, n_avg=1) -> int:
    h = ctypes.c_void_p()
    _check(_lib.cdd_fullband_create(ctypes.byref(h), float(f_center_mhz), float(bandwidth_mhz),
                                    int(n_chan), float(dm), int(n_fft), int(n_avg)),
           "cdd_fullband_create")
    return h.value


def cdd_fullband_set(plan: int, attr, value: int) -> None:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    _check(_lib.cdd_fullband_set(ctypes.c_void_p(plan), a, int(value)), "cdd_fullband_set")


def cdd_fullband_get(plan: int, attr) -> int:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    v = ctypes.c_int64()
    _check(_lib.cdd_fullband_get(ctypes.c_void_p(plan), a, ctypes.byref(v)), "cdd_fullband_get")
    return int(v.value)


def cdd_fullband_execute(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_fullband_execute(ctypes.c_void_p(plan), ctypes.c_void_p(d_in),
                                     ctypes.c_void_p(d_out), ctypes.c_void_p(stream)),
           "cdd_fullband_execute")


def cdd_fullband_reset(plan: int) -> None:
    _check(_lib.cdd_fullband_reset(ctypes.c_void_p(plan)), "cdd_fullband_reset")


def cdd_fullband_destroy(plan: int) -> None:
    _check(_lib.cdd_fullband_destroy(ctypes.c_void_p(plan)), "cdd_fullband_destroy")


def cdd_plan_commit(plan: int) -> None:
    _check(_lib.cdd_plan_commit(ctypes.c_void_p(plan)), "cdd_plan_commit")


def cdd_pool_create(hbm_budget_bytes: int, max_streams: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.cdd_pool_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_streams)),
           "cdd_pool_create")
    return h.value


def cdd_pool_admit(pool: int, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg,
                   segments_per_block, taper=0) -> int:
    sid = ctypes.c_int(-1)
    _check(_lib.cdd_pool_admit(ctypes.c_void_p(pool), float(f_center_mhz), float(bandwidth_mhz),
                               int(n_chan), float(dm), int(n_fft), int(n_avg),
                               int(segments_per_block), int(taper), ctypes.byref(sid)),
           "cdd_pool_admit")
    return sid.value


def cdd_pool_stream_get(pool: int, stream_id: int, attr) -> int:
    a = ATTR[attr] if isinstance(attr, str) else int(attr)
    v = ctypes.c_int64()
    _check(_lib.cdd_pool_stream_get(ctypes.c_void_p(pool), int(stream_id), a, ctypes.byref(v)),
           "cdd_pool_stream_get")
    return int(v.value)


def cdd_pool_submit(pool: int, stream_id: int, seq: int, d_in: int, d_out: int) -> int:
    t = ctypes.c_int64()
    _check(_lib.cdd_pool_submit(ctypes.c_void_p(pool), int(stream_id), int(seq),
                                ctypes.c_void_p(d_in), ctypes.c_void_p(d_out), ctypes.byref(t)),
           "cdd_pool_submit")
    return int(t.value)


def cdd_pool_wait(pool: int, ticket: int) -> float:
    lat = ctypes.c_double(-1.0)
    _check(_lib.cdd_pool_wait(ctypes.c_void_p(pool), int(ticket), ctypes.byref(lat)),
           "cdd_pool_wait")
    return float(lat.value)


def cdd_pool_release(pool: int, stream_id: int) -> None:
    _check(_lib.cdd_pool_release(ctypes.c_void_p(pool), int(stream_id)), "cdd_pool_release")


def cdd_pool_get(pool: int, attr) -> int:
    a = POOL_ATTR[attr] if isinstance(attr, str) else int(attr)
    v = ctypes.c_int64()
    _check(_lib.cdd_pool_get(ctypes.c_void_p(pool), a, ctypes.byref(v)), "cdd_pool_get")
    return int(v.value)


def cdd_pool_stream_export(pool: int, stream_id: int):
    """(state bytes, next sequence number) of an admitted stream."""
    n = ctypes.c_int64()
    _check(_lib.cdd_pool_stream_state_bytes(ctypes.c_void_p(pool), int(stream_id), ctypes.byref(n)),
           "cdd_pool_stream_state_bytes")
    buf = ctypes.create_string_buffer(n.value)
    seq = ctypes.c_int64()
    _check(_lib.cdd_pool_stream_export(ctypes.c_void_p(pool), int(stream_id), buf, n.value, ctypes.byref(seq)),
           "cdd_pool_stream_export")
    return buf.raw, seq.value


def cdd_pool_stream_import(pool: int, stream_id: int, state: bytes, next_seq: int) -> None:
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(_lib.cdd_pool_stream_import(ctypes.c_void_p(pool), int(stream_id), buf, len(state), int(next_seq)),
           "cdd_pool_stream_import")


def cdd_pool_destroy(pool: int) -> None:
    _check(_lib.cdd_pool_destroy(ctypes.c_void_p(pool)), "cdd_pool_destroy")


def cdd_execute_host_async(plan: int, h_in: int, h_out: int, stream: int = 0) -> None:
    _check(_lib.cdd_execute_host_async(ctypes.c_void_p(plan), ctypes.c_void_p(h_in),
                                       ctypes.c_void_p(h_out), ctypes.c_void_p(stream)),
           "cdd_execute_host_async")


def cdd_plan_prepare_host(plan: int) -> None:
    _check(_lib.cdd_plan_prepare_host(ctypes.c_void_p(plan)), "cdd_plan_prepare_host")


def cdd_pool_clock_ms() -> float:
    return float(_lib.cdd_pool_clock_ms())


def cdd_pool_admit_ex(pool: int, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg,
                      segments_per_block, taper, flags) -> int:
    sid = ctypes.c_int(-1)
    _check(_lib.cdd_pool_admit_ex(ctypes.c_void_p(pool), f_center_mhz, bandwidth_mhz, n_chan, dm,
                                  n_fft, n_avg, segments_per_block, taper, flags, ctypes.byref(sid)),
           "cdd_pool_admit_ex")
    return sid.value


def cdd_pool_request(pool: int, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg,
                     segments_per_block, taper, flags) -> int:
    req = ctypes.c_int64(0)
    _check(_lib.cdd_pool_request(ctypes.c_void_p(pool), f_center_mhz, bandwidth_mhz, n_chan, dm,
                                 n_fft, n_avg, segments_per_block, taper, flags, ctypes.byref(req)),
           "cdd_pool_request")
    return req.value


def cdd_pool_request_status(pool: int, request: int):
    """The admitted stream's id, or None while the request waits."""
    sid = ctypes.c_int(-1)
    rc = _lib.cdd_pool_request_status(ctypes.c_void_p(pool), request, ctypes.byref(sid))
    if rc == CDD_EBUSY:
        return None
    _check(rc, "cdd_pool_request_status")
    return sid.value


def cdd_pool_submit_at(pool: int, stream_id: int, seq: int, d_in: int, d_out: int,
                       t_arrival_ms: float) -> int:
    t = ctypes.c_int64(0)
    _check(_lib.cdd_pool_submit_at(ctypes.c_void_p(pool), stream_id, seq, ctypes.c_void_p(d_in),
                                   ctypes.c_void_p(d_out), t_arrival_ms, ctypes.byref(t)),
           "cdd_pool_submit_at")
    return t.value


def cdd_pool_submit_host(pool: int, stream_id: int, seq: int, h_in: int, h_out: int,
                         t_arrival_ms: float) -> int:
    t = ctypes.c_int64(0)
    _check(_lib.cdd_pool_submit_host(ctypes.c_void_p(pool), stream_id, seq, ctypes.c_void_p(h_in),
                                     ctypes.c_void_p(h_out), t_arrival_ms, ctypes.byref(t)),
           "cdd_pool_submit_host")
    return t.value


def cdd_pool_submit_many(pool: int, ids, seqs, ins, outs, arrivals=None, host=False):
    """Submit len(ids) blocks in one call; returns their tickets."""
    n = len(ids)
    c_ids = (ctypes.c_int * n)(*ids)
    c_seqs = (ctypes.c_int64 * n)(*seqs)
    c_ins = (ctypes.c_void_p * n)(*ins)
    c_outs = (ctypes.c_void_p * n)(*outs)
    c_arr = (ctypes.c_double * n)(*arrivals) if arrivals is not None else None
    tickets = (ctypes.c_int64 * n)()
    done = ctypes.c_int(0)
    rc = _lib.cdd_pool_submit_many(ctypes.c_void_p(pool), n, c_ids, c_seqs, c_ins, c_outs, c_arr,
                                   1 if host else 0, tickets, ctypes.byref(done))
    _check(rc, f"cdd_pool_submit_many (after {done.value} blocks)")
    return list(tickets)


def cdd_pool_stream_resync(pool: int, stream_id: int, seq: int) -> None:
    _check(_lib.cdd_pool_stream_resync(ctypes.c_void_p(pool), stream_id, seq), "cdd_pool_stream_resync")


# ------------------------------------------------------------------ convenience

class Plan:
    """Owning wrapper of one plan; tensors in, tensors out (no computation here)."""

    def __init__(self, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft=0, n_avg=1,
                 segments_per_block=1, taper="none", pipeline_chunks=None, polarisations=1,
                 stage_timing=False, precision="fp32", turn_tma=False):
        self.handle = cdd_plan_create(f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg)
        try:
            cdd_plan_set(self.handle, "segments_per_block", segments_per_block)
            if turn_tma:
                cdd_plan_set(self.handle, "turn_tma", 1)
            cdd_plan_set(self.handle, "taper", TAPER[taper])
            if precision != "fp32":
                cdd_plan_set(self.handle, "precision", PRECISION[precision])
            if stage_timing:
                cdd_plan_set(self.handle, "stage_timing", 1)
            if polarisations != 1:
                cdd_plan_set(self.handle, "polarisations", polarisations)
            if pipeline_chunks is not None:
                cdd_plan_set(self.handle, "pipeline_chunks", pipeline_chunks)
        except Exception:
            cdd_destroy(self.handle)
            raise
        self.n_chan = int(n_chan)

    def get(self, attr) -> int:
        return cdd_plan_get(self.handle, attr)

    @property
    def block_samples(self) -> int:
        return self.get("block_samples")

    @property
    def n_out(self) -> int:
        return self.get("n_out_per_block")

    def shifts(self):
        return cdd_plan_shifts(self.handle, self.n_chan)

    def export_state(self) -> bytes:
        """The stream's state after the blocks enqueued so far (waits for them)."""
        import torch
        return cdd_plan_export_state(self.handle, torch.cuda.current_stream().cuda_stream
                                     if torch.cuda.is_available() else 0)

    def import_state(self, state: bytes) -> None:
        """Continue the stream that `state` was exported from."""
        import torch
        cdd_plan_import_state(self.handle, state, torch.cuda.current_stream().cuda_stream
                              if torch.cuda.is_available() else 0)

    def _check_io(self, vin, out, device):
        import torch
        if vin.dtype != torch.int8 or tuple(vin.shape) != (self.block_samples, self.n_chan, 2):
            raise ValueError(f"input must be int8 [{self.block_samples}][{self.n_chan}][2]")
        if out.dtype != torch.float32 or tuple(out.shape) != (self.n_chan, self.n_out):
            raise ValueError(f"output must be float32 [{self.n_chan}][{self.n_out}]")
        for t in (vin, out):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
            if (t.device.type == "cuda") != device:
                raise ValueError("tensor on the wrong side of the host/device boundary")

    def execute(self, vin, out=None, volt=None):
        import torch
        if out is None:
            out = torch.empty((self.n_chan, self.n_out), dtype=torch.float32, device=vin.device)
        self._check_io(vin, out, device=True)
        stream = torch.cuda.current_stream(vin.device).cuda_stream
        if volt is None:
            cdd_execute(self.handle, vin.data_ptr(), out.data_ptr(), stream)
        else:
            if volt.dtype != torch.float32 or tuple(volt.shape) != (self.n_chan, self.block_samples, 2) \
                    or not volt.is_contiguous():
                raise ValueError("voltages must be contiguous float32 [C][block_samples][2]")
            cdd_execute_voltages(self.handle, vin.data_ptr(), out.data_ptr(), volt.data_ptr(), stream)
        return out

    def execute_host(self, vin, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.n_chan, self.n_out), dtype=torch.float32,
                              pin_memory=vin.is_pinned())
        self._check_io(vin, out, device=False)
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        cdd_execute_host(self.handle, vin.data_ptr(), out.data_ptr(), s)
        return out

    def execute_dual(self, vin_a, vin_b, out=None):
        import torch
        if out is None:
            out = torch.empty((self.n_chan, self.n_out), dtype=torch.float32, device=vin_a.device)
        self._check_io(vin_a, out, device=True)
        self._check_io(vin_b, out, device=True)
        cdd_execute_dual(self.handle, vin_a.data_ptr(), vin_b.data_ptr(), out.data_ptr(),
                         torch.cuda.current_stream(vin_a.device).cuda_stream)
        return out

    def reset(self):
        cdd_reset(self.handle)

    def close(self):
        if self.handle:
            cdd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owning wrapper of a batched (many-DM, tiered-N) plan."""

    def __init__(self, f_center_mhz, bandwidth_mhz, n_chan, dms, tier_nfft, n_avg,
                 segments_per_block=None, taper="none", form="tune"):
        self.handle = cdd_batch_create(f_center_mhz, bandwidth_mhz, n_chan, dms, tier_nfft, n_avg)
        try:
            if segments_per_block is not None:
                cdd_batch_set(self.handle, "segments_per_block", segments_per_block)
            if taper != "none":
                cdd_batch_set(self.handle, "taper", TAPER[taper])
            if form != "tune":
                cdd_batch_set(self.handle, "batch_form", BATCH_FORM[form])
        except Exception:
            cdd_batch_destroy(self.handle)
            raise
        self.n_chan, self.n_dm, self.n_tiers = int(n_chan), len(dms), len(tier_nfft)

    def get(self, attr) -> int:
        return cdd_batch_get(self.handle, attr)

    @property
    def block_samples(self) -> int:
        return self.get("block_samples")

    @property
    def n_out(self) -> int:
        return self.get("n_out_per_block")

    def tier(self, t):
        return cdd_batch_tier(self.handle, t)

    def shifts(self):
        return cdd_batch_shifts(self.handle, self.n_dm, self.n_chan)

    def export_state(self) -> bytes:
        """The stream state after the blocks executed so far (host bytes)."""
        import torch
        stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        return cdd_batch_export_state(self.handle, stream)

    def import_state(self, state: bytes) -> None:
        """Continue the stream an export_state() blob describes."""
        import torch
        stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        cdd_batch_import_state(self.handle, state, stream)

    def execute(self, vin, out=None):
        import torch
        if vin.dtype != torch.int8 or tuple(vin.shape) != (self.block_samples, self.n_chan, 2) \
                or not vin.is_contiguous() or vin.device.type != "cuda":
            raise ValueError(f"input must be contiguous device int8 [{self.block_samples}][{self.n_chan}][2]")
        if out is None:
            out = torch.empty((self.n_dm, self.n_chan, self.n_out), dtype=torch.float32, device=vin.device)
        if out.dtype != torch.float32 or tuple(out.shape) != (self.n_dm, self.n_chan, self.n_out) \
                or not out.is_contiguous() or out.device.type != "cuda":
            raise ValueError("output must be contiguous device float32 [n_dm][C][n_out]")
        cdd_batch_execute(self.handle, vin.data_ptr(), out.data_ptr(),
                          torch.cuda.current_stream(vin.device).cuda_stream)
        return out

    def reset(self):
        cdd_batch_reset(self.handle)

    def close(self):
        if self.handle:
            cdd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Fullband:
    """Owning wrapper of a full-band plan (the paper's own design)."""

    def __init__(self, f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft=0, n_avg=1,
                 segments_per_block=1):
        self.handle = cdd_fullband_create(f_center_mhz, bandwidth_mhz, n_chan, dm, n_fft, n_avg)
        try:
            cdd_fullband_set(self.handle, "segments_per_block", segments_per_block)
        except Exception:
            cdd_fullband_destroy(self.handle)
            raise
        self.n_chan = int(n_chan)

    def get(self, attr) -> int:
        return cdd_fullband_get(self.handle, attr)

    @property
    def frames(self) -> int:
        return self.get("block_samples")

    @property
    def n_out(self) -> int:
        return self.get("n_out_per_block")

    def execute(self, vin, out=None):
        import torch
        if vin.dtype != torch.int8 or tuple(vin.shape) != (self.frames, self.n_chan, 2) \
                or not vin.is_contiguous() or vin.device.type != "cuda":
            raise ValueError(f"input must be contiguous device int8 [{self.frames}][{self.n_chan}][2]")
        if out is None:
            out = torch.empty((self.n_out,), dtype=torch.float32, device=vin.device)
        if out.dtype != torch.float32 or tuple(out.shape) != (self.n_out,) or not out.is_contiguous():
            raise ValueError("output must be contiguous device float32 [n_out]")
        cdd_fullband_execute(self.handle, vin.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream(vin.device).cuda_stream)
        return out

    def reset(self):
        cdd_fullband_reset(self.handle)

    def close(self):
        if self.handle:
            cdd_fullband_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
