"""cdd_execute_static, the entry point that allocates no device memory.

Some callers cannot call cudaMalloc (real-time loops that may only allocate at
start-up, processes whose device memory belongs to another allocator or to a
fixed budget).  For them the library offers cdd_execute_static, which keeps all
of its scratch in one fixed device array compiled into the library.  This file
checks it through the C ABI against the plan-based entry point (cdd_plan_create
+ cdd_execute on a fresh plan) and against the FP64 oracle, on consecutive
calls that leave different tables in the shared array, and checks that calls
after the first on a device take no device memory.  The file name makes
pytest collect it last.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-5          # the relative RMS bound the parity tests use


def _input(seed, rows, n_chan):
    rng = np.random.default_rng(seed)
    return np.clip(np.rint(rng.normal(0, 20, (rows, n_chan, 2))), -127, 127).astype(np.int8)


def _plan_output(x, args, n_seg, taper):
    from paper_1509_00186_b300.cdd import Plan
    with Plan(*args, segments_per_block=n_seg, taper=taper) as plan:
        out = plan.execute(x)
    return out


def _static_output(x, args, n_seg, taper):
    import torch
    from paper_1509_00186_b300 import cdd
    f_c, bw, n_chan, dm, n_fft, n_avg = args
    geo = O.plan_geometry(*args)
    out = torch.full((n_chan, n_seg * geo.hop // n_avg), float("nan"), device=x.device)
    cdd.cdd_execute_static(f_c, bw, n_chan, dm, n_fft, n_avg, n_seg, cdd.TAPER[taper],
                           x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out


def test_static_entry_matches_plan_entry_on_consecutive_calls(cuda_device):
    import torch
    cases = [
        # (band args, segments, taper): a 64-channel cut of the 32 MHz / N 8192
        # shape, then a small-N shape with a taper, then the first one again
        ((309.0 + 2.0, 4.0, 64, 50.0, 8192, 16), 3, "none"),
        ((317.0 + 1.0, 2.0, 32, 10.0, 64, 4), 40, "hann"),
        ((309.0 + 2.0, 4.0, 64, 50.0, 8192, 16), 3, "none"),
    ]
    for i, (args, n_seg, taper) in enumerate(cases):
        geo = O.plan_geometry(*args)
        x = torch.from_numpy(_input(100 + (i % 2), n_seg * geo.hop, args[2])).to(cuda_device)
        got = _static_output(x, args, n_seg, taper)
        want = _plan_output(x, args, n_seg, taper)
        torch.cuda.synchronize()
        got, want = got.cpu().numpy(), want.cpu().numpy()
        assert np.all(np.isfinite(got)), i
        assert O.rel_rms(got, want) <= TOL, i
        # the oracle: one block of a fresh stream (zero history)
        oracle_out = O.dedisperse(x.cpu().numpy(), geo, taper)
        assert oracle_out.shape == got.shape
        assert O.rel_rms(got, oracle_out) <= TOL, i


def test_static_entry_takes_no_device_memory_after_the_first_call(cuda_device):
    """After one call on the device (which may load the library's device code
    and with it the fixed array), further calls leave the device's free memory
    and torch's allocations unchanged."""
    import torch
    args, n_seg, taper = (309.0 + 2.0, 4.0, 64, 50.0, 8192, 16), 3, "none"
    geo = O.plan_geometry(*args)
    x = torch.from_numpy(_input(7, n_seg * geo.hop, args[2])).to(cuda_device)
    first = _static_output(x, args, n_seg, taper)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    outs = [_static_output(x, args, n_seg, taper) for _ in range(2)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    del outs                            # the outputs were torch's own, made before each call
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 >= free0 - 2 * first.numel() * 4 - (4 << 20)   # no new device memory but the outputs
    again = _static_output(x, args, n_seg, taper)
    torch.cuda.synchronize()
    assert torch.equal(again, first)
