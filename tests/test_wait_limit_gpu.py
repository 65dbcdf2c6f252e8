"""The kernels' bounded waits (GPU).

Every spin-wait in the library's kernels gives up after a limit, sets the
plan's error flag and returns, so a wait that can never be met does not hang
the device.  The self-test entry runs the tensor-copy corner turn on one
tile whose mbarrier expects more bytes than the copy brings: its wait must
run out (flag bit 2), its bounded clean-up wait must end too, and the device
must still run a plan afterwards, bit for bit as before.
"""
import numpy as np
import pytest

from synth import complex_int8_voltages

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_device_stays_usable(cuda_device):
    import time
    import torch
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.cdd import Plan
    args = (325.0, 4.0, 64, 10.0, 1024, 8)

    def run():
        with Plan(*args, segments_per_block=3, turn_tma=True) as plan:
            vin = complex_int8_voltages(5, plan.block_samples, plan.n_chan, 20.0)
            out = plan.execute(torch.from_numpy(vin).cuda())
            torch.cuda.synchronize()
            assert plan.get("device_errors") == 0
            return out.cpu().numpy()

    before = run()
    t0 = time.monotonic()
    status = cdd.cdd_selftest_wait_limit()
    dt = time.monotonic() - t0
    assert status == 2
    assert dt < 5.0                       # two 20 ms waits, not a hang
    after = run()
    assert np.array_equal(before, after)
