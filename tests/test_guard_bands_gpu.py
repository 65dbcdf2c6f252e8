"""Guard bands around every output (GPU).

Each output of an entry point is a view into a larger device buffer.  The
buffer is first filled with a NaN bit pattern: the output itself and a guard
region on either side.  After the call the guards must hold the pattern bit for
bit, so no kernel wrote outside its output.  The output must hold no NaN, so
every element was written.  The shapes cover ragged tiles, the cluster and
tensor-core kernels, the tensor-copy corner turn, the batched tiers and the
full band's tile passes.
"""
import numpy as np
import pytest

from synth import complex_int8_voltages

pytestmark = pytest.mark.gpu
GUARD = 16384                      # floats on each side
PATTERN = 0x7FC0DEAD               # a quiet NaN with a payload


class Guarded:
    def __init__(self, shape):
        import torch
        self.n = int(np.prod(shape))
        self.raw = torch.full((self.n + 2 * GUARD,), PATTERN, dtype=torch.int32, device="cuda")
        self.view = self.raw.view(torch.float32)[GUARD:GUARD + self.n].view(*shape)

    def check(self):
        import torch
        torch.cuda.synchronize()
        raw = self.raw.cpu().numpy()
        assert np.all(raw[:GUARD] == PATTERN), "write before the output"
        assert np.all(raw[GUARD + self.n:] == PATTERN), "write after the output"
        out = self.view.cpu().numpy()
        assert not np.isnan(out).any(), "output element left unwritten"
        return out


@pytest.mark.parametrize("args, q, kw", [
    ((325.0, 4.0, 64, 50.0, 8192, 16), 3, {}),                       # N 8192, persistent kernel
    ((325.0, 2.3125, 37, 10.0, 512, 4), 5, {}),                      # ragged channels
    ((150.0, 4.0, 64, 100.0, 65536, 16), 1, {}),                     # cluster of eight
    ((325.0, 4.5, 72, 10.0, 1024, 8), 3, {"turn_tma": True}),        # tensor-copy corner turn
    ((325.0, 4.0, 64, 50.0, 8192, 16), 2, {"precision": "fp16x2"}),  # tensor-core form
])
def test_plan_outputs_and_voltages_stay_in_bounds(cuda_device, args, q, kw):
    import torch
    from paper_1509_00186_b300.cdd import Plan
    with Plan(*args, segments_per_block=q, **kw) as plan:
        bs, n_out, C = plan.block_samples, plan.n_out, plan.n_chan
        vin = torch.from_numpy(complex_int8_voltages(3, bs, C, 20.0)).cuda()
        out = Guarded((C, n_out))
        volt = Guarded((C, bs, 2))
        plan.execute(vin, out.view, volt.view)
        out.check()
        volt.check()
        assert plan.get("device_errors") == 0


def test_batch_output_stays_in_bounds(cuda_device):
    import torch
    from paper_1509_00186_b300.cdd import Batch
    args = (650.0, 0.78125, 8, [20.0, 30.0, 35.0, 40.0], (16384, 8192, 4096, 2048), 16)
    with Batch(*args, segments_per_block=2) as b:
        vin = torch.from_numpy(complex_int8_voltages(4, b.block_samples, b.n_chan, 20.0)).cuda()
        out = Guarded((b.n_dm, b.n_chan, b.n_out))
        b.execute(vin, out.view)
        out.check()


@pytest.mark.parametrize("args", [
    (610.0, 1.0, 32, 20.0, 0, 4),            # the shared-memory transform only
    (325.0, 2.0, 64, 5.0, 1 << 20, 8),       # a radix-128 tile pass, windows fused
    (325.0, 2.0, 64, 5.0, 1 << 21, 64),      # radix 64 then 4, the integration kernel
])
def test_fullband_output_stays_in_bounds(cuda_device, args):
    import torch
    from paper_1509_00186_b300.cdd import Fullband
    with Fullband(*args, segments_per_block=2) as f:
        vin = torch.from_numpy(complex_int8_voltages(5, f.frames, args[2], 20.0)).cuda()
        out = Guarded((f.n_out,))
        f.execute(vin, out.view)
        out.check()


def test_band_sum_output_stays_in_bounds(cuda_device):
    import torch
    from paper_1509_00186_b300 import cdd
    x = torch.rand((3, 37, 1001), device="cuda")
    res = Guarded((3, 1001))
    cdd.cdd_band_sum(x.data_ptr(), 3, 37, 1001, res.view.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = res.check()
    assert np.allclose(got, x.sum(1).cpu().numpy(), rtol=1e-5, atol=1e-5)
