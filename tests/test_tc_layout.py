"""Host check of the tensor-core form of the N = 8192 transform (CPU).

tests/tc_emulator.cpp replays the kernel's data flow for one segment with the
operand layouts, matrix descriptors and index maps of
csrc/cdd_tc_layout.h: operands written into an image of shared memory, each
tcgen05 product decoded from its descriptors by the canonical K-major
no-swizzle rule, FP32 accumulation, and the moves between passes.  Its
voltages are compared with the direct definition y = IDFT(DFT(x) c) / N in
FP64.  A wrong descriptor field, layout offset, index map, twiddle, chirp
position, conjugation or scale gives an error of order one; the bounds below
are the rounding of each operand form (hi + lo FP16 keeps about 22 bits, BF16
16; FP16 alone 11, BF16 8) with a factor of about two of margin.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tc_emulator.cpp")

BOUNDS = {"fp16x2": 3e-6, "bf16x2": 1.5e-5, "fp16": 1.5e-3, "bf16": 1.2e-2}


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("tc") / "tc_emulator")
    subprocess.run([gxx, "-O2", "-std=c++17", "-o", exe, SRC], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("precision", sorted(BOUNDS))
def test_tensor_core_transform_on_host(emulator, precision):
    res = subprocess.run([emulator, precision], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    err = float(res.stdout.split()[1])
    assert err <= BOUNDS[precision], f"{precision}: relative RMS {err:.3e}"
    # the split forms must be far more accurate than the plain ones
    if precision.endswith("x2"):
        assert err <= 2e-5
