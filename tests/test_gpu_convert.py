"""The library's FP64 <-> FP32 conversions (used by the precision casts of the
mixed-precision V-cycle, computed on the integer pipe) against the hardware
conversions, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2007_00056_gb300 import amg

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(11)
    n = 1 << 20
    # magnitudes across and beyond the FP32 range, both signs
    e = rng.uniform(-160.0, 140.0, n)
    x = np.sign(rng.uniform(-1, 1, n)) * rng.uniform(1.0, 2.0, n) * np.exp2(e)
    f = np.float32
    specials = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324,
                float(np.finfo(f).max), -float(np.finfo(f).max), float(np.finfo(f).tiny),
                float(np.finfo(f).tiny) * (1 - 2**-30), float(np.finfo(f).max) * (1 + 2**-25),
                float(np.finfo(f).max) * (1 + 2**-24), 1.0 + 2**-24, 1.0 + 3 * 2**-24, 1.0 - 2**-25,
                -(1.0 + 2**-24), 2**-126 * (1 + 2**-23), 1e-45, 3.0e38, 1.0 / 3.0]
    # exact halfway points between adjacent floats: ties go to the even mantissa
    base = rng.uniform(1.0, 2.0, 4096).astype(f).astype(np.float64)
    ulp = np.spacing(base.astype(f)).astype(np.float64)
    ties = base + ulp / 2
    return np.concatenate([x, np.array(specials), ties, -ties])


def test_conversions_match_hardware_bitwise():
    x = torch.from_numpy(_cases()).cuda()
    f32, f64 = amg.amg_selftest_convert(x)
    ref32 = x.float()
    ref64 = ref32.double()
    np.testing.assert_array_equal(f32.cpu().numpy().view(np.int32), ref32.cpu().numpy().view(np.int32))
    np.testing.assert_array_equal(f64.cpu().numpy().view(np.int64), ref64.cpu().numpy().view(np.int64))
