"""Measured FMA throughput of the CUDA cores (the ALU roofline of the plain
FP32 and FP64 paths) is positive and below the unit-count bound."""

import pytest

from tests.libutil import ensure_built


@pytest.mark.gpu
def test_fma_peak_is_plausible():
    ensure_built()
    from paper_1312_1638_b300 import fr
    f32, f64 = fr.fma_peak(0)
    nominal32 = 148 * 128 * 2 * 2.032e9 / 1e12          # SMs x FP32 lanes x 2 flop x max clock
    assert 0.3 * nominal32 < f32 < 1.05 * nominal32, f32
    assert 0.0 < f64 < f32, (f32, f64)
