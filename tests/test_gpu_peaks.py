"""The FP32 multiply-add microbenchmark (the non-tensor arithmetic ceiling of
the 16-bit storage modes) against the GB300's nominal rate."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_fma_peak_is_near_the_nominal_rate():
    from paper_2505_10171_gb300 import lbm
    nominal = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 FLOP x maximum SM clock
    tf = lbm.lbm_fp32_fma_peak()
    assert 0.5 * nominal < tf < 1.05 * nominal, tf
