"""The float64 FMA-rate probe (ch_fp64_fma_rate) that the float64 kernels' ALU roofline quotes
beside the nominal rate (152 SMs x 2 FMA per clock x 2.07 GHz = 1.26 TFLOP/s)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_near_the_nominal_rate():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01322_gb300 import build
    build.build_library()
    from paper_2406_01322_gb300 import binding
    nominal = 152 * 2.07e9 * 4 / 1e12
    rate = binding.fp64_fma_rate()
    assert 0.3 * nominal < rate < 1.3 * nominal, rate
