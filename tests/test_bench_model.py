"""Host logic of bench.py's roofline model (no GPU): the algorithmic work per launch of each step
kernel, the tensor-core method's coefficient-space z kernels, the DRAM-traffic lookup and the
ALU peaks the fractions divide by."""
import math

import pytest

import bench
from paper_2406_01322_gb300 import inputs

W = inputs.WORKLOADS["channel_128x128x129"]


def test_fft_method_counts_one_n_point_fft_per_dct_line():
    kernel = bench.kernel_work(W, 0)
    nx, ny, nz = W["nx"], W["ny"], W["nz"]
    lines, N = (nx // 2) * ny, nz - 1
    dct = 5 * N * math.log2(N)
    assert kernel["zrhs"][0] == pytest.approx(lines * (7 * dct + 9 * 4 * nz + 150 * nz))
    assert kernel["zbwd"][0] == pytest.approx(lines * (5 * dct + 2 * 4 * nz + 40 * nz))
    # eight entries: the six kernels of the FFT method and the two tensor-core transforms
    assert set(kernel) == {"zrhs", "zsolve", "zbwd", "ybwd", "xline", "yfwd", "cheb_fwd", "cheb_bwd"}


def test_tensor_core_method_drops_the_dcts_from_the_z_kernels():
    fft, tc = bench.kernel_work(W, 1, "fft"), bench.kernel_work(W, 1, "tc")
    nx, ny, nz = W["nx"], W["ny"], W["nz"]
    lines, S = (nx // 2) * ny, (nx // 2) * ny * nz
    assert tc["zrhs"][0] == pytest.approx(lines * (9 * 4 + 150) * nz)
    assert tc["zbwd"][0] == pytest.approx(lines * (2 * 4 + 40) * nz)
    assert tc["zrhs"][0] < fft["zrhs"][0] and tc["zbwd"][0] < fft["zbwd"][0]
    # the coefficients are float64 whatever the working precision: 9 fields of 16 bytes in
    assert tc["zrhs"][1] - fft["zrhs"][1] == S * 9 * (16 - 8)
    for k in ("zsolve", "ybwd", "xline", "yfwd", "cheb_fwd", "cheb_bwd"):
        assert tc[k] == fft[k]


def test_tensor_core_flops_follow_the_padded_tiles():
    Kp, NT, nNt = bench.tc_tiles(W["nz"])
    assert Kp % 16 == 0 and Kp >= W["nz"] and NT * nNt <= 512
    # the kernel sums the last output exactly on the producers; the slices cover n < N
    assert NT * nNt >= W["nz"] - 1
    rows = 2 * (W["nx"] // 2) * W["ny"]
    f = bench.kernel_work(W, 0)
    assert f["cheb_fwd"][0] == pytest.approx(36 * 2.0 * 9 * rows * NT * nNt * Kp)
    assert f["cheb_bwd"][0] == pytest.approx(f["cheb_fwd"][0] * 5 / 9)


def test_traffic_lookup_separates_the_coefficient_kernels():
    wl = "channel_128x128x129"
    fft = bench.traffic_bytes(wl, 1, "zrhs")
    tc = bench.traffic_bytes(wl, 1, "zrhs", "tc")
    assert fft is not None and tc is not None and fft != tc
    assert bench.traffic_bytes(wl, 0, "xline", "tc") == bench.traffic_bytes(wl, 0, "xline")
    assert bench.traffic_bytes(wl, 0, "no_such_kernel") is None
    assert bench.traffic_bytes("channel_512x256x257_mixed", 1, "zrhs") is None


def test_alu_peaks_follow_the_unit_counts_and_clock():
    # float64: 152 SMs x 2 DFMA (4 flops) per clock at 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 4 * 2.07e9 / 1e12)
    # double-float: float32 lanes / float32 instructions per float64-equivalent flop, with the
    # instruction mix of the transforms (10.2 M adds at 11, 5.4 M FMAs at 18 per 2 flops,
    # 2.4 M multiplications at 7)
    per_flop = (10.2 * 11 + 5.4 * 18 + 2.4 * 7) / (10.2 + 2 * 5.4 + 2.4)
    assert per_flop == pytest.approx(9.67, abs=0.01)
    assert bench.DF_PEAK_TFLOPS == pytest.approx(152 * 128 * 2.07e9 / 9.67 / 1e12)
    assert 0 < bench.DF_PEAK_TFLOPS < 152 * 128 * 2 * 2.07e9 / 1e12
