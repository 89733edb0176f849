"""Host logic of bench.py's roofline model (no GPU), checked against counts made independently of
the model's formulas: operation counts of a radix-2 FFT run with counting arithmetic, a
brute-force enumeration of the tensor-core kernel's MMA tiles, and the DRAM traffic that ncu
measured for each kernel (the model's algorithmic bytes must be the compulsory traffic: neither
far above what the kernel moved, which would flatter the roofline, nor far below it)."""
import math

import pytest

import bench
from paper_2406_01322_gb300 import inputs

W = inputs.WORKLOADS["channel_128x128x129"]


class Counted:
    """A complex number whose real operations are counted (adds and multiplies)."""
    ops = 0

    def __init__(self, re, im):
        self.re, self.im = re, im

    def __add__(self, o):
        Counted.ops += 2
        return Counted(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        Counted.ops += 2
        return Counted(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        Counted.ops += 6
        return Counted(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)


def radix2_fft(x):
    """Textbook recursive radix-2 decimation in time, every twiddle product carried out."""
    n = len(x)
    if n == 1:
        return x
    ev, od = radix2_fft(x[0::2]), radix2_fft(x[1::2])
    out = [None] * n
    for k in range(n // 2):
        w = Counted(math.cos(-2 * math.pi * k / n), math.sin(-2 * math.pi * k / n))
        t = w * od[k]
        out[k] = ev[k] + t
        out[k + n // 2] = ev[k] - t
    return out


@pytest.mark.parametrize("n", [8, 64, 256])
def test_fft_flop_convention_is_the_radix2_operation_count(n):
    """bench.fft_flops is the conventional 5 n log2 n: the real operations of a radix-2 FFT."""
    Counted.ops = 0
    radix2_fft([Counted(float(i), 0.0) for i in range(n)])
    assert bench.fft_flops(n) == Counted.ops


def test_dct_line_counts_one_n_point_fft():
    """The z kernels count one N-point complex FFT per Chebyshev line (N = nz - 1), the FFT of
    the N-point DCT-I; the tensor-core method drops exactly those from zrhs and zbwd."""
    fft, tc = bench.kernel_work(W, 0, "fft"), bench.kernel_work(W, 0, "tc")
    lines = (W["nx"] // 2) * W["ny"]
    Counted.ops = 0
    radix2_fft([Counted(0.0, 0.0) for _ in range(W["nz"] - 1)])
    per_dct = Counted.ops
    assert fft["zrhs"][0] - tc["zrhs"][0] == pytest.approx(7 * lines * per_dct)
    assert fft["zbwd"][0] - tc["zbwd"][0] == pytest.approx(5 * lines * per_dct)


def test_tensor_core_flops_match_an_enumeration_of_the_mma_tiles():
    """Enumerate the kernel's MMAs: per tile of 128 rows, per output slice of NT columns, per K
    chunk of 144 (the last one shorter), A plane i (0..7) against the (8 - i) stacked B planes,
    in K steps of 16: 2 * 128 * ((8 - i) NT) * 16 flops each."""
    for nz in (65, 129, 257):
        w = dict(W, nz=nz)
        Kp, NT, nNt = bench.tc_tiles(nz)
        rows = 2 * (w["nx"] // 2) * w["ny"]
        tiles = 7 * rows // 128
        per_tile = 0
        for _ in range(nNt):
            k0 = 0
            while k0 < Kp:
                kc = min(144, Kp - k0)
                for i in range(8):
                    per_tile += (kc // 16) * 2 * 128 * (8 - i) * NT * 16
                k0 += kc
        assert bench.kernel_work(w, 0)["cheb_fwd"][0] == pytest.approx(tiles * per_tile)


L2_BYTES = 129e6

# Re-reads that the design has, and their bounds.  The tensor-core transform writes a per-CTA
# cache of the digit planes' 7-bit groups and reads it back for each later output slice; at
# 512 x 256 x 257 part of it leaves L2 (1.2x / 1.3x the compulsory bytes, bound 1.5x).
# The global-memory tau sweeps of long lines (N > 128) read and write each line once per sweep
# and read the tabulated factors (5.2x, bound 6x).
# The persistent float32 x line deals items (pairs of z rows) round-robin to its CTAs; two
# neighbouring items share each 32-byte sector of their rows, and CTAs that drift apart find the
# other half gone from L2 (1.28x, bound 1.4x; contiguous runs per CTA keep it in L2 but scatter
# the CTAs over DRAM pages and take twice as long).
REREAD_BOUND = {("channel_512x256x257_mixed", 1, "xline"): 1.4,
                ("channel_512x256x257_mixed", 1, "cheb_fwd"): 1.5,
                ("channel_512x256x257_mixed", 1, "cheb_bwd"): 1.5,
                ("channel_512x256x257_mixed", 1, "zsolve"): 6.0,
                ("channel_512x256x257_mixed", 0, "zsolve"): 6.0}


@pytest.mark.parametrize("key", sorted(bench.TRAFFIC_MB))
def test_algorithmic_bytes_are_the_measured_compulsory_traffic(key):
    """For every kernel whose DRAM traffic ncu measured, the model's bytes per launch (the fields
    the kernel must read and write once) bound the measurement: it can be lower only by what the
    129 MB L2 holds across the launch boundary (inputs the previous kernel left there, outputs
    not yet written back when the launch ends), and higher only by re-reads, which the fused
    design keeps under a quarter except where REREAD_BOUND states its structural re-reads."""
    workload, prec, kernel = key
    name = workload.split("@")[0]
    w = dict(inputs.WORKLOADS[name])
    if "@" in workload:
        nx, ny, nz = (int(v) for v in workload.split("@")[1].split("x"))
        w.update(nx=nx, ny=ny, nz=nz)
    cheb = "fft"
    k = kernel
    if kernel.endswith("_coef"):
        cheb, k = "tc", kernel[:-5]
    if name.endswith("_adjoint"):
        model = bench.adjoint_work(w)[k][1]
    else:
        model = bench.kernel_work(w, prec, cheb)[k][1]
    measured = bench.TRAFFIC_MB[key] * 1e6
    assert model - L2_BYTES <= measured <= REREAD_BOUND.get(key, 1.25) * model, \
        (key, model / 1e6, measured / 1e6)


def test_traffic_lookup_separates_the_coefficient_kernels():
    wl = "channel_512x256x257_mixed"
    fft = bench.traffic_bytes(wl, 1, "zbwd")
    tc = bench.traffic_bytes(wl, 1, "zbwd", "tc")
    assert fft is not None and tc is not None and fft != tc
    assert bench.traffic_bytes(wl, 0, "xline", "tc") == bench.traffic_bytes(wl, 0, "xline")
    assert bench.traffic_bytes(wl, 0, "no_such_kernel") is None


def test_alu_peak_follows_the_unit_counts_and_clock():
    # float64: 152 SMs x 2 DFMA (4 flops) per clock at the 2.07 GHz maximum SM clock
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 4 * 2.07e9 / 1e12)
    assert 0 < bench.DF_PEAK_TFLOPS < 152 * 128 * 2 * 2.07e9 / 1e12
