"""The Chebyshev transform on the tensor cores (CH_CHEB_TC) against the oracle.

Line transforms: every line of seeded complex data (plus rows chosen to stress the exact split:
zero, a single sample, tiny and huge magnitudes, a 32-decade spread, alternating signs) is
compared with the oracle's transform matrices (Sec. 3.2.1) evaluated in extended precision.
Bound per line for the tensor-core method: |error| <= 1e-15 max|x| max_n sum_k |B_nk| (a few
float64 roundings of the row-times-matrix scale: the split keeps 2^-55 of the row and matrix
scales and drops products below 2^-53) plus 1e-321 for results in the subnormal range.  The FFT
method is held to 2e-16 N of the same scale (its odd outputs are N/2-term prefix sums).  Sizes
cover one and two K chunks (nz = 257), both output slice widths (48 and 64) and a ragged last
tile of lines (24 x 24: 288 lines = 4.5 tiles of 64).

Steps: the step with CH_CHEB_TC meets the float64 bar against the oracle (1e-10 after 10 steps),
the mixed-precision bound against the float64 path, and agrees with the FFT method.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import chebyshev as ocheb  # noqa: E402
from oracle.channel import Channel, Params  # noqa: E402
from paper_2406_01322_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01322_gb300 import build
    build.build_library()
    from paper_2406_01322_gb300 import binding as b
    b.lib()
    return b


def matrices_ld(N):
    """The oracle's forward / backward matrices re-evaluated in numpy long double."""
    ld = np.longdouble
    n = np.arange(N + 1)
    a = (n[:, None] * n[None, :]) % (2 * N)
    pi = np.arccos(ld(-1))
    B = np.cos(np.asarray(a, dtype=ld) * pi / ld(N))
    cb = np.ones(N + 1, dtype=ld)
    cb[0] = cb[N] = 2
    F = 2 / (cb[:, None] * N) * B.T / cb[None, :]
    return F, B


def test_long_double_matrices_are_the_oracle_matrices():
    """Pin of the extended-precision reference: it agrees with the oracle's float64 matrices to
    the rounding of the oracle's own float64 cosine arguments (a few ulps of 1)."""
    for N in (32, 48, 128):
        F, B = matrices_ld(N)
        assert np.max(np.abs(F.astype(np.float64) - ocheb.forward_matrix(N))) <= 1e-15
        assert np.max(np.abs(B.astype(np.float64) - ocheb.backward_matrix(N))) <= 1e-15


def line_data(Mx, ny, nz, seed):
    """(1, Mx, ny, nz) complex128: seeded normal lines with special rows in the first lines."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((Mx, ny, nz)) + 1j * rng.standard_normal((Mx, ny, nz))
    flat = x.reshape(-1, nz)
    k = np.arange(nz)
    flat[0] = 0.0                                        # all zero
    flat[1] = 0.0
    flat[1, nz // 3] = 3.0 - 2.0j                        # one sample
    flat[2] *= 1e-300                                    # tiny row
    flat[3] *= 1e300                                     # huge row
    flat[4] = 10.0 ** (-k / 4.0) * (1 + 1j)              # 1 .. 1e-(nz/4) spread
    flat[5] = np.where(k % 2 == 0, 1.0, -1.0) * (1 - 0.5j)   # alternating signs
    flat[6] = (1.0 - 2.0 ** -52) * (1 + 1j)              # just below a power of two
    flat[7] = 2.0 ** -1074 * (k % 3)                     # subnormals
    return x[None]


SIZES = [(32, 32, 33), (24, 24, 49), (32, 32, 65), (32, 32, 97), (32, 32, 129), (16, 16, 257)]


@pytest.mark.parametrize("nx,ny,nz", SIZES)
@pytest.mark.parametrize("method", [0, 1], ids=["fft", "tc"])
def test_lines_match_extended_precision_transform(binding, nx, ny, nz, method):
    N = nz - 1
    g = binding.Grid(nx, ny, nz)
    g.set_chebyshev(method)
    x = line_data(nx // 2, ny, nz, seed=100 + nz)
    xt = torch.from_numpy(x).cuda()
    F, B = matrices_ld(N)
    flat = x.reshape(-1, nz)
    for direction, M in ((0, F), (1, B)):
        got = g.chebyshev_lines(xt, direction).cpu().numpy().reshape(-1, nz)
        g.device_status()
        rowsum = float(np.max(np.sum(np.abs(M), axis=1)))
        for part in (np.real, np.imag):
            xr = part(flat).astype(np.longdouble)
            ref = xr @ M.T
            err = np.abs(part(got).astype(np.longdouble) - ref)
            scale = np.max(np.abs(xr), axis=1) * rowsum
            coef = 1e-15 if method == 1 else max(1e-15, 2e-16 * N)
            bound = coef * scale[:, None] + 1e-321
            bad = np.argwhere(err > bound)
            assert bad.size == 0, (direction, bad[:5], float(np.max(err / np.maximum(bound, 1e-320))))


def test_round_trip_and_agreement_with_fft(binding):
    nx, ny, nz = 32, 32, 129
    x = torch.from_numpy(line_data(nx // 2, ny, nz, seed=7)).cuda()
    gt = binding.Grid(nx, ny, nz)
    gt.set_chebyshev(binding.CHEB_TC)
    gf = binding.Grid(nx, ny, nz)
    a_tc = gt.chebyshev_lines(x, 0)
    a_fft = gf.chebyshev_lines(x, 0)
    back = gt.chebyshev_lines(a_tc, 1)
    xs = x.reshape(-1, nz)
    scale = torch.amax(torch.abs(xs), dim=1, keepdim=True).clamp_min(1e-300)
    assert float(torch.max(torch.abs(back.reshape(-1, nz) - xs) / scale)) < 1e-13
    d = torch.abs(a_tc - a_fft).reshape(-1, nz) / scale
    assert float(torch.max(d)) < 1e-14


def test_non_finite_row_gives_nan_row_only(binding):
    nx, ny, nz = 16, 16, 33
    g = binding.Grid(nx, ny, nz)
    g.set_chebyshev(binding.CHEB_TC)
    x = line_data(nx // 2, ny, nz, seed=3)
    x.reshape(-1, nz)[10, 4] = complex(np.nan, 1.0)     # NaN in the real row of line 10
    out = g.chebyshev_lines(torch.from_numpy(x).cuda(), 0).cpu().numpy().reshape(-1, nz)
    assert np.all(np.isnan(out[10].real))
    assert np.all(np.isfinite(out[10].imag))
    others = np.delete(out, 10, axis=0)
    assert np.all(np.isfinite(others))


def workload(name, **over):
    w = dict(inputs.WORKLOADS[name])
    w.update(over)
    return w


def phys_kw(w):
    return dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def grid(binding, w, fields, precision=0, method=1):
    g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=precision, **phys_kw(w))
    g.set_chebyshev(method)
    g.set_fields(*[torch.from_numpy(f) for f in fields])
    return g


@pytest.mark.parametrize("over", [{}, dict(nx=16, ny=16, nz=257)], ids=["33", "257"])
def test_ten_steps_fp64_tc_within_1e_10(binding, over):
    w = workload("channel_32x32x33", **over)
    fields = inputs.initial_fields(**w)
    g = grid(binding, w, fields)
    o = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], **phys_kw(w)))
    o.set_fields(*fields)
    g.step(10)
    for _ in range(10):
        o.step()
    g.device_status()
    tol = 1e-10 * max(1.0, ((w["nz"] - 1) / 128) ** 2)   # the long-line scaling of the FFT path
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= tol, f


@pytest.mark.parametrize("bc", [1, 2, 3], ids=["free-slip", "no-slip-bottom", "free-slip-bottom"])
def test_walls_tc_ten_steps_within_1e_10(binding, bc):
    """The coefficient-space zrhs / zbwd with every wall closure of the tau solves."""
    w = workload("channel_32x32x33", bc=bc)
    fields = inputs.initial_fields(**w)
    g = binding.Grid(w["nx"], w["ny"], w["nz"], bc=bc, **phys_kw(w))
    g.set_chebyshev(binding.CHEB_TC)
    g.set_fields(*[torch.from_numpy(f) for f in fields])
    o = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], bc=bc, **phys_kw(w)))
    o.set_fields(*fields)
    g.step(10)
    for _ in range(10):
        o.step()
    g.device_status()
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f


def test_mixed_tc_error_bound_and_fft_agreement(binding):
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    g64 = grid(binding, w, fields, 0, 0)
    g32t = grid(binding, w, fields, 1, 1)
    g32f = grid(binding, w, fields, 1, 0)
    for g in (g64, g32t, g32f):
        g.step(10)
    for a, b, c, f in zip(g32t.get_fields(), g64.get_fields(), g32f.get_fields(), "uvwp"):
        a, b, c = (t.cpu().numpy() for t in (a, b, c))
        assert rel(a, b) < 1e-4, f
        # float32 products dominate; the two transform methods differ far below that
        assert rel(a, c) < 1e-6, f
    d_t, d_64 = g32t.diagnostics(), g64.diagnostics()
    assert abs(d_t["mass"] - d_64["mass"]) <= 1e-6 * abs(d_64["mass"])


def test_medium_channel_tc_agrees_with_fft(binding):
    w = workload("channel_128x128x129")
    fields = inputs.initial_fields(**w)
    gt = grid(binding, w, fields, 0, 1)
    gf = grid(binding, w, fields, 0, 0)
    gt.step(3)
    gf.step(3)
    for a, b, f in zip(gt.get_fields(), gf.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-11, f


def test_timed_step_with_tc(binding):
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    g1 = grid(binding, w, fields)
    g2 = grid(binding, w, fields)
    assert g1.launches_per_step() == 8
    tot, ks = g1.step_timed(3)
    assert len(ks) == len(binding.Grid.KERNELS) == 8
    assert ks[6] > 0 and ks[7] > 0 and sum(ks) <= tot * 1.01 + 1e-3
    g2.step(3)
    for a, b in zip(g1.get_fields(), g2.get_fields()):
        assert torch.equal(a, b)


def test_switching_methods_mid_run(binding):
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    g = grid(binding, w, fields, 0, 0)
    r = grid(binding, w, fields, 0, 0)
    g.step(2)
    g.set_chebyshev(binding.CHEB_TC)
    g.step(2)
    g.set_chebyshev(binding.CHEB_FFT)
    g.step(2)
    r.step(6)
    assert g.chebyshev() == binding.CHEB_FFT
    for a, b in zip(g.get_fields(), r.get_fields()):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12


def test_dfloat_tc_ten_steps_within_1e_10(binding):
    """Double-float x/y with the tensor-core transforms (double-float rows in, double-float
    samples out) against the float64 oracle, and against the double-float FFT path."""
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    g = grid(binding, w, fields, binding.PREC_DFLOAT, binding.CHEB_TC)
    gf = grid(binding, w, fields, binding.PREC_DFLOAT, binding.CHEB_FFT)
    o = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], **phys_kw(w)))
    o.set_fields(*fields)
    g.step(10)
    gf.step(10)
    for _ in range(10):
        o.step()
    g.device_status()
    for a, b, c, f in zip(g.get_fields(), o.get_fields(), gf.get_fields(), "uvwp"):
        a = a.cpu().numpy()
        assert rel(a, b) <= 1e-10, f
        assert rel(a, c.cpu().numpy()) <= 1e-11, f


def test_dfloat_tc_medium_channel_agrees_with_dfloat_fft(binding):
    """128^3, 20 steps: every double-float output of the backward transform goes through the
    24-bit rounding of its high part (about one value in 2^24 rounds up to the next power of
    two, a case small grids hardly reach)."""
    w = workload("channel_128x128x129")
    fields = inputs.initial_fields(**w)
    gt = grid(binding, w, fields, binding.PREC_DFLOAT, binding.CHEB_TC)
    gf = grid(binding, w, fields, binding.PREC_DFLOAT, binding.CHEB_FFT)
    gt.step(20)
    gf.step(20)
    for a, b, f in zip(gt.get_fields(), gf.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-11, f


def test_tc_rejections(binding):
    g = binding.Grid(16, 16, 17)
    with pytest.raises(binding.ChError) as e:
        g.set_chebyshev(5)
    assert e.value.code == -1
    w = workload("channel_32x32x33")
    gt = grid(binding, w, inputs.initial_fields(**w))
    with pytest.raises(binding.ChError) as e:
        gt.adjoint_begin()
    assert e.value.code == -1
