"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance (FP64 path): max relative field error max|a - b| / max|b| per field of at most 1e-10
after 10 steps (u, v, w, phi on the unpadded grid); single-stage comparisons are held to the
rounding level of the stage (1e-12 relative).  Inputs come from the seeded generators.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def workload(name, **over):
    w = dict(inputs.WORKLOADS[name])
    w.update(over)
    return w


def phys_kw(w):
    return dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])


def make_pair(binding, w, precision=0, fields=None):
    if fields is None:
        fields = inputs.initial_fields(**w)
    bc = w.get("bc", 0)
    g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=precision, bc=bc, **phys_kw(w))
    g.set_fields(*[torch.from_numpy(f) for f in fields])
    o = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], bc=bc, **phys_kw(w)))
    o.set_fields(*fields)
    return g, o


def spec_to_oracle(t):
    """(Mx, Ny, Nz) device complex tensor -> (Nz, Ny, Mx) numpy (oracle layout)."""
    return t.cpu().numpy().transpose(2, 1, 0)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SIZES = [
    ("channel_32x32x33", {}),
    ("channel_32x32x33", dict(nx=24, ny=18, nz=17)),    # radix-3 lengths, ragged z tile
    ("channel_32x32x33", dict(nx=16, ny=36, nz=25)),    # Py = 54, N = 24
]


@pytest.mark.parametrize("name,over", SIZES)
def test_transform_forward_backward(binding, name, over):
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((w["nz"], w["ny"], w["nx"]))
    spec = g.transform_forward(torch.from_numpy(f))
    ref = o.physical_to_spectral(f)
    assert rel(spec_to_oracle(spec), ref) < 1e-13
    back = g.transform_backward(spec).cpu().numpy()
    assert rel(back, o.spectral_to_physical(ref)) < 1e-13


@pytest.mark.parametrize("name,over", SIZES)
def test_set_fields_projection(binding, name, over):
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    om, ww, ph = g.get_spectral()
    assert rel(spec_to_oracle(om), o.omega) < 1e-13
    assert rel(spec_to_oracle(ww), o.w) < 1e-13
    assert rel(spec_to_oracle(ph), o.phi) < 1e-13
    for a, b in zip(g.get_fields(), o.get_fields()):
        assert rel(a.cpu().numpy(), b) < 1e-12


@pytest.mark.parametrize("name,over", SIZES)
def test_nonlinear_terms(binding, name, over):
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    got = g.nonlinear()
    r = o.nonlinear_spectral()
    # the step carries Sxx - Szz and Syy - Szz (the isotropic stress is a pure gradient)
    ref = [r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9]]
    for k in range(9):
        assert rel(spec_to_oracle(got[k]), ref[k]) < 1e-12, k


@pytest.mark.parametrize("name,over", SIZES)
def test_one_step_state(binding, name, over):
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    g.step(1)
    o.step()
    om, ww, ph = g.get_spectral()
    assert rel(spec_to_oracle(om), o.omega) < 1e-11
    assert rel(spec_to_oracle(ww), o.w) < 1e-11
    assert rel(spec_to_oracle(ph), o.phi) < 1e-11


LONG_LINES = [("channel_32x32x33", dict(nz=257)),                  # N = 256: global zsolve,
              ("channel_32x32x33", dict(nx=16, ny=16, nz=193))]   # 8*8*4 DCT; N = 192: 8*8*3


def readout_floor(w, fields):
    """The rounding floor of the field error measure: the oracle's set_fields + get_fields with
    its dense Chebyshev matrices against the same with scipy's FFT-based DCT-I (two FP64
    evaluations of the same transforms), per field, max |a - b| / max |b|."""
    import scipy.fft
    N = w["nz"] - 1

    class ScipyDct(Channel):
        def cheb_fwd(self, fz):
            c = scipy.fft.dct(fz, type=1, axis=0) / N
            c[0] /= 2
            c[-1] /= 2
            return c

        def cheb_bwd(self, a):
            b = a.copy()
            b[0] *= 2
            b[-1] *= 2
            return scipy.fft.dct(b, type=1, axis=0) / 2

    p = Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], **phys_kw(w))
    o1, o2 = Channel(p), ScipyDct(p)
    o1.set_fields(*fields)
    o2.set_fields(*fields)
    return [rel(a, b) for a, b in zip(o2.get_fields(), o1.get_fields())]


@pytest.mark.parametrize("name,over", LONG_LINES)
def test_long_lines_ten_steps_within_1e_10(binding, name, over):
    """Lines long enough for the global-memory tau sweeps and multi-element scan chunks: every
    field within 1e-10 of the oracle after 10 steps, except where the measure's own rounding floor
    is higher.  That is v here: v (max 0.08) is about 1000 times smaller than u (max 75), so the
    rounding of u's transforms, which reaches v through the vorticity, is 1e-10 of max |v| at
    N = 256 for any two FP64 evaluations (the oracle against itself with another DCT algorithm:
    9e-11); v is held to 4 times that floor (measured: 2.0e-10, 2.6e-13 of max |u|)."""
    w = workload(name, **over)
    fields = inputs.initial_fields(**w)
    g, o = make_pair(binding, w, fields=fields)
    floor = readout_floor(w, fields)
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f, fl in zip(g.get_fields(), o.get_fields(), "uvwp", floor):
        assert rel(a.cpu().numpy(), b) <= max(1e-10, 4.0 * fl), (f, fl)


@pytest.mark.parametrize("name,over", LONG_LINES)
@pytest.mark.parametrize("method", ["fft", "tc"])
def test_long_lines_spectral_state_within_1e_10(binding, name, over, method):
    """The same long lines compared where the readout adds no rounding of its own: the spectral
    state (omega_z with the mean flow, w, phi coefficients) after 10 steps within 1e-10 of the
    oracle's, flat, with either Chebyshev method (the float64 DCT or the exact-split tensor-core
    product)."""
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    if method == "tc":
        g.set_chebyshev(binding.CHEB_TC)
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f in zip(g.get_spectral(), (o.omega, o.w, o.phi), ("omega", "w", "phi")):
        assert rel(spec_to_oracle(a), b) <= 1e-10, f
    g.close()


@pytest.mark.parametrize("name,over", SIZES)
def test_ten_steps_fp64_within_1e_10(binding, name, over):
    w = workload(name, **over)
    g, o = make_pair(binding, w)
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f


def test_diagnostics_match_oracle(binding):
    w = workload("channel_32x32x33")
    g, o = make_pair(binding, w)
    g.step(3)
    for _ in range(3):
        o.step()
    d = g.diagnostics()
    r = o.diagnostics()
    assert d["step"] == 3 and d["nan"] == 0
    for k in ("mass", "kinetic", "grad2", "free_energy", "cfl", "max_phi"):
        assert math.isclose(d[k], r[k], rel_tol=1e-10, abs_tol=1e-12), k


def test_poiseuille_fixed_point_on_gpu(binding):
    w = workload("channel_32x32x33")
    nz, ny, nx = w["nz"], w["ny"], w["nx"]
    z = np.cos(np.pi * np.arange(nz) / (nz - 1))
    u = np.broadcast_to((0.5 * w["re_tau"] * (1 - z * z))[:, None, None], (nz, ny, nx)).copy()
    zero = np.zeros((nz, ny, nx))
    g = binding.Grid(nx, ny, nz, **phys_kw(w))
    g.set_fields(*[torch.from_numpy(a) for a in (u, zero, zero, zero - 1.0)])
    g.step(20)
    uu, vv, ww, pp = [t.cpu().numpy() for t in g.get_fields()]
    # rounding drift per step: the odd Chebyshev outputs of the N-point DCT-I come from a
    # prefix sum, whose rounding grows with the number of terms (~1e-14 per step here)
    assert rel(uu, u) < 20 * 2e-14
    assert np.max(np.abs(vv)) < 1e-12 and np.max(np.abs(ww)) < 1e-12
    assert np.max(np.abs(pp + 1.0)) < 20 * 2e-15  # rounding drift per step


def test_checkpoint_resume_is_bitwise(binding):
    w = workload("channel_32x32x33", nx=24, ny=18, nz=17)
    g, _ = make_pair(binding, w)
    g.step(3)
    st = g.get_state()
    g.step(4)
    a = [t.clone() for t in g.get_fields()]
    g.set_state(st)
    g.step(4)
    b = g.get_fields()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_timed_step_matches_graph_step(binding):
    """ch_step_timed (events between launches) runs the same schedule as ch_step (graph)."""
    w = workload("channel_32x32x33", nx=24, ny=18, nz=17)
    fields = inputs.initial_fields(**w)
    a = binding.Grid(w["nx"], w["ny"], w["nz"], **phys_kw(w))
    b = binding.Grid(w["nx"], w["ny"], w["nz"], **phys_kw(w))
    for g in (a, b):
        g.set_fields(*[torch.from_numpy(f) for f in fields])
    a.step(5)
    tot, ks = b.step_timed(5)
    assert len(ks) == len(binding.Grid.KERNELS) and min(ks) >= 0 and sum(ks) <= tot * 1.01 + 1e-3
    for x, y in zip(a.get_fields(), b.get_fields()):
        assert torch.equal(x, y)
    assert a.diagnostics()["step"] == b.diagnostics()["step"] == 5


def test_host_entry_points_match_device(binding):
    w = workload("channel_32x32x33", nx=24, ny=18, nz=17)
    fields = inputs.initial_fields(**w)
    g = binding.Grid(w["nx"], w["ny"], w["nz"], **phys_kw(w))
    g.set_fields_host(*fields)
    g.step(2)
    h = g.get_fields_host()
    d = g.get_fields()
    for x, y in zip(h, d):
        assert torch.equal(x, y.cpu())


@pytest.mark.parametrize("name,over", SIZES)
def test_dfloat_nonlinear_terms(binding, name, over):
    """Double-float x/y transforms and products (CH_PREC_DFLOAT) against the FP64 oracle."""
    w = workload(name, **over)
    g, o = make_pair(binding, w, precision=binding.PREC_DFLOAT)
    got = g.nonlinear()
    r = o.nonlinear_spectral()
    ref = [r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9]]
    for k in range(9):
        assert rel(spec_to_oracle(got[k]), ref[k]) < 1e-11, k


@pytest.mark.parametrize("name,over", SIZES)
def test_dfloat_ten_steps_within_1e_10(binding, name, over):
    """The double-float path meets the FP64 path's bar: max relative field error <= 1e-10
    against the FP64 oracle after 10 steps."""
    w = workload(name, **over)
    g, o = make_pair(binding, w, precision=binding.PREC_DFLOAT)
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f


FREE_SLIP = [("channel_32x32x33", dict(bc=b)) for b in (1, 2, 3)] + \
            [("channel_32x32x33", dict(nx=24, ny=18, nz=17, bc=b)) for b in (1, 2, 3)]


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
@pytest.mark.parametrize("name,over", FREE_SLIP)
def test_free_slip_ten_steps_within_1e_10(binding, name, over, precision):
    """Free-slip walls (bc = 1) and the two combinations (bc = 2, 3: no-slip at one wall,
    free-slip at the other) from fields meeting those walls: 10 steps against the oracle."""
    w = workload(name, **over)
    g, o = make_pair(binding, w, precision)
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f


def test_free_slip_uniform_flow_accelerates_by_gx_dt(binding):
    nx, ny, nz = 16, 8, 17
    dt, U0, n = 2e-3, 3.0, 10
    g = binding.Grid(nx, ny, nz, re_tau=50.0, dt=dt, gx=1.0, bc=binding.BC_FREE_SLIP)
    zero = torch.zeros((nz, ny, nx), dtype=torch.float64)
    g.set_fields(zero + U0, zero, zero, zero - 1.0)
    g.step(n)
    u, v, ww, _ = [t.cpu() for t in g.get_fields()]
    assert float((u - (U0 + n * dt)).abs().max()) < 1e-12
    assert float(v.abs().max()) < 1e-14 and float(ww.abs().max()) < 1e-14


@pytest.mark.parametrize("bc", [2, 3])
def test_open_channel_laminar_profile_is_a_fixed_point_on_gpu(binding, bc):
    nx, ny, nz, re = 16, 8, 17, 50.0
    g = binding.Grid(nx, ny, nz, re_tau=re, dt=2e-3, gx=1.0, bc=bc)
    z = np.cos(np.pi * np.arange(nz) / (nz - 1))
    sz = z if bc == 2 else -z
    U = np.broadcast_to((0.5 * re * (3.0 - sz) * (1.0 + sz))[:, None, None], (nz, ny, nx)).copy()
    zero = np.zeros((nz, ny, nx))
    g.set_fields(*[torch.from_numpy(a) for a in (U, zero, zero, zero - 1.0)])
    g.step(10)
    u, v, ww, _ = [t.cpu().numpy() for t in g.get_fields()]
    assert rel(u, U) < 1e-12
    assert np.max(np.abs(v)) < 1e-14 and np.max(np.abs(ww)) < 1e-14


def test_free_slip_rejected_by_the_adjoint(binding):
    w = workload("channel_32x32x33", nx=16, ny=8, nz=17, bc=1)
    g, _ = make_pair(binding, w)
    with pytest.raises(binding.ChError) as e:
        g.adjoint_begin()
    assert e.value.code == -1


def test_mixed_precision_error_bounds(binding):
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    g64, o = make_pair(binding, w, 0, fields)
    g32, _ = make_pair(binding, w, 1, fields)
    g64.step(10)
    g32.step(10)
    for _ in range(10):
        o.step()
    for a, b, c, f in zip(g32.get_fields(), g64.get_fields(), o.get_fields(), "uvwp"):
        e = rel(a.cpu().numpy(), b.cpu().numpy())
        assert e < 1e-4, (f, e)
        assert rel(b.cpu().numpy(), c) < 1e-10
    d32, d64 = g32.diagnostics(), g64.diagnostics()
    assert abs(d32["mass"] - d64["mass"]) <= 1e-6 * abs(d64["mass"])


def test_error_codes(binding):
    with pytest.raises(binding.ChError) as e:
        binding.Grid(10, 16, 17)            # 10 = 2 * 5 is not {2,3}-smooth
    assert e.value.code == -2
    with pytest.raises(binding.ChError) as e:
        binding.Grid(16, 16, 18)            # nz - 1 odd
    assert e.value.code == -2
    with pytest.raises(binding.ChError) as e:
        binding.Grid(16, 16, 17, dt=0.0)
    assert e.value.code == -1
    g = binding.Grid(16, 16, 17)
    with pytest.raises(binding.ChError) as e:
        g.step(1)                           # no fields yet
    assert e.value.code == -7


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
def test_medium_channel_one_step_sampled_lines(binding, precision):
    """128x128x129 workload: one GPU step against the oracle on a sample of wavenumber lines
    (the oracle forms every non-linear term but solves only the sampled lines)."""
    w = workload("channel_128x128x129")
    g, o = make_pair(binding, w, precision)
    g.step(1)
    rng = np.random.default_rng(3)
    lines = [(0, 0), (1, 0), (0, 1), (w["ny"] - 1, 0), (5, 7), (w["ny"] // 2 + 3, 63)]
    lines += [(int(rng.integers(0, w["ny"])), int(rng.integers(0, w["nx"] // 2))) for _ in range(10)]
    lines = [(j, m) for (j, m) in lines if j != w["ny"] // 2]
    res = o.step(lines=lines)
    om, ww, ph = (spec_to_oracle(t) for t in g.get_spectral())
    got = {"omega": om, "w": ww, "phi": ph}
    for k, name in enumerate(("omega", "w", "phi")):
        # one scale per field (the largest sampled coefficient), as for the field error measure
        scale = max(np.max(np.abs(v[k])) for v in res.values())
        for (j, m), v in res.items():
            err = np.max(np.abs(got[name][:, j, m] - v[k])) / scale
            assert err < 1e-10, (name, j, m, err)


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
@pytest.mark.parametrize("name,over", SIZES + [("channel_512x256x257_mixed", dict(nz=17))])
def test_pruned_padded_transforms_ten_steps_within_1e_10(binding, name, over, precision):
    """The x/y transforms of the 3/2-rule padding pruned (radix 3 first: the zero middle third of
    the backward input and the unused middle third of the forward output are skipped): the
    non-linear fields within 1e-12 of the oracle (float64) and 10 steps within 1e-10."""
    w = workload(name, **over)
    g, o = make_pair(binding, w, precision)
    g.set_fft_pruning(1)
    assert g.fft_pruning() == 1
    if precision == 0:
        got = g.nonlinear()
        r = o.nonlinear_spectral()
        ref = [r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9]]
        for k in range(9):
            assert rel(spec_to_oracle(got[k]), ref[k]) < 1e-12, k
    g.step(10)
    for _ in range(10):
        o.step()
    for a, b, f in zip(g.get_fields(), o.get_fields(), "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f


def test_pruned_padded_transforms_mixed_match_unpruned(binding):
    """Mixed precision: the pruned and the default schedules round differently in float32 but
    agree within the mixed path's stated bounds, and switching back restores the default."""
    from paper_2406_01322_gb300.bounds import MIXED_BOUNDS
    w = workload("channel_32x32x33")
    fields = inputs.initial_fields(**w)
    a, _ = make_pair(binding, w, 1, fields)
    b, _ = make_pair(binding, w, 1, fields)
    b.set_fft_pruning(1)
    a.step(10)
    b.step(10)
    for x, y, f in zip(b.get_fields(), a.get_fields(), ("u", "v", "w", "phi")):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < MIXED_BOUNDS[f], f
    b.set_fft_pruning(0)
    assert b.fft_pruning() == 0
    with pytest.raises(binding.ChError):
        b.set_fft_pruning(2)
