"""Parity of the CUDA path with the FP64 oracle at the sizes of the benchmark workloads.

The single-stage and ten-step tests of test_gpu_parity.py run small grids; these run the x/y
lengths, line lengths and launch shapes of the workloads themselves (Sec. 2.2, step sequence
i)-v)):

* 512 x 256 x 17: the large channel's x/y transform lengths (Px = 768, Py = 384; the float64 x
  line then holds 17 x 768 complex pairs in shared memory) at a short Chebyshev line: transforms,
  projection, the nine non-linear fields in all three precisions, one full step;
* 512 x 256 x 257 (the large channel itself), float64 and double-float: one step on sampled
  wavenumber lines (the oracle forms every non-linear term and solves the sampled lines);
* 128 x 128 x 129 (the medium channel): the whole state after 10 steps;
* ensemble members of the uneven ensemble's sizes (nx 64 / 96 / 128, ny 64 / 128, nz 65 / 97 /
  129) advanced by the grouped launches, in float64 and in mixed precision.

Tolerances: float64 and double-float paths 1e-10 (max |a - b| / max |b| per field); single
stages 1e-12 (float64), 1e-11 (double-float), 1e-5 (mixed: float32 products and transforms,
about 2^-24 times log2 of the transform lengths, with room).  The mixed path's bounds against
float64 after many steps are the stated ones of MIXED_BOUNDS (see test_mixed_precision_bounds).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.channel import Channel, Params  # noqa: E402
from paper_2406_01322_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

# the stated bounds of the mixed path against float64 (per field, mass, energies)
from paper_2406_01322_gb300.bounds import MIXED_BOUNDS  # noqa: E402


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01322_gb300 import build
    build.build_library()
    from paper_2406_01322_gb300 import binding as b
    b.lib()
    return b


def phys_kw(w):
    return dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])


def oracle_for(w, fields):
    o = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], **phys_kw(w)))
    o.set_fields(*fields)
    return o


def grid_for(binding, w, fields, precision):
    g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=precision, **phys_kw(w))
    g.set_fields(*[torch.from_numpy(f) for f in fields])
    return g


def spec_to_oracle(t):
    return t.cpu().numpy().transpose(2, 1, 0)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---- 512 x 256 x 17: the large channel's x/y lengths ------------------------------------------
def wide():
    return dict(inputs.WORKLOADS["channel_512x256x257_mixed"], nz=17)


@pytest.fixture(scope="module")
def wide_case():
    w = wide()
    fields = inputs.initial_fields(**w)
    o = oracle_for(w, fields)
    r = o.nonlinear_spectral()
    nl = [r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9]]
    return w, fields, o, nl


def test_wide_grid_transforms_and_projection(binding, wide_case):
    w, fields, o, _ = wide_case
    g = grid_for(binding, w, fields, 0)
    rng = np.random.default_rng(9)
    f = rng.standard_normal((w["nz"], w["ny"], w["nx"]))
    spec = g.transform_forward(torch.from_numpy(f))
    ref = o.physical_to_spectral(f)
    assert rel(spec_to_oracle(spec), ref) < 1e-13
    back = g.transform_backward(spec).cpu().numpy()
    assert rel(back, o.spectral_to_physical(ref)) < 1e-13
    for a, b in zip(g.get_spectral(), (o.omega, o.w, o.phi)):
        assert rel(spec_to_oracle(a), b) < 1e-13
    g.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-11), (1, 1e-5)],
                         ids=["fp64", "dfloat", "mixed"])
def test_wide_grid_nonlinear_terms(binding, wide_case, precision, tol):
    w, fields, _, nl = wide_case
    g = grid_for(binding, w, fields, precision)
    got = g.nonlinear()
    for k in range(9):
        assert rel(spec_to_oracle(got[k]), nl[k]) < tol, k
    g.close()


@pytest.mark.parametrize("nx", [64, 128, 256, 512])
def test_float32_x_line_lengths(binding, nx):
    """The float32 x line at every padded length its warp-FFT kernel takes (Px = 96, 192, 384,
    768: 32 lanes x 3, 6, 12, 24 registers), on a short y/z grid: the nine non-linear fields
    against the oracle (1e-5, the mixed single-stage tolerance) and one mixed step against one
    float64 step (2e-5 of each spectral field: float32 products and transforms round at 6e-8,
    and the step's transforms and divergences of the products carry that to a few 1e-6)."""
    w = dict(inputs.WORKLOADS["channel_512x256x257_mixed"], nx=nx, ny=16, nz=9)
    fields = inputs.initial_fields(**w)
    o = oracle_for(w, fields)
    r = o.nonlinear_spectral()
    nl = [r[0] - r[2], r[1] - r[2], r[3], r[4], r[5], r[6], r[7], r[8], r[9]]
    g = grid_for(binding, w, fields, 1)
    got = g.nonlinear()
    for k in range(9):
        assert rel(spec_to_oracle(got[k]), nl[k]) < 1e-5, k
    g64 = grid_for(binding, w, fields, 0)
    g.step(1)
    g64.step(1)
    for a, b in zip(g.get_spectral(), g64.get_spectral()):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 2e-5
    g.close()
    g64.close()


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
def test_wide_grid_one_step(binding, wide_case, precision):
    w, fields, _, _ = wide_case
    o = oracle_for(w, fields)
    o.step()
    g = grid_for(binding, w, fields, precision)
    g.step(1)
    for a, b in zip(g.get_spectral(), (o.omega, o.w, o.phi)):
        assert rel(spec_to_oracle(a), b) < 1e-11
    g.close()


# ---- 512 x 256 x 257: one step, sampled lines ---------------------------------------------------
@pytest.fixture(scope="module")
def large_step():
    w = dict(inputs.WORKLOADS["channel_512x256x257_mixed"])
    fields = inputs.initial_fields(**w)
    o = oracle_for(w, fields)
    rng = np.random.default_rng(5)
    ny, Mx = w["ny"], w["nx"] // 2
    lines = [(0, 0), (1, 0), (0, 1), (ny - 1, 0), (3, 5), (ny // 2 + 1, Mx - 1), (ny - 1, Mx - 1)]
    lines += [(int(rng.integers(0, ny)), int(rng.integers(0, Mx))) for _ in range(13)]
    lines = [(j, m) for (j, m) in lines if j != ny // 2]
    res = o.step(lines=lines)
    return w, fields, res


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
def test_large_channel_one_step_sampled_lines(binding, large_step, precision):
    """512x256x257 (Re_tau = 300, 64 drops): one step of the CUDA path (global-memory tau sweeps,
    N = 256 DCTs, Px = 768, Py = 384) against the oracle on sampled lines."""
    w, fields, res = large_step
    g = grid_for(binding, w, fields, precision)
    g.step(1)
    om, ww, ph = (spec_to_oracle(t) for t in g.get_spectral())
    got = {"omega": om, "w": ww, "phi": ph}
    for k, name in enumerate(("omega", "w", "phi")):
        scale = max(np.max(np.abs(v[k])) for v in res.values())
        for (j, m), v in res.items():
            err = np.max(np.abs(got[name][:, j, m] - v[k])) / scale
            assert err < 1e-10, (name, j, m, err)
    g.close()


# ---- 128 x 128 x 129: the whole state after 10 steps ---------------------------------------------
@pytest.fixture(scope="module")
def medium_ten_steps():
    w = dict(inputs.WORKLOADS["channel_128x128x129"])
    fields = inputs.initial_fields(**w)
    o = oracle_for(w, fields)
    for _ in range(10):
        o.step()
    return w, fields, o.get_fields(), (o.omega, o.w, o.phi), o.diagnostics()


@pytest.mark.parametrize("precision", [0, 2], ids=["fp64", "dfloat"])
def test_medium_channel_ten_steps_full_state(binding, medium_ten_steps, precision):
    """128x128x129 (8 drops): every field after 10 steps within 1e-10 of the oracle, the
    spectral state too, and the diagnostics (mass to 1e-12, the rest to 1e-10)."""
    w, fields, ref, spec, diag = medium_ten_steps
    g = grid_for(binding, w, fields, precision)
    g.step(10)
    for a, b, f in zip(g.get_fields(), ref, "uvwp"):
        assert rel(a.cpu().numpy(), b) <= 1e-10, f
    for a, b in zip(g.get_spectral(), spec):
        assert rel(spec_to_oracle(a), b) <= 1e-10
    d = g.diagnostics()
    assert math.isclose(d["mass"], diag["mass"], rel_tol=1e-12)
    for k in ("kinetic", "grad2", "free_energy", "cfl", "max_phi"):
        assert math.isclose(d[k], diag[k], rel_tol=1e-10), k
    g.close()


# ---- ensemble members of the uneven ensemble's sizes ---------------------------------------------
ENS_SIZES = [(64, 64, 65), (96, 128, 97), (128, 64, 129)]
ENS_STEPS = 5


def ensemble_members():
    base = dict(inputs.ensemble_members(1)[0])
    out = []
    for i, (nx, ny, nz) in enumerate(ENS_SIZES):
        m = dict(base, nx=nx, ny=ny, nz=nz, seed=1000 + i)
        out.append(m)
    return out


@pytest.fixture(scope="module")
def ensemble_oracle():
    ms = ensemble_members()
    res = []
    for m in ms:
        fields = inputs.initial_fields(**m)
        o = oracle_for(m, fields)
        for _ in range(ENS_STEPS):
            o.step()
        res.append((fields, o.get_fields(), o.diagnostics()))
    return ms, res


def field_errors(got, ref):
    errs = {n: rel(a, b) for n, a, b in zip(("u", "v", "w", "phi"), got, ref)}
    umax = np.max(np.abs(ref[0]))
    errs["velocity_scale"] = max(float(np.max(np.abs(a - b))) / umax
                                 for a, b in zip(got[:3], ref[:3]))
    return errs


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_ensemble_members_of_workload_sizes_match_oracle(binding, ensemble_oracle, precision):
    """Members of 64/96/128 x 64/128 x 65/97/129 advanced together by the grouped persistent
    launches: float64 within 1e-10 of the oracle after 5 steps, mixed within its stated bounds."""
    ms, res = ensemble_oracle
    ens = binding.Ensemble([dict(m, precision=precision) for m in ms], precision=precision)
    for g, (fields, _, _) in zip(ens.grids, res):
        g.set_fields(*[torch.from_numpy(f) for f in fields])
    ens.step(ENS_STEPS)
    for g, m, (_, ref, diag) in zip(ens.grids, ms, res):
        got = [t.cpu().numpy() for t in g.get_fields()]
        errs = field_errors(got, ref)
        d = g.diagnostics()
        if precision == 0:
            for n in ("u", "v", "w", "phi"):
                assert errs[n] <= 1e-10, (m["nx"], m["ny"], m["nz"], n, errs[n])
            assert math.isclose(d["mass"], diag["mass"], rel_tol=1e-12)
        else:
            for n, e in errs.items():
                assert e <= MIXED_BOUNDS[n], (m["nx"], m["ny"], m["nz"], n, e)
            assert abs(d["mass"] - diag["mass"]) <= MIXED_BOUNDS["mass"] * abs(diag["mass"])
    ens.close()


# ---- the mixed path's stated bounds at the large channel ------------------------------------------
def test_mixed_precision_bounds_on_the_large_channel(binding):
    """512x256x257, the workload's 200 steps from the same fields: the mixed path against the
    float64 path within MIXED_BOUNDS per field, for the mass of phi and for the energies."""
    w = dict(inputs.WORKLOADS["channel_512x256x257_mixed"])
    fields = inputs.initial_fields(**w)
    out = {}
    for prec in (0, 1):
        g = grid_for(binding, w, fields, prec)
        g.step(w["steps"])
        out[prec] = ([t.cpu().numpy() for t in g.get_fields()], g.diagnostics())
        g.close()
        torch.cuda.empty_cache()
    (f64, d64), (f32, d32) = out[0], out[1]
    errs = field_errors(f32, f64)
    for n, e in errs.items():
        assert e <= MIXED_BOUNDS[n], (n, e)
    for k in ("mass", "kinetic", "grad2", "free_energy"):
        assert abs(d32[k] - d64[k]) <= MIXED_BOUNDS[k] * abs(d64[k]), k
