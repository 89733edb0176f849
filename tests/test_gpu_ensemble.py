"""Ensemble of uneven channels advanced by grouped persistent launches (a CUDA graph per step).

Each member must evolve exactly as the same channel stepped alone: with the default radix
schedules the arithmetic is identical (bitwise); after autotuning the radix schedules may differ,
so the members agree to rounding.  Autotuning leaves every member's state unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_01322_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

PHYS = dict(re_tau=150.0, we=1.0, ch=0.05, pe=20.0, dt=1e-4)
SIZES = [(32, 32, 33), (24, 18, 17), (16, 36, 25), (48, 24, 33)]


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01322_gb300 import build
    build.build_library()
    from paper_2406_01322_gb300 import binding as b
    b.lib()
    return b


def members():
    return [dict(nx=nx, ny=ny, nz=nz, **PHYS) for nx, ny, nz in SIZES]


def fields_of(m, seed):
    return inputs.initial_fields(m["nx"], m["ny"], m["nz"], m["re_tau"], m["ch"], 1, 0.4, seed)


def setup(binding, precision):
    ms = members()
    ens = binding.Ensemble(ms, precision=precision)
    singles = [binding.Grid(precision=precision, **m) for m in ms]
    for i, (g, s, m) in enumerate(zip(ens.grids, singles, ms)):
        f = [torch.from_numpy(a) for a in fields_of(m, 1000 + i)]
        g.set_fields(*f)
        s.set_fields(*f)
    return ens, singles


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_ensemble_members_match_single_grids_bitwise(binding, precision):
    ens, singles = setup(binding, precision)
    ens.step(6)
    for s in singles:
        s.step(6)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            assert torch.equal(a, b)
        assert g.diagnostics()["step"] == 6
    ens.close()


def test_warp_fft_members_match_single_grids_bitwise(binding):
    """Members whose float32 x and y lines take the warp-level FFTs (Px, Py = 96 and 192: nx, ny
    = 64 and 128), beside one that takes the block passes: each evolves exactly as the same
    channel stepped alone (mixed precision, 6 steps)."""
    ms = [dict(nx=nx, ny=ny, nz=nz, **PHYS) for nx, ny, nz in [(64, 64, 17), (128, 16, 9),
                                                                (32, 32, 17)]]
    ens = binding.Ensemble(ms, precision=1)
    singles = [binding.Grid(precision=1, **m) for m in ms]
    for i, (g, s, m) in enumerate(zip(ens.grids, singles, ms)):
        f = [torch.from_numpy(a) for a in fields_of(m, 2000 + i)]
        g.set_fields(*f)
        s.set_fields(*f)
    ens.step(6)
    for s in singles:
        s.step(6)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            assert torch.equal(a, b)
    ens.close()


def test_ensemble_timed_steps_match_graph_steps(binding):
    ens, singles = setup(binding, 0)
    tot, ks = ens.step_timed(3)
    assert len(ks) == 6 and tot > 0 and min(ks) >= 0
    for s in singles:
        s.step(3)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            assert torch.equal(a, b)
    ens.close()


def test_autotune_keeps_state_and_results(binding):
    ens, singles = setup(binding, 0)
    ens.step(2)
    for s in singles:
        s.step(2)
    before = [[t.clone() for t in g.get_fields()] for g in ens.grids]
    tuning = ens.autotune(reps=1)
    assert tuning["tuned"] == 1
    after = [g.get_fields() for g in ens.grids]
    for x, y in zip(before, after):
        for a, b in zip(x, y):
            assert torch.equal(a, b)
    ens.step(4)
    for s in singles:
        s.step(4)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            rel = float((a - b).abs().max() / b.abs().max())
            assert rel < 1e-12
    ens.close()


def test_ensemble_requires_every_member_set(binding):
    ens = binding.Ensemble(members()[:2], precision=0)
    with pytest.raises(binding.ChError) as e:
        ens.step(1)
    assert e.value.code == -7
    ens.close()


def test_ensemble_rejects_mixed_precisions(binding):
    """All members share one precision (one grouped kernel per stage)."""
    ms = members()[:2]
    ms[1]["precision"] = binding.PREC_MIXED
    with pytest.raises(binding.ChError) as e:
        binding.Ensemble(ms, precision=binding.PREC_FP64)
    assert e.value.code == -1


def test_ensemble_of_mixed_wall_conditions_matches_single_grids(binding):
    """Members with the four wall cases (no-slip, free-slip, and the two combinations) in one
    ensemble: each member's grouped solve takes its own wall rows and matches the member stepped
    alone bitwise."""
    ms = members()
    for i, m in enumerate(ms):
        m["bc"] = i % 4
    ens = binding.Ensemble(ms, precision=0)
    singles = [binding.Grid(precision=0, **m) for m in ms]
    for i, (g, s, m) in enumerate(zip(ens.grids, singles, ms)):
        f = [torch.from_numpy(a) for a in inputs.initial_fields(
            m["nx"], m["ny"], m["nz"], m["re_tau"], m["ch"], 1, 0.4, 2000 + i, bc=m["bc"])]
        g.set_fields(*f)
        s.set_fields(*f)
    ens.step(4)
    for s in singles:
        s.step(4)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            assert torch.equal(a, b)
    ens.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_ensemble_tensor_core_chebyshev_matches_single_grids_bitwise(binding, precision):
    """CHEB_TC in the ensemble: each member's z transforms are the single-grid tensor-core
    launches and the grouped zrhs / zbwd run the single-grid coefficient kernels' arithmetic, so
    every member matches the same channel stepped alone with CHEB_TC bit for bit."""
    ens, singles = setup(binding, precision)
    ens.set_chebyshev(binding.CHEB_TC)
    assert ens.chebyshev() == binding.CHEB_TC
    assert all(g.chebyshev() == binding.CHEB_TC for g in ens.grids)
    assert ens.tuning()["chebyshev"] == binding.CHEB_TC
    for s in singles:
        s.set_chebyshev(binding.CHEB_TC)
    ens.step(6)
    for s in singles:
        s.step(6)
    for g, s in zip(ens.grids, singles):
        g.device_status()
        for a, b in zip(g.get_fields(), s.get_fields()):
            assert torch.equal(a, b)
        assert g.diagnostics()["step"] == 6
    ens.close()


def test_ensemble_tensor_core_chebyshev_agrees_with_fft_method(binding):
    """FP64 ensemble, ten steps with each Chebyshev method: both transforms are float64-accurate
    (the tensor-core one within 1e-15 of the exact transform per line), so the fields agree to
    rounding; the timed step (member transforms counted in stages 0 and 2) gives the graph step's
    fields."""
    ens_f, _ = setup(binding, 0)
    ens_t, singles = setup(binding, 0)
    ens_t.set_chebyshev(binding.CHEB_TC)
    ens_f.step(10)
    tot, ks = ens_t.step_timed(4)
    assert len(ks) == 6 and tot > 0 and min(ks) >= 0
    ens_t.step(6)
    for s in singles:
        s.set_chebyshev(binding.CHEB_TC)
        s.step(10)
    for gf, gt, s in zip(ens_f.grids, ens_t.grids, singles):
        for a, b, c in zip(gt.get_fields(), gf.get_fields(), s.get_fields()):
            assert torch.equal(a, c)
            rel = float((a - b).abs().max() / b.abs().max())
            assert rel < 1e-11
    ens_f.close()
    ens_t.close()


def test_ensemble_switches_chebyshev_method_and_autotunes(binding):
    """Switching the ensemble's method mid-run continues the same trajectory (to rounding), an
    unknown method is rejected without a change, and autotuning under CHEB_TC keeps the state."""
    ens, singles = setup(binding, 0)
    ens.step(2)
    ens.set_chebyshev(binding.CHEB_TC)
    ens.step(2)
    with pytest.raises(binding.ChError) as e:
        ens.set_chebyshev(7)
    assert e.value.code == -1 and ens.chebyshev() == binding.CHEB_TC
    before = [[t.clone() for t in g.get_fields()] for g in ens.grids]
    assert ens.autotune(reps=1)["tuned"] == 1
    for x, g in zip(before, ens.grids):
        for a, b in zip(x, g.get_fields()):
            assert torch.equal(a, b)
    ens.set_chebyshev(binding.CHEB_FFT)
    ens.step(2)
    for s in singles:
        s.step(6)
    for g, s in zip(ens.grids, singles):
        for a, b in zip(g.get_fields(), s.get_fields()):
            rel = float((a - b).abs().max() / b.abs().max())
            assert rel < 1e-11
    ens.close()
