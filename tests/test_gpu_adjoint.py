"""Discrete adjoint on the GPU (through the C ABI) against the oracle's reverse-mode gradient
(float64 torch autograd through the oracle step) and against central differences of the GPU
objective along directions that keep the wall conditions.

Tolerances: the objective to 1e-12 relative; gradients field by field to 1e-10 of the field's
largest oracle value (both sides differentiate the same discrete map in float64, so they differ
only by rounding order); central differences along 16 seeded directions (direction j from seed
100 + j; eps = 2e-4 and 1e-4 Richardson-extrapolated, since the directions carry grid-scale
content and one central difference keeps an O(eps^2) error of a few 1e-6) to 1e-6 of the
directional derivative.
Checkpointing must not change a single bit of the gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint  # noqa: E402
from oracle.channel import Params  # noqa: E402
from paper_2406_01322_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

PHYS = dict(re_tau=50.0, ch=0.15, pe=10.0, we=1.0, dt=2e-3)
CASES = [dict(nx=12, ny=8, nz=9, steps=3), dict(nx=24, ny=18, nz=17, steps=2),
         dict(nx=32, ny=32, nz=33, steps=5)]


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_01322_gb300 import build
    build.build_library()
    from paper_2406_01322_gb300 import binding as b
    b.lib()
    return b


def fields(c, seed=3):
    f = inputs.initial_fields(c["nx"], c["ny"], c["nz"], PHYS["re_tau"], PHYS["ch"], 1, 0.6,
                              seed, amp=0.5)
    return [np.ascontiguousarray(a) for a in f]


def grid(binding, c, **kw):
    return binding.Grid(c["nx"], c["ny"], c["nz"], **PHYS, **kw)


def dev(f):
    return [torch.from_numpy(a).cuda() for a in f]


def admissible_direction(rng, shape):
    """Seeded direction that keeps the wall conditions exactly: at every (x, y) point
    u, v = (1 - z^2) q(z) with deg q <= N - 2 and w = (1 - z^2)^2 q(z) with deg q <= N - 4
    (random Chebyshev coefficients), so the degree-N interpolants vanish at the walls and w's
    wall derivative is zero; phi is any field.  The CUDA step solves Crank-Nicolson for
    q^{n+1} + q^n, which is the literal Crank-Nicolson step (the map the adjoint differentiates)
    only on states that meet the wall conditions, so finite differences of the CUDA step are
    taken along such directions."""
    nz, ny, nx = shape
    N = nz - 1
    j = np.arange(nz)
    z = np.cos(np.pi * j / N)

    def poly(deg):
        c = rng.standard_normal((deg + 1, ny, nx))
        T = np.cos(np.pi * np.outer(j, np.arange(deg + 1)) / N)   # T_k(z_j)
        return np.tensordot(T, c, axes=(1, 0))

    b1 = (1.0 - z * z)[:, None, None]
    return [b1 * poly(N - 2), b1 * poly(N - 2), b1 * b1 * poly(N - 4), rng.standard_normal(shape)]


def richardson_fd(g, f, d, steps, eps=1e-4):
    """Directional derivative of the GPU objective after `steps` steps along d: central
    differences at 2 eps and eps combined to cancel the O(eps^2) truncation."""
    def central(e):
        js = []
        for sgn in (1.0, -1.0):
            g.set_fields(*dev([a + sgn * e * b for a, b in zip(f, d)]))
            g.step(steps)
            js.append(g.objective())
        return (js[0] - js[1]) / (2 * e)
    return (4.0 * central(eps) - central(2 * eps)) / 3.0


def gpu_gradient(binding, c, f, every):
    g = grid(binding, c)
    ts = [t.clone().requires_grad_(True) for t in dev(f)]
    J = binding.objective_after(g, *ts, c["steps"], checkpoint_every=every)
    J.backward()
    out = float(J.detach()), [t.grad.detach().cpu().numpy() for t in ts]
    g.close()
    return out


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"{c['nx']}x{c['ny']}x{c['nz']}")
def test_objective_matches_oracle(binding, c):
    f = fields(c)
    g = grid(binding, c)
    g.set_fields(*dev(f))
    t = adjoint.TorchChannel(Params(nx=c["nx"], ny=c["ny"], nz=c["nz"], **PHYS))
    st = t.set_fields(*[torch.tensor(a) for a in f])
    ref = float(t.objective(st))
    assert abs(g.objective() - ref) <= 1e-12 * abs(ref)
    hist = None
    for _ in range(c["steps"]):
        st, hist = t.step(st, hist)
    g.step(c["steps"])
    ref = float(t.objective(st))
    assert abs(g.objective() - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"{c['nx']}x{c['ny']}x{c['nz']}")
def test_gradient_matches_oracle_adjoint(binding, c):
    f = fields(c)
    J, gg = gpu_gradient(binding, c, f, every=2)
    Jr, gr = adjoint.gradient(Params(nx=c["nx"], ny=c["ny"], nz=c["nz"], **PHYS), f, c["steps"])
    assert abs(J - Jr) <= 1e-12 * abs(Jr)
    for name, a, b in zip("uvwp", gg, gr):
        err = np.max(np.abs(a - b))
        scale = np.max(np.abs(b))
        assert err <= 1e-10 * scale, (name, err, scale)


def test_gradient_with_zero_steps(binding):
    c = dict(CASES[0], steps=0)
    f = fields(c, seed=8)
    J, gg = gpu_gradient(binding, c, f, every=1)
    Jr, gr = adjoint.gradient(Params(nx=c["nx"], ny=c["ny"], nz=c["nz"], **PHYS), f, 0)
    assert abs(J - Jr) <= 1e-12 * abs(Jr)
    for a, b in zip(gg, gr):
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_checkpointing_is_bitwise_neutral(binding):
    c = dict(CASES[2], steps=7)
    f = fields(c, seed=5)
    _, g1 = gpu_gradient(binding, c, f, every=1)
    for every in (3, 7, 100):
        _, g2 = gpu_gradient(binding, c, f, every=every)
        for a, b in zip(g1, g2):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("c", CASES[1:], ids=lambda c: f"{c['nx']}x{c['ny']}x{c['nz']}")
def test_gradient_matches_central_differences(binding, c):
    f = fields(c, seed=11)
    _, gg = gpu_gradient(binding, c, f, every=2)
    g = grid(binding, c)
    for trial in range(16):
        d = admissible_direction(np.random.default_rng(100 + trial), f[0].shape)
        fd = richardson_fd(g, f, d, c["steps"])
        an = sum(float(np.sum(a * b)) for a, b in zip(gg, d))
        assert abs(fd - an) <= 1e-6 * abs(an), (trial, fd, an)
    g.close()


def test_full_size_directional_derivative(binding):
    """Adjoint workload at full size (128 x 128 x 129, 50 steps, checkpoints every 10 steps):
    the gradient's directional derivative along a seeded admissible direction against central
    differences of the GPU objective (a property that holds at any size).  The direction has
    content up to the grid scale, so the O(eps^2) truncation of one central difference is
    about 5e-6 relative at eps = 1e-4; Richardson extrapolation of eps = 2e-4 and 1e-4 removes
    it, leaving rounding (about 1e-7 relative)."""
    w = inputs.WORKLOADS["channel_128x128x129_adjoint"]
    f = [np.ascontiguousarray(a) for a in inputs.initial_fields(**w)]
    kw = dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])
    g = binding.Grid(w["nx"], w["ny"], w["nz"], **kw)
    ts = [t.clone().requires_grad_(True) for t in dev(f)]
    J = binding.objective_after(g, *ts, w["steps"], checkpoint_every=10)
    J.backward()
    rng = np.random.default_rng(12)
    d = admissible_direction(rng, f[0].shape)
    an = sum(float(torch.sum(t.grad * torch.from_numpy(b).cuda())) for t, b in zip(ts, d))

    fd = richardson_fd(g, f, d, w["steps"])
    assert np.isfinite(an) and abs(fd - an) <= 2e-6 * abs(an), (fd, an)
    g.close()


def test_segment_reversal_equals_step_by_step_bitwise(binding):
    """ch_adjoint_segment (recompute keeping the y-padded fields, reverse) against reversing the
    same steps one by one from saved states (ch_adjoint_step recomputes those fields)."""
    c = dict(CASES[2], steps=6)
    f = fields(c, seed=9)
    grads = []
    for mode in ("segment", "steps"):
        g = grid(binding, c)
        g.set_fields(*dev(f))
        states = []
        for _ in range(c["steps"]):
            states.append(g.get_state())
            g.step(1)
        g.adjoint_begin()
        if mode == "segment":
            g.adjoint_segment(states[3], 3)
            g.adjoint_segment(states[0], 3)
        else:
            for st in reversed(states):
                g.adjoint_step(st)
        grads.append([t.cpu() for t in g.adjoint_gradient()])
        g.adjoint_end()
        g.close()
    for a, b in zip(*grads):
        assert torch.equal(a, b)


def test_adjoint_call_order_and_precision(binding):
    c = CASES[0]
    f = fields(c)
    g = grid(binding, c)
    with pytest.raises(binding.ChError) as e:
        g.objective()                      # no fields yet
    assert e.value.code == -7
    g.set_fields(*dev(f))
    s0 = g.get_state()
    with pytest.raises(binding.ChError) as e:
        g.adjoint_step(s0)                 # before adjoint_begin
    assert e.value.code == -7
    g.step(1)
    g.adjoint_begin()
    g.adjoint_step(s0)
    with pytest.raises(binding.ChError) as e:
        g.step(1)                          # products of the restored state not recomputed
    assert e.value.code == -7
    g.adjoint_end()
    g.set_state(s0)
    g.step(1)                              # usable again
    g.close()
    m = grid(binding, c, precision=binding.PREC_MIXED)
    m.set_fields(*dev(f))
    with pytest.raises(binding.ChError) as e:
        m.objective()
    assert e.value.code == -1
    m.close()
