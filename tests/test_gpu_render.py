"""Headless interface image on the GPU (through the C ABI) against the oracle's ray caster on the
same state.  The hit/miss decision of a ray is taken in float64 on both sides; rays that graze
the surface can decide differently under different rounding, so up to 0.3 % of the pixels may
differ in the hit mask (each such pixel must be a rim pixel of the other image); where both hit,
the depths agree to 1e-9 relative and the colours to one level."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import render  # noqa: E402
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


def compare(rgb_g, dep_g, rgb_o, dep_o):
    hg, ho = dep_g >= 0, dep_o >= 0
    diff = hg != ho
    assert diff.mean() <= 0.003, diff.mean()
    # a differing pixel sits next to a pixel on which the two images agree about a hit
    pad = np.pad(ho & hg, 1)
    near = pad[:-2, 1:-1] | pad[2:, 1:-1] | pad[1:-1, :-2] | pad[1:-1, 2:]
    assert np.all(~diff | near)
    both = hg & ho
    assert np.max(np.abs(dep_g[both] - dep_o[both]) / dep_o[both]) < 1e-9
    assert np.max(np.abs(rgb_g[both].astype(int) - rgb_o[both].astype(int))) <= 1
    assert np.array_equal(rgb_g[~hg & ~ho], rgb_o[~hg & ~ho])


@pytest.mark.parametrize("case", ["drop", "channel_128x128x129"])
def test_render_matches_oracle(binding, case):
    if case == "drop":
        w = dict(nx=32, ny=32, nz=33, lx=2.0, ly=2.0, re_tau=50.0, ch=0.1, pe=10.0, we=1.0, dt=1e-3)
        f = inputs.initial_fields(32, 32, 33, 50.0, 0.1, 1, 0.5, 1, amp=0.0, lx=2.0, ly=2.0)
        cam = ((1.0, -3.0, 0.0), (1.0, 1.0, 0.0), (0.0, 0.0, 1.0), 30.0)
        W, H = 64, 64
    else:
        w = dict(inputs.WORKLOADS[case])
        f = inputs.initial_fields(**w)
        w.setdefault("lx", 4 * np.pi)
        w.setdefault("ly", 2 * np.pi)
        cam = ((-4.0, -5.0, 2.5), (2 * np.pi, np.pi, 0.0), (0.0, 0.0, 1.0), 45.0)
        W, H = 96, 64
    kw = dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])
    g = binding.Grid(w["nx"], w["ny"], w["nz"], lx=w["lx"], ly=w["ly"], **kw)
    g.set_fields(*[torch.from_numpy(a) for a in f])
    rgb, dep = g.render_interface(W, H, cam[0], cam[1], cam[2], cam[3])
    c = Channel(Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], lx=w["lx"], ly=w["ly"], **kw))
    c.set_fields(*f)
    rgb_o, dep_o = render.render(c, W, H, cam[0], cam[1], cam[2], cam[3])
    assert (dep_o >= 0).mean() > 0.01          # the view shows the interface
    compare(rgb.cpu().numpy(), dep.cpu().numpy(), rgb_o, dep_o)


def test_render_rejects_bad_arguments(binding):
    g = binding.Grid(16, 16, 17)
    with pytest.raises(binding.ChError) as e:
        g.render_interface(8, 8, (0, 0, 0), (1, 0, 0))   # fields not set
    assert e.value.code == -7
    f = inputs.initial_fields(16, 16, 17, 150.0, 0.05, 1, 0.4, 1)
    g.set_fields(*[torch.from_numpy(a) for a in f])
    with pytest.raises(binding.ChError) as e:
        g.render_interface(8, 8, (1, 1, 0), (1, 1, 0))   # eye == target
    assert e.value.code == -1
