"""Failure detection without faulting the GPU: a state carrying NaN is reported as diverged, an
allocator that fails part-way through ch_init_grid surfaces as CH_ERR_ALLOC with everything
already obtained released, invalid arguments are rejected on the host, and a bounded device wait
that runs out returns CH_ERR_TIMEOUT with the context intact."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def test_nan_state_is_reported_as_diverged(binding):
    f = [np.array(a) for a in inputs.initial_fields(16, 16, 17, 150.0, 0.05, 1, 0.4, 1)]
    f[0][3, 2, 1] = math.nan
    g = binding.Grid(16, 16, 17)
    g.set_fields(*[torch.from_numpy(a) for a in f])
    g.step(2)                                  # runs to completion, no device-side trap
    d = g.diagnostics()                        # CH_ERR_DIVERGED is returned with the record
    assert d["nan"] == 1
    code = binding.lib().ch_diagnostics(g.h, binding.ctypes.byref(binding.Diag()))
    assert code == -5


def test_allocator_failure_surfaces_as_alloc_error(binding):
    class Failing(binding.TorchAllocator):
        """torch-backed allocator that returns NULL from the k-th request on"""

        def __init__(self, device, k):
            super().__init__(device)
            self.k, self.n, self.freed = k, 0, 0

        def _alloc(self, nbytes, ctx):
            self.n += 1
            return None if self.n >= self.k else super()._alloc(nbytes, ctx)

        def _free(self, ptr, ctx):
            self.freed += 1
            super()._free(ptr, ctx)

    for k in (1, 5, 12):
        a = Failing(torch.device("cuda:0"), k)
        with pytest.raises(binding.ChError) as e:
            binding.Grid(16, 16, 17, allocator=a)
        assert e.value.code == -3
        assert a.freed == k - 1 and not a.live       # every successful allocation released
    g = binding.Grid(16, 16, 17)                     # the library is still usable
    g.set_fields(*[torch.from_numpy(x) for x in inputs.initial_fields(16, 16, 17, 150.0, 0.05, 1, 0.4, 1)])
    g.step(1)
    assert g.diagnostics()["nan"] == 0


def test_invalid_arguments_are_rejected_on_the_host(binding):
    for kw, code in ((dict(re_tau=-1.0), -1), (dict(ch=0.0), -1), (dict(precision=7), -1),
                     (dict(bc=4), -1)):
        with pytest.raises(binding.ChError) as e:
            binding.Grid(16, 16, 17, **kw)
        assert e.value.code == code, kw
    for n in ((14, 16, 17), (16, 16, 16), (16, 10, 17)):   # nx = 2*7, nz - 1 odd, ny = 2*5
        with pytest.raises(binding.ChError) as e:
            binding.Grid(*n)
        assert e.value.code == -2, n


def test_bounded_device_wait_runs_out_and_reports_timeout(binding):
    """A loop of waits on mbarrier phases that nothing completes (the shape of the tensor-core
    kernel's pipeline): the first wait gives up after its bound (about one second) and every
    later one returns at once, so the whole loop ends within two bounds, not one bound per wait;
    the kernel records the failure and returns CH_ERR_TIMEOUT, and the context stays usable (a
    step runs afterwards)."""
    import ctypes
    import time
    spun = ctypes.c_int(-1)
    t0 = time.perf_counter()
    assert binding.lib().ch_selftest_bounded_wait(1, ctypes.byref(spun)) == -6
    one = time.perf_counter() - t0
    assert spun.value == 1 and 0.9 < one < 2.0, (spun.value, one)
    t0 = time.perf_counter()
    assert binding.lib().ch_selftest_bounded_wait(4096, ctypes.byref(spun)) == -6
    many = time.perf_counter() - t0
    assert spun.value == 1 and 0.9 < many < 2.0, (spun.value, many)
    assert binding.lib().ch_selftest_bounded_wait(0, None) == -1
    f = [torch.from_numpy(a) for a in inputs.initial_fields(16, 16, 17, 150.0, 0.05, 1, 0.4, 3)]
    g = binding.Grid(16, 16, 17)
    g.set_fields(*f)
    g.step(2)
    d = g.diagnostics()
    assert d["step"] == 2 and not d["nan"]
