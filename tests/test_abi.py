"""The C-ABI library builds, loads without a GPU, and exports every function include/*.h declares.

No compute call is made here (no GPU on this runner)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ch_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_01322_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ch_init_grid", "ch_set_fields", "ch_step", "ch_get_fields",
                     "ch_diagnostics", "ch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    from paper_2406_01322_gb300 import binding
    assert set(declared_functions()) <= set(binding._SIGS)
    lib = binding.load_library(libpath)
    assert lib.ch_status_string(-2) == b"unsupported grid size"


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2406_01322_gb300 import binding
    with pytest.raises(RuntimeError):
        binding.load_library(str(tmp_path / "nope.so"))


def test_noalloc_binding_rejects_host_tensors_before_the_library_call(libpath):
    """A host tensor's pointer must never reach the device kernels: the binding checks that
    both tensors are CUDA tensors on one device before it calls the library."""
    import torch
    from paper_2406_01322_gb300 import binding
    phys = torch.zeros((17, 16, 16), dtype=torch.float64)
    spec = torch.zeros((8, 16, 17), dtype=torch.complex128)
    with pytest.raises(ValueError):
        binding.transform_forward_noalloc(phys, spec)


def _params(binding, **kw):
    p = dict(nx=16, ny=16, nz=17, lx=4.0 * 3.141592653589793, ly=2.0 * 3.141592653589793,
             re_tau=150.0, we=1.0, ch=0.05, pe=20.0, dt=1e-4, gx=0.0, gy=0.0, precision=0,
             dealias_z=0, bc=0)
    p.update(kw)
    return binding.Params(**p)


def test_invalid_grids_are_rejected_before_any_device_call(libpath):
    """ch_init_grid validates sizes and parameters on the host, before it touches the device, so
    the checks run here without a GPU: CH_ERR_SIZE (-2) for the size rules of the header (nx, ny
    even with 3nx/2, 3ny/2 {2,3}-smooth; nz - 1 even and {2,3}-smooth), CH_ERR_ARG (-1) for
    non-positive physical parameters, unknown precision or wall codes, a z dealiasing request,
    and an allocator given without its free function; the out-handle stays NULL."""
    from paper_2406_01322_gb300 import binding
    lib = binding.load_library(libpath)
    cases = [(dict(nx=14), -2),            # 3 nx / 2 = 21 = 3 * 7
             (dict(ny=10), -2),            # 3 ny / 2 = 15 = 3 * 5
             (dict(nx=15), -2),            # odd
             (dict(nz=16), -2),            # nz - 1 odd
             (dict(nz=15), -2),            # nz - 1 = 14 = 2 * 7
             (dict(nz=3), -2),             # too short a Chebyshev line
             (dict(re_tau=0.0), -1), (dict(we=-1.0), -1), (dict(ch=0.0), -1),
             (dict(pe=float("nan")), -1), (dict(dt=0.0), -1), (dict(lx=-1.0), -1),
             (dict(precision=3), -1), (dict(bc=4), -1), (dict(bc=-1), -1),
             (dict(dealias_z=1), -1)]
    for kw, code in cases:
        p = _params(binding, **kw)
        out = ctypes.c_void_p(1234)
        r = lib.ch_init_grid(ctypes.byref(p), binding.ALLOC_FN(), binding.FREE_FN(), None, None,
                             ctypes.byref(out))
        assert r == code, kw
        assert out.value is None, kw
    alloc = binding.ALLOC_FN(lambda n, ctx: None)
    p = _params(binding)
    out = ctypes.c_void_p()
    assert lib.ch_init_grid(ctypes.byref(p), alloc, binding.FREE_FN(), None, None,
                            ctypes.byref(out)) == -1


def test_null_handles_and_arguments_are_rejected(libpath):
    """Every entry point that takes a handle answers a NULL one with CH_ERR_ARG (or the neutral
    value of a query) instead of dereferencing it."""
    from paper_2406_01322_gb300 import binding
    lib = binding.load_library(libpath)
    assert lib.ch_step(None, 1) == -1
    assert lib.ch_set_fields(None, None, None, None, None) == -1
    assert lib.ch_get_chebyshev(None) == -1
    assert lib.ch_get_fft_pruning(None) == -1
    assert lib.ch_launches_per_step(None) == 0
    assert lib.ch_ensemble_size(None) == 0
    assert lib.ch_ensemble_get_chebyshev(None) == -1
    # the allocation-free transform: NULL pointers, then a size the rules reject
    assert lib.ch_transform_forward_noalloc(16, 16, 17, None, None, None) == -1
    assert lib.ch_transform_forward_noalloc(14, 16, 17, ctypes.c_void_p(16),
                                            ctypes.c_void_p(16), None) == -2
    # an ensemble of no members, and one whose members mix precisions
    out = ctypes.c_void_p()
    ps = (binding.Params * 2)(_params(binding), _params(binding, precision=1))
    assert lib.ch_ensemble_init(ps, 0, binding.ALLOC_FN(), binding.FREE_FN(), None, None,
                                ctypes.byref(out)) == -1
    assert lib.ch_ensemble_init(ps, 2, binding.ALLOC_FN(), binding.FREE_FN(), None, None,
                                ctypes.byref(out)) == -1
