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
