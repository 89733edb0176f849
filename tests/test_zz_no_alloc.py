"""The allocation-free forward transform (ch_transform_forward_noalloc) against ch_transform_forward.

ch_transform_forward_noalloc exists for callers that must not allocate device memory when they
transform a field (for example a plug-in whose host application's memory pool owns the GPU, or a
fixed-latency loop that must stay out of the allocator).  It works in a fixed static device array
instead of buffers from an allocator, and equals the handle path to rounding (its twiddles come
from the device's sincospi).  This file is collected last so that a run stopping at the first
failure has run every other test first; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_forward_matches_handle_path_on_two_calls(binding):
    rng = np.random.default_rng(2024)
    # two calls in a row, the second on a different grid, each checked against the handle path
    for nx, ny, nz in ((32, 32, 33), (24, 36, 25)):
        phys = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
        spec = torch.empty((nx // 2, ny, nz), dtype=torch.complex128, device="cuda")
        binding.transform_forward_noalloc(phys, spec)
        g = binding.Grid(nx, ny, nz)
        ref = g.transform_forward(phys)
        torch.cuda.synchronize()
        assert rel(spec, ref) < 1e-13
        g.close()


def test_noalloc_rejects_grids_beyond_its_scratch(binding):
    assert binding.lib().ch_noalloc_scratch_bytes() == 64 << 20
    nx, ny, nz = 192, 192, 257     # two (96, 192, 257) complex work fields exceed 64 MiB
    phys = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    spec = torch.empty((nx // 2, ny, nz), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.ChError) as e:
        binding.transform_forward_noalloc(phys, spec)
    assert e.value.code == -2


def test_noalloc_forward_replays_in_a_captured_graph(binding):
    """The call inside CUDA-graph stream capture: one uncaptured call first (it looks up the
    static array's address and settles the kernels' shared-memory limits), then the call is
    captured once and replayed on new data copied into the same input tensor; each replay
    matches the handle path (and the two replays differ, so the graph reads its input anew)."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 32, 24, 33
    phys = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
    spec = torch.empty((nx // 2, ny, nz), dtype=torch.complex128, device="cuda")
    binding.transform_forward_noalloc(phys, spec)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        binding.transform_forward_noalloc(phys, spec)
    g = binding.Grid(nx, ny, nz)
    outs = []
    for seed in (12, 13):
        src = torch.from_numpy(np.random.default_rng(seed).standard_normal((nz, ny, nx))).cuda()
        phys.copy_(src)
        graph.replay()
        torch.cuda.synchronize()
        ref = g.transform_forward(src)
        torch.cuda.synchronize()
        assert rel(spec, ref) < 1e-13
        outs.append(spec.clone())
    assert not torch.equal(outs[0], outs[1])
    g.close()
