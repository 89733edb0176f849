"""Thin ctypes binding of libchflow.so (include/ch_flow.h): argument marshalling only.

Every computation happens in the library's CUDA kernels.  PyTorch provides device memory (the
library's internal buffers come from torch's caching allocator through the allocator callbacks)
and the CUDA stream.  Importing this module loads the library and raises if it is missing; there
is no CPU fallback.
"""
import ctypes
import math
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchflow.so")

CH_OK = 0
STATUS = {0: "ok", -1: "CH_ERR_ARG", -2: "CH_ERR_SIZE", -3: "CH_ERR_ALLOC", -4: "CH_ERR_CUDA",
          -5: "CH_ERR_DIVERGED", -6: "CH_ERR_TIMEOUT", -7: "CH_ERR_STATE"}
PREC_FP64 = 0
PREC_MIXED = 1
PREC_DFLOAT = 2
BC_NO_SLIP = 0
BC_FREE_SLIP = 1
BC_NO_SLIP_BOTTOM_FREE_SLIP_TOP = 2
BC_FREE_SLIP_BOTTOM_NO_SLIP_TOP = 3
CHEB_FFT = 0
CHEB_TC = 1


class ChError(RuntimeError):
    def __init__(self, fn, code, detail=None):
        msg = f"{fn} failed: {STATUS.get(code, code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("re_tau", ctypes.c_double), ("we", ctypes.c_double), ("ch", ctypes.c_double),
                ("pe", ctypes.c_double), ("dt", ctypes.c_double), ("gx", ctypes.c_double),
                ("gy", ctypes.c_double), ("precision", ctypes.c_int), ("dealias_z", ctypes.c_int),
                ("bc", ctypes.c_int)]


class Diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_longlong), ("mass", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("grad2", ctypes.c_double),
                ("free_energy", ctypes.c_double), ("cfl", ctypes.c_double),
                ("max_phi", ctypes.c_double), ("nan", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# exported names of include/ch_flow.h and their signatures
_P = ctypes.c_void_p
_SIGS = {
    "ch_init_grid": (ctypes.c_int, [ctypes.POINTER(Params), ALLOC_FN, FREE_FN, _P, _P,
                                    ctypes.POINTER(_P)]),
    "ch_set_stream": (ctypes.c_int, [_P, _P]),
    "ch_set_fields": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ch_set_fields_host": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ch_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_step_timed": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "ch_launches_per_step": (ctypes.c_int, [_P]),
    "ch_get_fields": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ch_get_fields_host": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ch_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(Diag)]),
    "ch_state_bytes": (ctypes.c_size_t, [_P]),
    "ch_get_state": (ctypes.c_int, [_P, _P]),
    "ch_set_state": (ctypes.c_int, [_P, _P]),
    "ch_get_spectral": (ctypes.c_int, [_P, _P, _P, _P]),
    "ch_set_spectral": (ctypes.c_int, [_P, _P, _P, _P]),
    "ch_transform_forward": (ctypes.c_int, [_P, _P, _P]),
    "ch_transform_backward": (ctypes.c_int, [_P, _P, _P]),
    "ch_nonlinear": (ctypes.c_int, [_P, _P]),
    "ch_transform_forward_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    _P, _P, _P]),
    "ch_noalloc_scratch_bytes": (ctypes.c_size_t, []),
    "ch_render_interface": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                           ctypes.c_double]),
    "ch_objective": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ch_adjoint_begin": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ch_adjoint_step": (ctypes.c_int, [_P, _P]),
    "ch_adjoint_segment": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "ch_adjoint_step_timed": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ch_adjoint_gradient": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ch_adjoint_end": (ctypes.c_int, [_P]),
    "ch_ensemble_init": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ALLOC_FN, FREE_FN,
                                        _P, _P, ctypes.POINTER(_P)]),
    "ch_ensemble_size": (ctypes.c_int, [_P]),
    "ch_ensemble_member": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "ch_ensemble_step": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_ensemble_step_timed": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "ch_ensemble_autotune": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_ensemble_tuning": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "ch_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ch_fp64_fma_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "ch_ensemble_set_chebyshev": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_ensemble_get_chebyshev": (ctypes.c_int, [_P]),
    "ch_ensemble_destroy": (None, [_P]),
    "ch_destroy": (None, [_P]),
    "ch_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ch_last_cuda_error": (ctypes.c_char_p, []),
    "ch_set_chebyshev": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_set_fft_pruning": (ctypes.c_int, [_P, ctypes.c_int]),
    "ch_get_fft_pruning": (ctypes.c_int, [_P]),
    "ch_get_chebyshev": (ctypes.c_int, [_P]),
    "ch_chebyshev_lines": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int]),
    "ch_device_status": (ctypes.c_int, [_P]),
}


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2406_01322_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _ck(name, code):
    if code != CH_OK:
        detail = None
        if code == -4:
            detail = lib().ch_last_cuda_error().decode()
        raise ChError(name, code, detail)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def transform_forward_noalloc(phys, spec, stream=None):
    """Allocation-free forward transform into a caller-provided spectral tensor.

    phys: float64 CUDA tensor (nz, ny, nx); spec: complex128 CUDA tensor (nx/2, ny, nz) on the
    same device, which receives the coefficients.  The library allocates nothing for this call
    (its working memory is a fixed static device array); see ch_transform_forward_noalloc in
    include/ch_flow.h.  The call runs with phys's device current, on `stream` (default: that
    device's current stream)."""
    if phys.dim() != 3:
        raise ValueError("phys must be a (nz, ny, nx) tensor")
    nz, ny, nx = phys.shape
    if not (phys.is_cuda and spec.is_cuda) or spec.device != phys.device:
        raise ValueError("phys and spec must be CUDA tensors on the same device")
    if stream is not None and stream.device != phys.device:
        raise ValueError("stream must belong to phys's device")
    if not (phys.is_contiguous() and spec.is_contiguous()):
        raise ValueError("contiguous tensors required")
    if phys.dtype != torch.float64 or spec.dtype != torch.complex128:
        raise ValueError("phys must be float64 and spec complex128")
    if tuple(spec.shape) != (nx // 2, ny, nz):
        raise ValueError(f"spec must have shape {(nx // 2, ny, nz)}")
    with torch.cuda.device(phys.device):
        s = stream if stream is not None else torch.cuda.current_stream(phys.device)
        _ck("ch_transform_forward_noalloc",
            lib().ch_transform_forward_noalloc(nx, ny, nz, _ptr(phys), _ptr(spec),
                                               ctypes.c_void_p(s.cuda_stream)))
    return spec


def fp64_fma_rate():
    """Measured float64 FMA rate of the current device in TFLOP/s (ch_fp64_fma_rate)."""
    v = ctypes.c_double()
    _ck("ch_fp64_fma_rate", lib().ch_fp64_fma_rate(ctypes.byref(v)))
    return v.value


class TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device):
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except Exception:  # noqa: BLE001 - the C side sees NULL and returns CH_ERR_ALLOC
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, _ctx):
        self.live.pop(ptr, None)


class Grid:
    """One channel on one GPU.  Fields are torch float64 CUDA tensors shaped (nz, ny, nx);
    spectral arrays are complex128 tensors shaped (nx/2, ny, nz) ([mx][j][n] layout)."""

    def __init__(self, nx, ny, nz, re_tau=150.0, we=1.0, ch=0.05, pe=20.0, dt=1e-4,
                 lx=4 * math.pi, ly=2 * math.pi, gx=1.0, gy=0.0, precision=PREC_FP64,
                 device="cuda:0", stream=None, use_torch_allocator=True, bc=BC_NO_SLIP,
                 allocator=None):
        self.device = torch.device(device)
        self.shape = (nz, ny, nx)
        self.spec_shape = (nx // 2, ny, nz)
        self.params = Params(nx, ny, nz, lx, ly, re_tau, we, ch, pe, dt, gx, gy, precision, 0, bc)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        # allocator: an object with alloc_cb / free_cb (e.g. TorchAllocator); default: torch's
        # caching allocator, or the library's cudaMalloc when use_torch_allocator is False
        if allocator is not None:
            self._alloc = allocator
        else:
            self._alloc = TorchAllocator(self.device) if use_torch_allocator else None
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = lib().ch_init_grid(
                ctypes.byref(self.params),
                self._alloc.alloc_cb if self._alloc else ALLOC_FN(),
                self._alloc.free_cb if self._alloc else FREE_FN(),
                None, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _ck("ch_init_grid", code)
        self.h = h
        self._owned = True

    @classmethod
    def _view(cls, handle, params, device, stream):
        """A Grid over a handle owned elsewhere (an ensemble member); close() does not free it."""
        g = cls.__new__(cls)
        g.device = torch.device(device)
        g.shape = (params.nz, params.ny, params.nx)
        g.spec_shape = (params.nx // 2, params.ny, params.nz)
        g.params = params
        g.stream = stream
        g._alloc = None
        g.h = handle
        g._owned = False
        return g

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib().ch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _f64(self, a):
        t = torch.as_tensor(a, dtype=torch.float64, device=self.device).contiguous()
        if tuple(t.shape) != self.shape:
            raise ValueError(f"expected shape {self.shape}, got {tuple(t.shape)}")
        return t

    def set_fields(self, u, v, w, phi):
        ts = [self._f64(a) for a in (u, v, w, phi)]
        _ck("ch_set_fields", lib().ch_set_fields(self.h, *[_ptr(t) for t in ts]))
        self._keep = ts

    def set_fields_host(self, u, v, w, phi):
        """Host float64 arrays/tensors (C-contiguous); copies happen inside the library."""
        ts = [torch.as_tensor(a, dtype=torch.float64).contiguous() for a in (u, v, w, phi)]
        _ck("ch_set_fields_host", lib().ch_set_fields_host(self.h, *[_ptr(t) for t in ts]))

    def step(self, n=1):
        _ck("ch_step", lib().ch_step(self.h, int(n)))

    KERNELS = ("zrhs", "zsolve", "zbwd", "ybwd", "xline", "yfwd", "cheb_fwd", "cheb_bwd")

    def set_chebyshev(self, method):
        """CHEB_FFT (default) or CHEB_TC: how the step does its Chebyshev transforms."""
        _ck("ch_set_chebyshev", lib().ch_set_chebyshev(self.h, int(method)))

    def chebyshev(self):
        return int(lib().ch_get_chebyshev(self.h))

    def set_fft_pruning(self, on):
        """Pruned x/y transforms of the 3/2-rule padding (1) or the default schedules (0)."""
        _ck("ch_set_fft_pruning", lib().ch_set_fft_pruning(self.h, int(on)))

    def fft_pruning(self):
        return int(lib().ch_get_fft_pruning(self.h))

    def chebyshev_lines(self, x, direction):
        """Chebyshev transform along z of complex lines x (nf, nx/2, ny, nz) complex128 on the
        device with the selected method: direction 0 samples -> coefficients, 1 the inverse."""
        x = x.contiguous()
        assert x.dtype == torch.complex128 and tuple(x.shape[1:]) == tuple(self.spec_shape)
        out = torch.empty_like(x)
        _ck("ch_chebyshev_lines", lib().ch_chebyshev_lines(self.h, int(direction), _ptr(x),
                                                           _ptr(out), int(x.shape[0])))
        return out

    def device_status(self):
        """Synchronise; raises ChError(CH_ERR_TIMEOUT) if a bounded device wait gave up."""
        _ck("ch_device_status", lib().ch_device_status(self.h))

    def step_timed(self, n):
        """n steps with CUDA events between launches; returns (total_ms, per-kernel summed ms in
        the order of Grid.KERNELS).  Synchronises the stream."""
        ks = (ctypes.c_double * len(self.KERNELS))()
        tot = ctypes.c_double()
        _ck("ch_step_timed", lib().ch_step_timed(self.h, int(n), ks, ctypes.byref(tot)))
        return tot.value, list(ks)

    def launches_per_step(self):
        return int(lib().ch_launches_per_step(self.h))

    def get_fields(self):
        outs = [torch.empty(self.shape, dtype=torch.float64, device=self.device) for _ in range(4)]
        _ck("ch_get_fields", lib().ch_get_fields(self.h, *[_ptr(t) for t in outs]))
        return outs

    def get_fields_host(self, outs=None):
        if outs is None:
            outs = [torch.empty(self.shape, dtype=torch.float64).pin_memory() for _ in range(4)]
        _ck("ch_get_fields_host", lib().ch_get_fields_host(self.h, *[_ptr(t) for t in outs]))
        return outs

    def diagnostics(self):
        d = Diag()
        code = lib().ch_diagnostics(self.h, ctypes.byref(d))
        if code not in (CH_OK, -5):
            _ck("ch_diagnostics", code)
        return {k: getattr(d, k) for k, _ in Diag._fields_}

    def state_bytes(self):
        return int(lib().ch_state_bytes(self.h))

    def get_state(self):
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _ck("ch_get_state", lib().ch_get_state(self.h, _ptr(buf)))
        return buf

    def set_state(self, buf):
        _ck("ch_set_state", lib().ch_set_state(self.h, _ptr(buf)))

    def get_spectral(self):
        outs = [torch.empty(self.spec_shape, dtype=torch.complex128, device=self.device)
                for _ in range(3)]
        _ck("ch_get_spectral", lib().ch_get_spectral(self.h, *[_ptr(t) for t in outs]))
        return outs

    def set_spectral(self, om, w, phi):
        ts = [torch.as_tensor(a, dtype=torch.complex128, device=self.device).contiguous()
              for a in (om, w, phi)]
        _ck("ch_set_spectral", lib().ch_set_spectral(self.h, *[_ptr(t) for t in ts]))
        self._keep = ts

    def transform_forward(self, phys):
        f = self._f64(phys)
        out = torch.empty(self.spec_shape, dtype=torch.complex128, device=self.device)
        _ck("ch_transform_forward", lib().ch_transform_forward(self.h, _ptr(f), _ptr(out)))
        return out

    def transform_backward(self, spec):
        s = torch.as_tensor(spec, dtype=torch.complex128, device=self.device).contiguous()
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        _ck("ch_transform_backward", lib().ch_transform_backward(self.h, _ptr(s), _ptr(out)))
        return out

    def nonlinear(self):
        out = torch.empty((9,) + self.spec_shape, dtype=torch.complex128, device=self.device)
        _ck("ch_nonlinear", lib().ch_nonlinear(self.h, _ptr(out)))
        return out

    def render_interface(self, width, height, eye, target, up=(0.0, 0.0, 1.0), fov_deg=40.0,
                         step=0.0):
        """Image of the interface phi = 0: (rgb uint8 (height, width, 3), depth float64
        (height, width), -1 where the ray misses), both CUDA tensors."""
        rgb = torch.empty((height, width, 3), dtype=torch.uint8, device=self.device)
        depth = torch.empty((height, width), dtype=torch.float64, device=self.device)
        cam = (ctypes.c_double * 9)(*(list(eye) + list(target) + list(up)))
        _ck("ch_render_interface", lib().ch_render_interface(
            self.h, _ptr(rgb), _ptr(depth), int(width), int(height), cam, float(fov_deg),
            float(step)))
        return rgb, depth

    # ---- discrete adjoint (float64 grids) ----
    def objective(self):
        """J = 1/2 int |u|^2 + int |grad phi|^2 of the current state (a Python float)."""
        J = ctypes.c_double()
        _ck("ch_objective", lib().ch_objective(self.h, ctypes.byref(J)))
        return J.value

    def adjoint_begin(self):
        """Seed the reverse sweep with dJ/ds of the current (final) state; returns J."""
        J = ctypes.c_double()
        _ck("ch_adjoint_begin", lib().ch_adjoint_begin(self.h, ctypes.byref(J)))
        return J.value

    def adjoint_step(self, state):
        """Reverse the forward step that started from `state` (a get_state() buffer)."""
        _ck("ch_adjoint_step", lib().ch_adjoint_step(self.h, _ptr(state)))

    def adjoint_segment(self, checkpoint, nsteps):
        """Reverse the nsteps forward steps that follow `checkpoint` (a get_state() buffer):
        recomputation and reverse sweep in one library call."""
        _ck("ch_adjoint_segment", lib().ch_adjoint_segment(self.h, _ptr(checkpoint), int(nsteps)))

    ADJ_KERNELS = ("zbwd", "ybwd", "adj_zsolve", "adj_zrhs", "adj_ybwd", "adj_xline",
                   "adj_yfwd", "fold_dy", "adj_zbwd")

    def adjoint_step_timed(self, state):
        """adjoint_step with CUDA events between its launches; returns per-kernel ms in the
        order of Grid.ADJ_KERNELS (synchronises the stream)."""
        ks = (ctypes.c_double * len(self.ADJ_KERNELS))()
        _ck("ch_adjoint_step_timed", lib().ch_adjoint_step_timed(self.h, _ptr(state), ks))
        return list(ks)

    def adjoint_gradient(self):
        """dJ/d(u0, v0, w0, phi0) after the first forward step was reversed."""
        outs = [torch.empty(self.shape, dtype=torch.float64, device=self.device) for _ in range(4)]
        _ck("ch_adjoint_gradient", lib().ch_adjoint_gradient(self.h, *[_ptr(t) for t in outs]))
        return outs

    def adjoint_end(self):
        _ck("ch_adjoint_end", lib().ch_adjoint_end(self.h))


class ChannelObjective(torch.autograd.Function):
    """J(s_K) after K steps from the physical initial fields, differentiable in (u, v, w, phi).

    Forward: set_fields, K steps, J.  Saved: the state every `every` steps (checkpoints) and the
    final state.  Backward: segment by segment from the last, the library recomputes the segment
    from its checkpoint and reverses it (ch_adjoint_segment); the gradient of the first state
    maps back to the physical fields."""

    @staticmethod
    def forward(ctx, u, v, w, phi, grid, nsteps, every):
        every = max(1, int(every))
        grid.set_fields(u, v, w, phi)
        ckpts = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append(grid.get_state())
            grid.step(1)
        final = grid.get_state()
        J = grid.objective()
        ctx.grid, ctx.nsteps, ctx.every = grid, nsteps, every
        ctx.ckpts, ctx.final = ckpts, final
        ctx.devices = [(t.device, t.dtype) for t in (u, v, w, phi)]
        return torch.tensor(J, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        g, K, every = ctx.grid, ctx.nsteps, ctx.every
        g.set_state(ctx.final)
        g.adjoint_begin()
        try:
            for c in range(len(ctx.ckpts) - 1, -1, -1):
                n0 = c * every
                n1 = min(K, n0 + every)
                g.adjoint_segment(ctx.ckpts[c], n1 - n0)
            grads = g.adjoint_gradient()
        finally:
            g.adjoint_end()
        scale = gJ.to(dtype=torch.float64, device=grads[0].device)
        out = [(gr * scale).to(device=d, dtype=dt) for gr, (d, dt) in zip(grads, ctx.devices)]
        return out[0], out[1], out[2], out[3], None, None, None


def write_ppm(path, rgb):
    """Write an (height, width, 3) uint8 image (tensor or array) as a binary PPM file."""
    import numpy as np
    a = np.ascontiguousarray(rgb.cpu().numpy() if hasattr(rgb, "cpu") else rgb, dtype=np.uint8)
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (a.shape[1], a.shape[0]))
        f.write(a.tobytes())


def objective_after(grid, u, v, w, phi, nsteps, checkpoint_every=10):
    """J after `nsteps` steps of `grid` from (u, v, w, phi); differentiable through autograd."""
    return ChannelObjective.apply(u, v, w, phi, grid, int(nsteps), int(checkpoint_every))


class Ensemble:
    """Independent channels of uneven sizes advanced together by grouped persistent launches
    (one per stage, replayed from a CUDA graph).  members: list of dicts with the Grid keyword
    arguments (nx, ny, nz, re_tau, we, ch, pe, dt, ...); all members share one precision
    (`precision`, or a member's own "precision" key, which must then agree).
    ensemble.grids[i] is a Grid view of member i (set_fields, get_fields, diagnostics ...)."""

    def __init__(self, members, precision=PREC_FP64, device="cuda:0", stream=None):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = len(members)
        arr = (Params * n)()
        for i, m in enumerate(members):
            arr[i] = Params(m["nx"], m["ny"], m["nz"], m.get("lx", 4 * math.pi),
                            m.get("ly", 2 * math.pi), m.get("re_tau", 150.0), m.get("we", 1.0),
                            m.get("ch", 0.05), m.get("pe", 20.0), m.get("dt", 1e-4),
                            m.get("gx", 1.0), m.get("gy", 0.0), m.get("precision", precision), 0,
                            m.get("bc", BC_NO_SLIP))
        self._params = arr
        self._alloc = TorchAllocator(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = lib().ch_ensemble_init(arr, n, self._alloc.alloc_cb, self._alloc.free_cb, None,
                                          ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(h))
        _ck("ch_ensemble_init", code)
        self.h = h
        self.grids = []
        for i in range(n):
            gh = ctypes.c_void_p()
            _ck("ch_ensemble_member", lib().ch_ensemble_member(self.h, i, ctypes.byref(gh)))
            self.grids.append(Grid._view(gh, arr[i], self.device, self.stream))

    def step(self, n=1):
        _ck("ch_ensemble_step", lib().ch_ensemble_step(self.h, int(n)))

    STAGES = ("zrhs", "zsolve", "zbwd", "ybwd", "xline", "yfwd")

    def step_timed(self, n):
        ks = (ctypes.c_double * len(self.STAGES))()
        tot = ctypes.c_double()
        _ck("ch_ensemble_step_timed", lib().ch_ensemble_step_timed(self.h, int(n), ks,
                                                                   ctypes.byref(tot)))
        return tot.value, list(ks)

    def autotune(self, reps=2):
        _ck("ch_ensemble_autotune", lib().ch_ensemble_autotune(self.h, int(reps)))
        return self.tuning()

    def set_chebyshev(self, method):
        """CHEB_FFT or CHEB_TC for the grouped step (and every member); see ch_flow.h."""
        _ck("ch_ensemble_set_chebyshev", lib().ch_ensemble_set_chebyshev(self.h, int(method)))

    def chebyshev(self):
        return int(lib().ch_ensemble_get_chebyshev(self.h))

    def tuning(self):
        import json
        buf = ctypes.create_string_buffer(1024)
        _ck("ch_ensemble_tuning", lib().ch_ensemble_tuning(self.h, buf, 1024))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "h", None):
            for g in self.grids:
                g.h = None
            lib().ch_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
