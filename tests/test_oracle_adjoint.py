"""Pins of the oracle's discrete adjoint (``oracle.adjoint``): its float64 torch step is the numpy
oracle's step, its objective is the exact integral of the interpolants, and its reverse-mode
gradient agrees with central finite differences of the objective after several steps."""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest
import torch

from oracle import adjoint
from oracle import chebyshev as cheb
from oracle.channel import Channel, Params
from paper_2406_01322_gb300 import inputs

P = dict(nx=12, ny=8, nz=9, re_tau=50.0, ch=0.15, pe=10.0, we=1.0, dt=2e-3)


def fields(p, seed=3):
    return inputs.initial_fields(p.nx, p.ny, p.nz, p.re_tau, p.ch, 1, 0.6, seed, amp=0.5)


def test_torch_step_equals_numpy_oracle():
    p = Params(**P)
    f = fields(p)
    c = Channel(p)
    c.set_fields(*f)
    t = adjoint.TorchChannel(p)
    st = t.set_fields(*[torch.tensor(a) for a in f])
    hist = None
    for _ in range(3):
        c.step()
        st, hist = t.step(st, hist)
    for a, b in zip(st, (c.omega, c.w, c.phi)):
        assert np.max(np.abs(a.numpy() - b)) < 1e-12 * max(1.0, np.max(np.abs(b)))


def test_objective_is_the_exact_integral():
    p = Params(**P)
    f = fields(p)
    t = adjoint.TorchChannel(p)
    st = t.set_fields(*[torch.tensor(a) for a in f])
    J = float(t.objective(st))
    # brute force: evaluate the interpolants on a grid fine enough for exact quadrature of
    # products (2x in x, y; 2N+1 Chebyshev-Gauss-Lobatto points in z)
    c = Channel(p)
    c.set_fields(*f)
    uh, vh, wh = c.velocity_spectral()
    ph = c.phi
    N2 = 2 * (p.nz - 1)
    zf = cheb.points(N2)
    wz = cheb.clenshaw_curtis_weights(N2)
    from oracle import fourier
    Ny2, Nx2 = 2 * p.ny, 2 * p.nx

    def phys(a):
        vals = np.stack([npc.chebval(zf, a[:, j, m]) for j in range(p.ny) for m in range(p.nx // 2)],
                        axis=-1).reshape(len(zf), p.ny, p.nx // 2)
        return fourier.from_modes(vals, Ny2, Nx2)

    dA = p.lx * p.ly / (Nx2 * Ny2)
    integ = lambda g: float(np.sum(g * wz[:, None, None]) * dA)
    u, v, w = phys(uh), phys(vh), phys(wh)
    fx, fy, fz = phys(c.ikx * ph), phys(c.iky * ph), phys(c.dz(ph))
    ref = 0.5 * integ(u * u + v * v + w * w) + integ(fx * fx + fy * fy + fz * fz)
    assert math.isclose(J, ref, rel_tol=1e-12)


@pytest.mark.parametrize("nsteps", [1, 3])
def test_gradient_matches_central_differences(nsteps):
    p = Params(**P)
    f = [np.ascontiguousarray(a) for a in fields(p)]
    J, g = adjoint.gradient(p, f, nsteps)
    rng = np.random.default_rng(100 + nsteps)
    for trial in range(3):
        d = [rng.standard_normal(a.shape) for a in f]
        eps = 1e-4   # central differences: O(eps^2) truncation, rounding ~ eps_mach J / eps
        jp = float(adjoint.objective_after(p, [torch.tensor(a + eps * b) for a, b in zip(f, d)], nsteps))
        jm = float(adjoint.objective_after(p, [torch.tensor(a - eps * b) for a, b in zip(f, d)], nsteps))
        fd = (jp - jm) / (2 * eps)
        an = sum(float(np.sum(gi * di)) for gi, di in zip(g, d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12 * abs(J)), (trial, fd, an)
