"""Pins of the oracle's spectral assembly (``Channel.assemble``) and of its diagnostics against
closed-form derivatives of band-limited fields.

The assembly turns the non-linear coefficient arrays into the explicit terms of the three
implicit problems (Sec. 2.2):

* S_i = d_j Sigma_ij, the divergence of the momentum flux and Korteweg stress (Eqs. (NSE),
  (kort));
* h_omega = d_x S_y - d_y S_x (Eq. (omegaz)), h_w = lap S_z - d_z div S (Eq. (ww));
* S_phi = -div(u phi) + (1/Pe) lap(phi^3 - (1 + shat) phi) (Eq. (CHE) with the split of
  Eq. (phisplit));
* on the mean line kx = ky = 0: the x and y means of S_x, S_y plus the pressure gradient.

The fields here are finite sums of Fourier modes times polynomials in z of degree <= N, written
down term by term (``Field``): their derivatives are exact (numpy.polynomial's chebder for d/dz,
cos/sin swaps for d/dx and d/dy), so every coefficient the assembly produces is fixed up to
rounding.  Independently, a radially symmetric phase field exerts a Korteweg force that is a
gradient (kappa (1/2 grad |grad phi|^2 - lap(phi) grad phi) with lap(phi) and phi both functions
of r), so its curls h_omega and h_w vanish up to the truncation of the discretisation: that pins
the non-linear products and the assembly together.
"""
import inspect
import math
import textwrap
import types

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import chebyshev as cheb
from oracle.channel import Channel, Params


class Field:
    """sum over terms of A(z) cos(kx x + ky y) + B(z) sin(kx x + ky y), A and B Chebyshev series.

    Terms are keyed by the integer modes (mx >= 0, my); kx = 2 pi mx / Lx, ky = 2 pi my / Ly."""

    def __init__(self, p, terms=None):
        self.p = p
        self.terms = {} if terms is None else terms

    def k(self, mx, my):
        return 2 * math.pi * mx / self.p.lx, 2 * math.pi * my / self.p.ly

    def _map(self, fn):
        return Field(self.p, {key: fn(key, A, B) for key, (A, B) in self.terms.items()})

    def __add__(self, o):
        t = dict(self.terms)
        for key, (A, B) in o.terms.items():
            if key in t:
                a0, b0 = t[key]
                t[key] = (npc.chebadd(a0, A), npc.chebadd(b0, B))
            else:
                t[key] = (A, B)
        return Field(self.p, t)

    def __neg__(self):
        return self._map(lambda key, A, B: (-A, -B))

    def __sub__(self, o):
        return self + (-o)

    def scale(self, s):
        return self._map(lambda key, A, B: (s * A, s * B))

    def dx(self):
        # d/dx [A cos + B sin] = kx (B cos - A sin)
        return self._map(lambda key, A, B: (self.k(*key)[0] * B, -self.k(*key)[0] * A))

    def dy(self):
        return self._map(lambda key, A, B: (self.k(*key)[1] * B, -self.k(*key)[1] * A))

    def dz(self):
        return self._map(lambda key, A, B: (npc.chebder(A), npc.chebder(B)))

    def lap(self):
        return self.dx().dx() + self.dy().dy() + self.dz().dz()

    def coefficients(self):
        """The oracle's (Nz, Ny, Mx) complex coefficient array of this real field.

        A cos t + B sin t = Re[(A - i B) e^{i t}]: the mode (mx > 0, my) stores (A - i B) / 2 (its
        mirror -mx is implied by Hermitian symmetry); mx = 0 stores (A - i B) / 2 at my and its
        conjugate at -my; the mean mode stores A."""
        p = self.p
        out = np.zeros((p.nz, p.ny, p.nx // 2), complex)
        for (mx, my), (A, B) in self.terms.items():
            a = np.zeros(p.nz, complex)
            n = min(len(A), p.nz)
            a[:n] += A[:n]
            n = min(len(B), p.nz)
            a[:n] -= 1j * B[:n]
            assert np.all(np.abs(A[p.nz:]) == 0) and np.all(np.abs(B[p.nz:]) == 0)
            if mx == 0 and my == 0:
                out[:, 0, 0] += a.real
            elif mx == 0:
                out[:, my % p.ny, 0] += a / 2
                out[:, (-my) % p.ny, 0] += np.conj(a) / 2
            else:
                out[:, my % p.ny, mx] += a / 2
        return out

    def values(self, X, Y, Z):
        out = 0.0
        for (mx, my), (A, B) in self.terms.items():
            kx, ky = self.k(mx, my)
            t = kx * X + ky * Y
            out = out + npc.chebval(Z, A) * np.cos(t) + npc.chebval(Z, B) * np.sin(t)
        return out


def random_field(p, rng, modes, deg):
    terms = {}
    for (mx, my) in modes:
        A = rng.standard_normal(deg + 1)
        B = rng.standard_normal(deg + 1) if (mx, my) != (0, 0) else np.zeros(deg + 1)
        terms[(mx, my)] = (A, B)
    return Field(p, terms)


MODES = [(0, 0), (1, 0), (0, 1), (0, 2), (1, 1), (2, -1), (3, -3), (1, 3)]


def params():
    return Params(nx=8, ny=8, nz=13, ch=0.07, pe=13.0, we=2.5, dt=3e-4, gx=1.0, gy=0.25)


def test_field_coefficients_follow_the_oracle_convention():
    """The coefficient layout used below agrees with a direct evaluation of the field on the
    collocation grid (the oracle's backward transform, itself pinned by brute-force sums)."""
    p = params()
    c = Channel(p)
    f = random_field(p, np.random.default_rng(1), MODES, p.nz - 1)
    x = np.arange(p.nx) * p.lx / p.nx
    y = np.arange(p.ny) * p.ly / p.ny
    z = cheb.points(p.nz - 1)
    vals = f.values(x[None, None, :], y[None, :, None], z[:, None, None])
    got = c.spectral_to_physical(f.coefficients())
    assert np.max(np.abs(got - vals)) < 1e-12 * np.max(np.abs(vals))


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def assembly_case(seed=3):
    p = params()
    c = Channel(p)
    rng = np.random.default_rng(seed)
    deg = p.nz - 1
    names = ("sxx", "syy", "szz", "sxy", "sxz", "syz", "p3", "fu", "fv", "fw")
    F = {n: random_field(p, rng, MODES, deg) for n in names}
    phi = random_field(p, rng, MODES, deg)
    c.phi = phi.coefficients()
    nl = [F[n].coefficients() for n in names]
    # the physics, written with the Field algebra
    Sx = F["sxx"].dx() + F["sxy"].dy() + F["sxz"].dz()
    Sy = F["sxy"].dx() + F["syy"].dy() + F["syz"].dz()
    Sz = F["sxz"].dx() + F["syz"].dy() + F["szz"].dz()
    divS = Sx.dx() + Sy.dy() + Sz.dz()
    h_om = Sy.dx() - Sx.dy()
    h_w = Sz.lap() - divS.dz()
    G = F["p3"] - phi.scale(1.0 + c.shat)
    s_phi = -(F["fu"].dx() + F["fv"].dy() + F["fw"].dz()) + G.lap().scale(1.0 / p.pe)
    ref_om = h_om.coefficients()
    ref_w = h_w.coefficients()
    # mean line: the (0,0) parts of S_x and S_y plus the driving pressure gradient (gx, gy)
    sx0 = Sx.coefficients()[:, 0, 0].real
    sy0 = Sy.coefficients()[:, 0, 0].real
    ref_om[:, 0, 0] = sx0 + 1j * sy0
    ref_om[0, 0, 0] += p.gx + 1j * p.gy
    ref_w[:, 0, 0] = 0.0
    return c, nl, (ref_om, ref_w, s_phi.coefficients())


def test_assembly_matches_closed_form_derivatives():
    c, nl, ref = assembly_case()
    got = c.assemble(nl)
    for g, r, name in zip(got, ref, ("h_omega", "h_w", "S_phi")):
        assert rel_err(g, r) < 1e-12, name
    # the mean line on its own (its scale is far below that of the whole field)
    assert np.max(np.abs(got[0][:, 0, 0] - ref[0][:, 0, 0])) < 1e-12 * np.max(np.abs(ref[0][:, 0, 0]))
    assert np.all(got[1][:, 0, 0] == 0)


def test_assembly_pin_catches_sign_and_index_mistakes():
    """Plant each plausible mistake (a flipped sign, a swapped index, a dropped term) in a copy of
    the oracle's assembly on the CPU: the pin above must fail for every one of them."""
    src = textwrap.dedent(inspect.getsource(Channel.assemble))
    mutants = [
        ("Sx = ikx * sxx + iky * sxy", "Sx = ikx * sxx - iky * sxy"),
        ("Sx = ikx * sxx + iky * sxy + self.dz(sxz)", "Sx = ikx * sxx + iky * sxy - self.dz(sxz)"),
        ("Sx = ikx * sxx", "Sx = -ikx * sxx"),
        ("Sy = ikx * sxy + iky * syy", "Sy = ikx * sxy - iky * syy"),
        ("Sy = ikx * sxy", "Sy = ikx * sxz"),
        ("iky * syy + self.dz(syz)", "iky * syy - self.dz(syz)"),
        ("Sz = ikx * sxz + iky * syz + self.dz(szz)", "Sz = ikx * sxz + iky * syz - self.dz(szz)"),
        ("Sz = ikx * sxz", "Sz = -ikx * sxz"),
        ("Sz = ikx * sxz + iky * syz", "Sz = ikx * sxz - iky * syz"),
        ("h_om = ikx * Sy - iky * Sx", "h_om = ikx * Sy + iky * Sx"),
        ("h_om = ikx * Sy - iky * Sx", "h_om = iky * Sy - ikx * Sx"),
        ("h_w = -k2 * Sz - self.dz(", "h_w = k2 * Sz - self.dz("),
        ("h_w = -k2 * Sz - self.dz(", "h_w = -k2 * Sz + self.dz("),
        ("self.dz(ikx * Sx + iky * Sy)", "self.dz(ikx * Sx - iky * Sy)"),
        ("Sx[:, 0, 0].real + 1j * Sy[:, 0, 0].real", "Sx[:, 0, 0].real - 1j * Sy[:, 0, 0].real"),
        ("(self.p.gx + 1j * self.p.gy)", "(self.p.gx - 1j * self.p.gy)"),
        ("G = p3 - (1.0 + self.shat) * self.phi", "G = p3 + (1.0 + self.shat) * self.phi"),
        ("G = p3 - (1.0 + self.shat) * self.phi", "G = p3 - self.shat * self.phi"),
        ("-(ikx * fu + iky * fv + self.dz(fw))", "(ikx * fu + iky * fv + self.dz(fw))"),
        ("-(ikx * fu + iky * fv + self.dz(fw))", "-(ikx * fu - iky * fv + self.dz(fw))"),
        ("-(ikx * fu + iky * fv + self.dz(fw))", "-(ikx * fu + iky * fv - self.dz(fw))"),
        ("self.dz(self.dz(G)) - k2 * G", "self.dz(self.dz(G)) + k2 * G"),
        ("(1.0 / self.p.pe)", "(-1.0 / self.p.pe)"),
    ]
    c, nl, ref = assembly_case()
    ns = {}
    module = inspect.getmodule(Channel)
    for old, new in mutants:
        assert old in src, old
        code = src.replace(old, new, 1)
        ns.clear()
        exec(compile(code, "<mutant>", "exec"), module.__dict__, ns)
        fn = types.MethodType(ns["assemble"], c)
        got = fn(nl)
        worst = max(rel_err(g, r) for g, r in zip(got, ref))
        mean = np.max(np.abs(got[0][:, 0, 0] - ref[0][:, 0, 0])) / np.max(np.abs(ref[0][:, 0, 0]))
        assert max(worst, mean) > 1e-6, (old, new)


def test_korteweg_force_of_a_radial_drop_has_no_curl():
    """phi(r) radially symmetric, u = 0: the capillary force is a gradient, so h_omega and h_w
    (both curls of S) vanish to the truncation of the discretisation while S itself does not;
    a sign slip in one Korteweg component breaks the gradient structure by O(1)."""
    p = Params(nx=64, ny=32, nz=33, ch=0.1, we=1.0, pe=10.0, dt=1e-4, gx=0.0)
    c = Channel(p)
    x = np.arange(p.nx) * p.lx / p.nx
    y = np.arange(p.ny) * p.ly / p.ny
    z = cheb.points(p.nz - 1)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    r2 = (X - p.lx / 2) ** 2 + (Y - p.ly / 2) ** 2 + Z ** 2
    phi = np.exp(-r2 / 0.6 ** 2) + 0 * X + 0 * Y
    zero = np.zeros_like(phi)
    c.set_fields(zero, zero, zero, phi)
    nl = c.nonlinear_spectral()
    h_om, h_w, _ = c.assemble(nl)
    k2 = c.k2[None]
    Sx = c.ikx * nl[0] + c.iky * nl[3] + c.dz(nl[4])
    Sy = c.ikx * nl[3] + c.iky * nl[1] + c.dz(nl[5])
    scale_om = np.max(np.abs(c.ikx * Sy)) + np.max(np.abs(c.iky * Sx))
    Sz = c.ikx * nl[4] + c.iky * nl[5] + c.dz(nl[2])
    scale_w = np.max(np.abs(k2 * Sz))
    h_om[:, 0, 0] = 0.0          # the mean line carries the mean forcing, not a curl
    # truncation level of this resolution: 2e-9 (h_omega) and 1.5e-8 (h_w) relative
    assert np.max(np.abs(h_om)) < 1e-7 * scale_om
    assert np.max(np.abs(h_w)) < 1e-7 * scale_w
    # the same drop with the Korteweg term of Sigma_xy flipped: the curls no longer vanish
    bad = list(nl)
    bad[3] = -nl[3]
    h_om_bad, h_w_bad, _ = c.assemble(bad)
    h_om_bad[:, 0, 0] = 0.0
    assert np.max(np.abs(h_om_bad)) > 1e-1 * scale_om
    assert np.max(np.abs(h_w_bad)) > 1e-1 * scale_w


def test_diagnostics_gradient_energy_and_cfl_closed_forms():
    """int |grad phi|^2 and the free energy of phi = a cos(kx x) (1 - z^2) + b sin(ky y) z and
    the CFL number of a uniform flow (U, V) (Sec. 2.1.1 free energy; CFL = dt max(|u|/dx +
    |v|/dy + |w|/dz_local))."""
    p = Params(nx=16, ny=8, nz=17, ch=0.05, dt=2e-4, gx=0.0)
    c = Channel(p)
    x = np.arange(p.nx) * p.lx / p.nx
    y = np.arange(p.ny) * p.ly / p.ny
    z = cheb.points(p.nz - 1)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    a, b = 0.7, -0.3
    kx, ky = 2 * math.pi / p.lx, 2 * math.pi / p.ly
    phi = a * np.cos(kx * X) * (1 - Z * Z) + b * np.sin(ky * Y) * Z + 0 * X * Y * Z
    U, V = 3.0, -1.5
    one = np.ones_like(phi)
    c.set_fields(U * one, V * one, 0 * one, phi)
    d = c.diagnostics()
    area = p.lx * p.ly
    # |grad phi|^2 averaged over x and y: cross terms average out
    # a^2 [kx^2 (1-z^2)^2 / 2 + 4 z^2 / 2] + b^2 [ky^2 z^2 / 2 + 1 / 2]; phi^4 reaches the
    # y mode 4 and x mode 4, which the uniform sums over 8 and 16 points still integrate exactly
    zi = lambda coef: npc.chebval(1.0, npc.chebint(coef)) - npc.chebval(-1.0, npc.chebint(coef))
    one_m_z2_sq = npc.poly2cheb([1, 0, -2, 0, 1])
    z2 = npc.poly2cheb([0, 0, 1])
    grad2 = area * (a * a * (kx * kx * zi(one_m_z2_sq) / 2 + 4 * zi(z2) / 2)
                    + b * b * (ky * ky * zi(z2) / 2 + 2.0 / 2))
    assert math.isclose(d["grad2"], grad2, rel_tol=1e-13)
    assert math.isclose(d["cfl"], p.dt * (abs(U) / (p.lx / p.nx) + abs(V) / (p.ly / p.ny)),
                        rel_tol=1e-13)
    assert math.isclose(d["kinetic"], 0.5 * (U * U + V * V) * 2 * area, rel_tol=1e-13)
    # the free energy's gradient part is Ch^2/2 of grad2 (the bulk part is checked in
    # test_diagnostics_closed_forms); here the difference of two amplitudes isolates it
    c2 = Channel(p)
    c2.set_fields(U * one, V * one, 0 * one, 2 * phi)
    d2 = c2.diagnostics()
    bulk = lambda dd: dd["free_energy"] - 0.5 * p.ch ** 2 * dd["grad2"]
    assert math.isclose(d2["grad2"], 4 * grad2, rel_tol=1e-13)
    # bulk part: int 1/4 (phi^2 - 1)^2 evaluated by brute force on a fine grid
    xf = np.arange(64) * p.lx / 64
    yf = np.arange(32) * p.ly / 32
    zg, wg = np.polynomial.legendre.leggauss(24)
    Xf, Yf, Zf = xf[None, None, :], yf[None, :, None], zg[:, None, None]
    for amp, dd in ((1.0, d), (2.0, d2)):
        ph = amp * (a * np.cos(kx * Xf) * (1 - Zf * Zf) + b * np.sin(ky * Yf) * Zf)
        ref = np.sum(0.25 * (ph * ph - 1.0) ** 2 * wg[:, None, None]) * (p.lx / 64) * (p.ly / 32)
        assert math.isclose(bulk(dd), ref, rel_tol=1e-12)
