"""The full time step of the coupled Navier-Stokes + Cahn-Hilliard channel solver, plain FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What the paper fixes (Roccon, arXiv:2406.01322):

* Eq. (CHE) with the chemical potential mu = phi^3 - phi - Ch^2 lap(phi) (Sec. 2.1.1).
* Eqs. (cont), (NSE): incompressible NS, matched density and viscosity, with the capillary force
  of Eq. (kort), f = (3 / sqrt 8) (Ch / We) div(|grad phi|^2 I - grad phi (x) grad phi).
* Eqs. (omegaz), (ww), (omegadef): wall-normal vorticity omega_z (2nd order) and wall-normal
  velocity w (4th order, solved as a system of two Helmholtz problems); u, v from continuity and
  the definition of omega_z.
* Eq. (phisplit): the CH equation split with a coefficient s into two Helmholtz problems.
* Sec. 2.2: Fourier x Fourier x Chebyshev pseudo-spectral discretisation, non-linear terms in
  physical space, IMEX: Adams-Bashforth on non-linear terms, Crank-Nicolson on the NS linear terms,
  implicit Euler on the CH linear terms, step sequence i)-v).

Readings taken where the paper is silent or garbled (the CUDA path takes the same ones):

R1  The split coefficient: write shat = s Ch^2; implicit part (shat / Pe) lap(phi)
    - (Ch^2 / Pe) lap^2(phi); explicit part S_phi = -div(u phi) + (1/Pe) lap(phi^3 - (1+shat) phi).
    shat is the smallest value that makes the implicit-Euler operator a perfect square of one
    real Helmholtz operator: shat = 2 lam Ch^2, lam = sqrt(Pe / (Ch^2 dt)), so that
    (Ch^2/Pe) (lap - lam)^2 phi^{n+1} = phi^n / dt + AB2(S_phi).
R2  Adams-Bashforth is second order (3/2, -1/2); the first step after set_fields uses
    h^{n-1} = h^n (forward Euler on the non-linear terms).
R3  Crank-Nicolson for omega_z, theta = lap(w) and the mean flow; theta^n := (D^2 - k^2) w^n.
R4  Mean flow (kx = ky = 0): driven by a constant pressure gradient, -dp/dx = gx = 1, gy = 0;
    ubar, vbar obey (ubar)_t = Sbar_x + gx + (1/Re) ubar'' with ubar(+-1) = 0, and w_00 = 0.
    Sbar = real parts of the (0,0) Fourier coefficients of S_x, S_y.  The (0,0) line of the
    omega array carries U = ubar + i vbar, and its history carries Sbar_x + i Sbar_y + gx + i gy.
R5  Non-linear terms in divergence form: S_i = d_j(-u_i u_j + kappa T_ij),
    kappa = 3/sqrt(8) Ch/We, T_ij = |grad phi|^2 delta_ij - d_i phi d_j phi;
    CH convection in flux form -div(u phi).
R6  Dealiasing: 3/2 rule in x and y (zero padding), none in z; x and y Nyquist modes are zero.
R7  phi boundary conditions: d phi/dz = 0 for both split problems (no flux); velocity no-slip:
    u = v = w = dw/dz = 0, omega_z = 0 at z = +-1.
R8  Both S and S_phi are evaluated from (u^n, phi^n).
R9  Mass of phi = Lx Ly sum_{n even} 2 Re(phihat_00,n) / (1 - n^2) (exact integral).
R10 Chebyshev-tau with the Gottlieb-Orszag rows (``oracle.chebyshev``).
R13 Free-slip walls (Params.bc = 1; Sec. 2.1 allows no-slip or free-slip at the walls; the same
    condition at both walls): du/dz = dv/dz = 0 and w = 0, so d omega_z/dz = 0 and the mean flow
    takes Neumann rows; continuity then gives d2w/dz2 = 0, and the (theta, w) pair takes its four
    wall rows on w (w = w'' = 0), as for no-slip (w = w' = 0).  Params.bc = 2 / 3 combine the two
    (no-slip at z = -1 and free-slip at z = +1, or the reverse), each wall with its own rows.

State: omega (Nz, Ny, Mx), w, phi complex Chebyshev x Fourier coefficients, [n, j(my), mx].
"""
from dataclasses import dataclass
import math

import numpy as np

from . import chebyshev as cheb
from . import fourier


# wall conditions by Params.bc: (z = +1, z = -1)
WALLS = {0: ("no-slip", "no-slip"), 1: ("free-slip", "free-slip"),
         2: ("free-slip", "no-slip"), 3: ("no-slip", "free-slip")}


@dataclass
class Params:
    nx: int
    ny: int
    nz: int
    lx: float = 4.0 * math.pi
    ly: float = 2.0 * math.pi
    re_tau: float = 150.0
    we: float = 1.0
    ch: float = 0.05
    pe: float = 20.0
    dt: float = 1e-4
    gx: float = 1.0
    gy: float = 0.0
    bc: int = 0          # walls (Sec. 2.1): 0 no-slip, 1 free-slip (both walls), 2 no-slip at
                         # z = -1 and free-slip at z = +1, 3 free-slip at z = -1, no-slip at +1


class Channel:
    """FP64 oracle of one channel: set_fields / step / get_fields / diagnostics."""

    def __init__(self, p: Params):
        self.p = p
        self.N = p.nz - 1
        self.Mx = p.nx // 2
        self.Px = 3 * p.nx // 2
        self.Py = 3 * p.ny // 2
        kx, ky = fourier.wavenumbers(p.nx, p.ny, p.lx, p.ly)
        self.kx = kx
        self.ky = ky
        self.ikx = (1j * kx)[None, None, :]
        self.iky = (1j * ky)[None, :, None]
        self.k2 = (kx[None, :] ** 2 + ky[:, None] ** 2)  # (Ny, Mx)
        # time-scheme constants (R1, R3)
        self.beta = 2.0 * p.re_tau / p.dt
        self.lam = math.sqrt(p.pe / (p.ch ** 2 * p.dt))
        self.shat = 2.0 * self.lam * p.ch ** 2
        self.kappa = 3.0 / math.sqrt(8.0) * p.ch / p.we
        # Chebyshev operators
        self.Fm = cheb.forward_matrix(self.N)
        self.Bm = cheb.backward_matrix(self.N)
        self.D = cheb.deriv_matrix(self.N)
        shape = (p.nz, p.ny, self.Mx)
        self.omega = np.zeros(shape, complex)
        self.w = np.zeros(shape, complex)
        self.phi = np.zeros(shape, complex)
        self.hist = None
        self.t = 0.0
        self.nstep = 0

    # ---- helpers along the Chebyshev axis -------------------------------------------------
    def cheb_fwd(self, f):
        return np.tensordot(self.Fm, f, axes=(1, 0))

    def cheb_bwd(self, a):
        return np.tensordot(self.Bm, a, axes=(1, 0))

    def dz(self, a):
        return np.tensordot(self.D, a, axes=(1, 0))

    def physical_to_spectral(self, f, Nx=None, Ny=None):
        """(Nz, Py, Px) samples -> (Nz, Ny, Mx) coefficients (Fourier x, y then Chebyshev z)."""
        return self.cheb_fwd(fourier.to_modes(f, self.p.nx, self.p.ny))

    def spectral_to_physical(self, a, padded=False):
        """(Nz, Ny, Mx) coefficients -> (Nz, Py, Px) samples (unpadded grid unless padded)."""
        Py, Px = (self.Py, self.Px) if padded else (self.p.ny, self.p.nx)
        return fourier.from_modes(self.cheb_bwd(a), Py, Px)

    # ---- state <-> primitive fields ------------------------------------------------------
    def set_fields(self, u, v, w, phi):
        """Physical (Nz, Ny, Nx) fields -> (omega_z, w, U, phi) state; resets the AB2 history.

        omega_z = i kx v - i ky u (Eq. (omegadef)); the (0,0) line keeps U = ubar + i vbar (R4)."""
        uh = self.physical_to_spectral(u)
        vh = self.physical_to_spectral(v)
        wh = self.physical_to_spectral(w)
        ph = self.physical_to_spectral(phi)
        om = self.ikx * vh - self.iky * uh
        om[:, 0, 0] = uh[:, 0, 0].real + 1j * vh[:, 0, 0].real
        wh[:, 0, 0] = 0.0
        self.omega, self.w, self.phi = om, wh, ph
        self.hist = None

    def velocity_spectral(self, omega=None, w=None):
        """u, v from continuity (Eq. (cont)) and the omega_z definition (Eq. (omegadef)).

        i kx u + i ky v = -Dw and i kx v - i ky u = omega  =>
        u = (i kx Dw + i ky omega) / k^2,  v = (i ky Dw - i kx omega) / k^2  (k != 0)."""
        om = self.omega if omega is None else omega
        ww = self.w if w is None else w
        Dw = self.dz(ww)
        k2 = self.k2[None]
        safe = np.where(k2 > 0, k2, 1.0)
        uh = (self.ikx * Dw + self.iky * om) / safe
        vh = (self.iky * Dw - self.ikx * om) / safe
        uh[:, 0, 0] = om[:, 0, 0].real
        vh[:, 0, 0] = om[:, 0, 0].imag
        return uh, vh, ww

    def get_fields(self):
        """State -> physical (Nz, Ny, Nx) u, v, w, phi on the unpadded grid."""
        uh, vh, wh = self.velocity_spectral()
        return tuple(self.spectral_to_physical(a) for a in (uh, vh, wh, self.phi))

    # ---- step ii) / vi): non-linear terms in physical space -------------------------------
    def nonlinear_spectral(self):
        """The ten non-linear products (R5) on the 3/2-padded grid, returned as coefficients.

        Order: Sxx, Syy, Szz, Sxy, Sxz, Syz (Sigma_ij = -u_i u_j + kappa T_ij), phi^3,
        u phi, v phi, w phi."""
        uh, vh, wh = self.velocity_spectral()
        ph = self.phi
        fields = (uh, vh, wh, ph, self.ikx * ph, self.iky * ph, self.dz(ph))
        u, v, w, f, fx, fy, fz = (self.spectral_to_physical(a, padded=True) for a in fields)
        k = self.kappa
        g2 = fx * fx + fy * fy + fz * fz
        prods = (
            -u * u + k * (g2 - fx * fx),
            -v * v + k * (g2 - fy * fy),
            -w * w + k * (g2 - fz * fz),
            -u * v - k * fx * fy,
            -u * w - k * fx * fz,
            -v * w - k * fy * fz,
            f * f * f,
            u * f,
            v * f,
            w * f,
        )
        return [self.physical_to_spectral(q) for q in prods]

    def assemble(self, nl):
        """Spectral assembly of h_omega, h_w, S_phi from the non-linear coefficients.

        S_i = i kx Sigma_ix + i ky Sigma_iy + D Sigma_iz;
        h_omega = i kx S_y - i ky S_x                      (Eq. (omegaz));
        h_w = -k^2 S_z - D (i kx S_x + i ky S_y)            (Eq. (ww): lap S_z - d_z div S);
        S_phi = -(i kx (u phi) + i ky (v phi) + D (w phi)) + (1/Pe)(D^2 - k^2)(phi^3 - (1+shat) phi)."""
        sxx, syy, szz, sxy, sxz, syz, p3, fu, fv, fw = nl
        ikx, iky, k2 = self.ikx, self.iky, self.k2[None]
        Sx = ikx * sxx + iky * sxy + self.dz(sxz)
        Sy = ikx * sxy + iky * syy + self.dz(syz)
        Sz = ikx * sxz + iky * syz + self.dz(szz)
        h_om = ikx * Sy - iky * Sx
        h_w = -k2 * Sz - self.dz(ikx * Sx + iky * Sy)
        e0 = np.zeros(self.N + 1)
        e0[0] = 1.0
        h_om[:, 0, 0] = Sx[:, 0, 0].real + 1j * Sy[:, 0, 0].real + (self.p.gx + 1j * self.p.gy) * e0
        h_w[:, 0, 0] = 0.0
        G = p3 - (1.0 + self.shat) * self.phi
        s_phi = -(ikx * fu + iky * fv + self.dz(fw)) + (1.0 / self.p.pe) * (
            self.dz(self.dz(G)) - k2 * G)
        return h_om, h_w, s_phi

    # ---- steps iv) and v): implicit solves ---------------------------------------------------
    def rhs(self, H):
        """Literal right-hand sides of the three implicit problems (R1, R3).

        CN for omega:  (D^2 - k^2 - beta) om^{n+1} = -(D^2 - k^2 + beta) om^n - 2 Re H_om
        CN for theta:  (D^2 - k^2 - beta) th^{n+1} = -(D^2 - k^2 + beta) th^n - 2 Re H_w
        IE for phi:    (D^2 - k^2 - lam)^2 phi^{n+1} = (Pe/Ch^2)(phi^n / dt + H_phi)
        with beta = 2 Re / dt."""
        p = self.p
        k2 = self.k2[None]
        D2 = lambda a: self.dz(self.dz(a))
        om, w, ph = self.omega, self.w, self.phi
        H_om, H_w, H_phi = H
        r_om = -(D2(om) - k2 * om + self.beta * om) - 2.0 * p.re_tau * H_om
        th = D2(w) - k2 * w
        r_th = -(D2(th) - k2 * th + self.beta * th) - 2.0 * p.re_tau * H_w
        r_psi = (p.pe / p.ch ** 2) * (ph / p.dt + H_phi)
        return r_om, r_th, r_psi

    def solve_line(self, j, m, r_om, r_th, r_psi):
        """Solve the implicit problems of one (my, mx) line; returns (omega, w, phi)^{n+1}."""
        return self.solve_k2(self.k2[j, m], j == 0 and m == 0, r_om, r_th, r_psi)

    def solve_k2(self, k2, mean, r_om, r_th, r_psi):
        """Solve the implicit problems of the lines whose right-hand sides are the columns of
        r_om, r_th, r_psi ((Nz,) or (Nz, L)); all of them have the wavenumber magnitude k2, so
        they share the three operators (one factorisation each).  mean: the kx = ky = 0 line."""
        top, bottom = WALLS[self.p.bc]
        # omega_z and the mean flow: Dirichlet at a no-slip wall, Neumann at a free-slip wall
        # (du/dz = dv/dz = 0)
        kind = {"no-slip": "dirichlet", "free-slip": "neumann"}
        om = cheb.solve_helmholtz(r_om, k2 + self.beta, (kind[top], kind[bottom]))
        if mean:
            w = np.zeros_like(r_th)
        else:
            _, w = cheb.solve_coupled_w(r_th, k2, self.beta, (top, bottom))
        psi = cheb.solve_helmholtz(r_psi, k2 + self.lam, "neumann")
        ph = cheb.solve_helmholtz(psi, k2 + self.lam, "neumann")
        return om, w, ph

    def all_lines(self):
        return [(j, m) for j in range(self.p.ny) for m in range(self.Mx) if j != self.p.ny // 2]

    def solve_lines(self, lines, r_om, r_th, r_psi):
        """Solve the listed (j, m) lines, grouped by equal k2 (the mean line on its own);
        returns {(j, m): (omega, w, phi)}."""
        groups = {}
        for (j, m) in lines:
            key = "mean" if (j == 0 and m == 0) else float(self.k2[j, m])
            groups.setdefault(key, []).append((j, m))
        out = {}
        for key, ls in groups.items():
            js = np.array([j for j, _ in ls])
            ms = np.array([m for _, m in ls])
            k2 = 0.0 if key == "mean" else key
            om, w, ph = self.solve_k2(k2, key == "mean", r_om[:, js, ms], r_th[:, js, ms],
                                      r_psi[:, js, ms])
            for i, jm in enumerate(ls):
                out[jm] = (om[:, i], w[:, i], ph[:, i])
        return out

    def step(self, lines=None):
        """One time step n -> n+1 (Sec. 2.2 i)-v)).

        lines=None advances the whole state.  Otherwise only the listed (j, m) lines are solved
        and their new (omega, w, phi) columns are returned without changing the state (for
        sampled comparisons on large grids)."""
        nl = self.nonlinear_spectral()
        h = self.assemble(nl)
        prev = h if self.hist is None else self.hist
        H = tuple(1.5 * a - 0.5 * b for a, b in zip(h, prev))
        r_om, r_th, r_psi = self.rhs(H)
        todo = self.all_lines() if lines is None else lines
        out = self.solve_lines(todo, r_om, r_th, r_psi)
        if lines is not None:
            return out
        om = np.zeros_like(self.omega)
        w = np.zeros_like(self.w)
        ph = np.zeros_like(self.phi)
        for (j, m), (a, b, c) in out.items():
            om[:, j, m], w[:, j, m], ph[:, j, m] = a, b, c
        self.omega, self.w, self.phi = om, w, ph
        self.hist = h
        self.t += self.p.dt
        self.nstep += 1
        return None

    # ---- diagnostics -------------------------------------------------------------------------
    def mass(self):
        """Integral of phi over the box (R9): Lx Ly sum_n q_n Re(phihat_00,n)."""
        q = cheb.integral_weights(self.N)
        return self.p.lx * self.p.ly * float(q @ self.phi[:, 0, 0].real)

    def diagnostics(self):
        """t, step, mass, kinetic energy, int |grad phi|^2, free energy, CFL, max|phi|, nan flag.

        Volume integrals use uniform weights in x, y and Clenshaw-Curtis weights in z on the
        unpadded grid.  Free energy = int 1/4 (phi^2-1)^2 + Ch^2/2 |grad phi|^2 (Sec. 2.1.1)."""
        p = self.p
        u, v, w, f = self.get_fields()
        ph = self.phi
        fx, fy, fz = (self.spectral_to_physical(a) for a in (self.ikx * ph, self.iky * ph,
                                                             self.dz(ph)))
        wz = cheb.clenshaw_curtis_weights(self.N)[:, None, None]
        dA = p.lx / p.nx * p.ly / p.ny
        integ = lambda g: float(np.sum(g * wz) * dA)
        g2 = fx * fx + fy * fy + fz * fz
        z = cheb.points(self.N)
        dzl = np.empty(self.N + 1)
        dzl[1:-1] = 0.5 * (z[:-2] - z[2:])
        dzl[0] = z[0] - z[1]
        dzl[-1] = z[-2] - z[-1]
        cfl = p.dt * np.max(np.abs(u) / (p.lx / p.nx) + np.abs(v) / (p.ly / p.ny)
                            + np.abs(w) / dzl[:, None, None])
        allv = np.concatenate([a.ravel() for a in (u, v, w, f)])
        return dict(
            t=self.t,
            step=self.nstep,
            mass=self.mass(),
            kinetic=0.5 * integ(u * u + v * v + w * w),
            grad2=integ(g2),
            free_energy=integ(0.25 * (f * f - 1.0) ** 2 + 0.5 * p.ch ** 2 * g2),
            cfl=float(cfl),
            max_phi=float(np.max(np.abs(f))),
            nan=int(not np.all(np.isfinite(allv))),
        )
