"""Discrete adjoint of the oracle's time step, by reverse-mode differentiation of a float64 PyTorch
restatement of the same step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The step below repeats ``oracle.channel.Channel`` operation for operation (same Fourier helpers,
same dense Chebyshev matrices, same literal Crank-Nicolson / implicit-Euler right-hand sides, same
dense Gottlieb-Orszag tau systems), written with torch CPU float64/complex128 tensors so that
autograd yields the exact discrete adjoint of the oracle's discretisation.  Pins
(``tests/test_oracle_adjoint.py``): the step equals the numpy oracle's to rounding, and gradients
agree with central finite differences.

Objective (the workload's final-time objective: kinetic energy + interfacial area):
    J = 1/2 int |u|^2 dV + int |grad phi|^2 dV,
integrated exactly for the Fourier x Chebyshev interpolants: Parseval in x, y (weight 1 for
mx = 0, 2 for mx > 0) and the Chebyshev Gram matrix G_nm = int T_n T_m dz
= (q_{n+m} + q_{|n-m|}) / 2 with q_k = 2 / (1 - k^2) for even k, 0 for odd k.
"""
import math

import numpy as np
import torch

from . import chebyshev as cheb
from . import fourier
from .channel import Params

TD = torch.float64
TC = torch.complex128


def gram_matrix(N):
    """G[n, m] = integral_{-1}^{1} T_n T_m dz (T_n T_m = (T_{n+m} + T_{|n-m|}) / 2)."""
    q = np.zeros(2 * N + 1)
    for k in range(0, 2 * N + 1, 2):
        q[k] = 2.0 / (1.0 - k * k)
    n = np.arange(N + 1)
    return 0.5 * (q[n[:, None] + n[None, :]] + q[np.abs(n[:, None] - n[None, :])])


class TorchChannel:
    """The oracle step in torch; state tensors (Nz, Ny, Mx) complex128 as in oracle.channel."""

    def __init__(self, p: Params):
        self.p = p
        self.N = p.nz - 1
        self.Mx = p.nx // 2
        self.Px = 3 * p.nx // 2
        self.Py = 3 * p.ny // 2
        kx, ky = fourier.wavenumbers(p.nx, p.ny, p.lx, p.ly)
        self.kx = torch.tensor(kx, dtype=TD)
        self.ky = torch.tensor(ky, dtype=TD)
        self.ikx = (1j * self.kx.to(TC))[None, None, :]
        self.iky = (1j * self.ky.to(TC))[None, :, None]
        self.k2 = self.kx[None, :] ** 2 + self.ky[:, None] ** 2
        self.beta = 2.0 * p.re_tau / p.dt
        self.lam = math.sqrt(p.pe / (p.ch ** 2 * p.dt))
        self.shat = 2.0 * self.lam * p.ch ** 2
        self.kappa = 3.0 / math.sqrt(8.0) * p.ch / p.we
        N = self.N
        self.Fm = torch.tensor(cheb.forward_matrix(N), dtype=TD).to(TC)
        self.Bm = torch.tensor(cheb.backward_matrix(N), dtype=TD).to(TC)
        self.D = torch.tensor(cheb.deriv_matrix(N), dtype=TD).to(TC)
        self.G = torch.tensor(gram_matrix(N), dtype=TD).to(TC)
        self.my = fourier.mode_index(p.ny)
        # dense tau matrices of every line, as in oracle.chebyshev
        self._mat = {}

    # ---- transforms (same conventions as oracle.fourier / oracle.chebyshev) -------------------
    def cheb_fwd(self, f):
        return torch.tensordot(self.Fm, f, dims=([1], [0]))

    def cheb_bwd(self, a):
        return torch.tensordot(self.Bm, a, dims=([1], [0]))

    def dz(self, a):
        return torch.tensordot(self.D, a, dims=([1], [0]))

    def to_modes(self, f):
        Py, Px = f.shape[-2:]
        F = torch.fft.rfft2(f, dim=(-2, -1)) / (Px * Py)
        rows = []
        for j, my in enumerate(self.my):
            if j == self.p.ny // 2:
                rows.append(torch.zeros(f.shape[:-2] + (self.Mx,), dtype=TC))
            else:
                rows.append(F[..., my % Py, : self.Mx])
        return torch.stack(rows, dim=-2)

    def from_modes(self, s, Py, Px):
        F = torch.zeros(s.shape[:-2] + (Py, Px // 2 + 1), dtype=TC)
        for j, my in enumerate(self.my):
            if j == self.p.ny // 2:
                continue
            F[..., my % Py, : self.Mx] = s[..., j, :]
        return torch.fft.irfft2(F, s=(Py, Px), dim=(-2, -1)) * (Px * Py)

    def phys_to_spec(self, f):
        return self.cheb_fwd(self.to_modes(f))

    def spec_to_phys(self, a, padded=False):
        Py, Px = (self.Py, self.Px) if padded else (self.p.ny, self.p.nx)
        return self.from_modes(self.cheb_bwd(a), Py, Px)

    # ---- state ---------------------------------------------------------------------------------
    def set_fields(self, u, v, w, phi):
        uh, vh, wh, ph = (self.phys_to_spec(f) for f in (u, v, w, phi))
        om = self.ikx * vh - self.iky * uh
        mean = uh[:, 0, 0].real + 1j * vh[:, 0, 0].real
        om = _set_line(om, 0, 0, mean)
        wh = _set_line(wh, 0, 0, torch.zeros_like(mean))
        return om, wh, ph

    def velocity(self, om, w):
        Dw = self.dz(w)
        k2 = self.k2[None].to(TC)
        safe = torch.where(self.k2[None] > 0, k2, torch.ones_like(k2))
        uh = (self.ikx * Dw + self.iky * om) / safe
        vh = (self.iky * Dw - self.ikx * om) / safe
        uh = _set_line(uh, 0, 0, om[:, 0, 0].real.to(TC))
        vh = _set_line(vh, 0, 0, om[:, 0, 0].imag.to(TC))
        return uh, vh, w

    def nonlinear(self, om, w, ph):
        uh, vh, wh = self.velocity(om, w)
        fields = (uh, vh, wh, ph, self.ikx * ph, self.iky * ph, self.dz(ph))
        u, v, ww, f, fx, fy, fz = (self.spec_to_phys(a, padded=True) for a in fields)
        k = self.kappa
        g2 = fx * fx + fy * fy + fz * fz
        prods = (-u * u + k * (g2 - fx * fx), -v * v + k * (g2 - fy * fy),
                 -ww * ww + k * (g2 - fz * fz), -u * v - k * fx * fy, -u * ww - k * fx * fz,
                 -v * ww - k * fy * fz, f * f * f, u * f, v * f, ww * f)
        return [self.phys_to_spec(q) for q in prods]

    def assemble(self, nl, ph):
        sxx, syy, szz, sxy, sxz, syz, p3, fu, fv, fw = nl
        ikx, iky, k2 = self.ikx, self.iky, self.k2[None].to(TC)
        Sx = ikx * sxx + iky * sxy + self.dz(sxz)
        Sy = ikx * sxy + iky * syy + self.dz(syz)
        Sz = ikx * sxz + iky * syz + self.dz(szz)
        h_om = ikx * Sy - iky * Sx
        h_w = -k2 * Sz - self.dz(ikx * Sx + iky * Sy)
        e0 = torch.zeros(self.N + 1, dtype=TC)
        e0[0] = 1.0
        mean = Sx[:, 0, 0].real + 1j * Sy[:, 0, 0].real + (self.p.gx + 1j * self.p.gy) * e0
        h_om = _set_line(h_om, 0, 0, mean)
        h_w = _set_line(h_w, 0, 0, torch.zeros_like(mean))
        Gq = p3 - (1.0 + self.shat) * ph
        s_phi = -(ikx * fu + iky * fv + self.dz(fw)) + (1.0 / self.p.pe) * (
            self.dz(self.dz(Gq)) - k2 * Gq)
        return h_om, h_w, s_phi

    def _matrices(self, j, m):
        key = (j, m)
        if key not in self._mat:
            N = self.N
            k2 = float(self.k2[j, m])
            mats = (cheb.helmholtz_matrix(N, k2 + self.beta, "dirichlet"),
                    cheb.coupled_w_matrix(N, k2, self.beta),
                    cheb.helmholtz_matrix(N, k2 + self.lam, "neumann"))
            self._mat[key] = tuple(torch.tensor(a, dtype=TD) for a in mats)
        return self._mat[key]

    def step(self, state, hist):
        """One step: (omega, w, phi), history (or None) -> new state, new history."""
        p = self.p
        om, w, ph = state
        nl = self.nonlinear(om, w, ph)
        h = self.assemble(nl, ph)
        prev = h if hist is None else hist
        H = tuple(1.5 * a - 0.5 * b for a, b in zip(h, prev))
        k2 = self.k2[None].to(TC)
        D2 = lambda a: self.dz(self.dz(a))
        r_om = -(D2(om) - k2 * om + self.beta * om) - 2.0 * p.re_tau * H[0]
        th = D2(w) - k2 * w
        r_th = -(D2(th) - k2 * th + self.beta * th) - 2.0 * p.re_tau * H[1]
        r_psi = (p.pe / p.ch ** 2) * (ph / p.dt + H[2])
        Gt = torch.tensor(cheb.go_matrix(self.N), dtype=TD).to(TC)
        n1 = self.N + 1
        cols_om, cols_w, cols_ph = {}, {}, {}
        for j in range(p.ny):
            for m in range(self.Mx):
                if j == p.ny // 2:
                    continue
                Mo, Mw, Mp = self._matrices(j, m)
                ro = Gt @ r_om[:, j, m]
                ro = torch.cat([torch.zeros(2, dtype=TC), ro[2:]])
                cols_om[(j, m)] = _csolve(Mo, ro)
                if j == 0 and m == 0:
                    cols_w[(j, m)] = torch.zeros(n1, dtype=TC)
                else:
                    rw = torch.zeros(2 * n1, dtype=TC)
                    rw = torch.cat([torch.zeros(2, dtype=TC), (Gt @ r_th[:, j, m])[2:],
                                    torch.zeros(n1, dtype=TC)])
                    cols_w[(j, m)] = _csolve(Mw, rw)[n1:]
                rp = Gt @ r_psi[:, j, m]
                rp = torch.cat([torch.zeros(2, dtype=TC), rp[2:]])
                psi = _csolve(Mp, rp)
                rp2 = torch.cat([torch.zeros(2, dtype=TC), (Gt @ psi)[2:]])
                cols_ph[(j, m)] = _csolve(Mp, rp2)
        new = []
        for cols in (cols_om, cols_w, cols_ph):
            out = torch.zeros((n1, p.ny, self.Mx), dtype=TC)
            out = out.clone()
            rows = []
            for j in range(p.ny):
                row = []
                for m in range(self.Mx):
                    row.append(cols[(j, m)] if (j, m) in cols else torch.zeros(n1, dtype=TC))
                rows.append(torch.stack(row, dim=-1))
            new.append(torch.stack(rows, dim=-2))
        return tuple(new), h

    def objective(self, state):
        """J = 1/2 int |u|^2 + int |grad phi|^2 (exact integrals of the interpolants)."""
        om, w, ph = state
        uh, vh, wh = self.velocity(om, w)
        wmx = torch.where(torch.arange(self.Mx) == 0, 1.0, 2.0).to(TD)[None, None, :]
        area = self.p.lx * self.p.ly

        def quad(a):  # sum over lines of w_mx Re(a^H G a)
            Ga = torch.tensordot(self.G, a, dims=([1], [0]))
            return torch.sum(wmx * (a.conj() * Ga).real)

        ke = 0.5 * (quad(uh) + quad(vh) + quad(wh))
        g2 = quad(self.ikx * ph) + quad(self.iky * ph) + quad(self.dz(ph))
        return area * (ke + g2)


def _set_line(a, j, m, col):
    """a with a[:, j, m] replaced (out of place, autograd-friendly)."""
    mask = torch.zeros(a.shape[1:], dtype=torch.bool)
    mask[j, m] = True
    return torch.where(mask[None], col[:, None, None].to(a.dtype), a)


def _csolve(M, r):
    """Solve the real matrix M against a complex right-hand side."""
    sol = torch.linalg.solve(M, torch.stack([r.real, r.imag], dim=-1))
    return sol[..., 0] + 1j * sol[..., 1]


def objective_after(p: Params, fields, nsteps):
    """J after nsteps from physical initial fields (torch tensors, requires_grad allowed)."""
    c = TorchChannel(p)
    state = c.set_fields(*fields)
    hist = None
    for _ in range(nsteps):
        state, hist = c.step(state, hist)
    return c.objective(state)


def gradient(p: Params, fields_np, nsteps):
    """(J, dJ/du0, dJ/dv0, dJ/dw0, dJ/dphi0) by reverse-mode differentiation of the step."""
    ts = [torch.tensor(np.ascontiguousarray(f), dtype=TD, requires_grad=True) for f in fields_np]
    J = objective_after(p, ts, nsteps)
    J.backward()
    return float(J.detach()), tuple(t.grad.numpy().copy() for t in ts)
