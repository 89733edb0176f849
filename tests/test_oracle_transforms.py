"""Pins of the oracle's transforms and spectral derivatives against brute force and closed forms.

Paper: Sec. 2.2 (Fourier x Fourier x Chebyshev representation), Sec. 3.2.1 (the Chebyshev transform
is a DCT-I; its backward transform is again a DCT-I).  The oracle is checked against:
* brute-force O(N^2) DFT sums written with explicit exponentials;
* Chebyshev polynomials generated by the three-term recurrence T_{n+1} = 2 z T_n - T_{n-1} and
  numpy.polynomial.chebyshev (chebval, chebder);
* analytic derivatives of sin/cos/exp fields.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import chebyshev as cheb
from oracle import fourier
from oracle.channel import Channel, Params


def cheb_recurrence(N, z):
    """T_0..T_N at points z by the three-term recurrence (independent of cos(n theta))."""
    T = np.zeros((N + 1, len(z)))
    T[0] = 1.0
    if N >= 1:
        T[1] = z
    for n in range(1, N):
        T[n + 1] = 2 * z * T[n] - T[n - 1]
    return T


@pytest.mark.parametrize("N", [8, 16, 32, 96])
def test_backward_matrix_is_chebyshev_polynomials(N):
    z = cheb.points(N)
    T = cheb_recurrence(N, z)
    assert np.max(np.abs(cheb.backward_matrix(N) - T.T)) < 1e-12


@pytest.mark.parametrize("N", [8, 32, 128, 256])
def test_forward_recovers_coefficients_of_polynomials(N):
    rng = np.random.default_rng(N)
    a = rng.standard_normal(N + 1)
    z = cheb.points(N)
    vals = npc.chebval(z, a)                       # library evaluation of sum a_n T_n(z)
    # rounding of a length-N sum of terms of size |a|_1: N eps |a|_1
    tol = 4 * N * np.finfo(float).eps * np.sum(np.abs(a))
    assert np.max(np.abs(cheb.forward_matrix(N) @ vals - a)) < tol
    assert np.max(np.abs(cheb.backward_matrix(N) @ a - vals)) < tol


@pytest.mark.parametrize("N", [9, 32, 129])
def test_chebyshev_round_trip(N):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N + 1)
    back = cheb.backward_matrix(N) @ (cheb.forward_matrix(N) @ f)
    assert np.max(np.abs(back - f)) < 1e-14 * N


def test_dct_is_its_own_inverse_up_to_scale():
    # Sec. 3.2.1: the backward transform of a DCT-I is a DCT-I.  With C[j,n] = cos(pi n j / N)
    # and W = diag(1/cbar): C W C W = (N/2) I.
    N = 24
    C = cheb.backward_matrix(N)
    W = np.diag(1.0 / cheb.cbar_weights(N))
    assert np.max(np.abs(C @ W @ C @ W - (N / 2) * np.eye(N + 1))) < 1e-12


@pytest.mark.parametrize("N", [8, 33, 100])
def test_derivative_matrix_matches_chebder(N):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(N + 1)
    d = npc.chebder(a)
    d = np.concatenate([d, [0.0]])
    assert np.max(np.abs(cheb.deriv_matrix(N) @ a - d)) < 1e-12 * N * N


@pytest.mark.parametrize("N", [16, 32])
def test_derivative_of_exponential_is_spectrally_accurate(N):
    # e^z is resolved to machine precision by N >= 16; what remains is the usual roundoff growth
    # of coefficient-space differentiation, O(N^2 eps) per derivative.
    z = cheb.points(N)
    a = cheb.forward_matrix(N) @ np.exp(z)
    da = cheb.deriv_matrix(N) @ a
    d2a = cheb.deriv_matrix(N) @ da
    eps = np.finfo(float).eps * np.e
    assert np.max(np.abs(cheb.backward_matrix(N) @ da - np.exp(z))) < 4 * N ** 2 * eps
    assert np.max(np.abs(cheb.backward_matrix(N) @ d2a - np.exp(z))) < 4 * N ** 4 * eps


def test_integral_weights_and_clenshaw_curtis():
    N = 16
    rng = np.random.default_rng(3)
    a = rng.standard_normal(N + 1)
    exact = npc.chebval(1.0, npc.chebint(a)) - npc.chebval(-1.0, npc.chebint(a))
    assert abs(cheb.integral_weights(N) @ a - exact) < 1e-13
    vals = npc.chebval(cheb.points(N), a)
    assert abs(cheb.clenshaw_curtis_weights(N) @ vals - exact) < 1e-13


def brute_dft2(f, Lx, Ly, Nx, Ny):
    """fhat(my, mx) = (1/(Px Py)) sum_{y,x} f exp(-i (kx x + ky y)) by explicit double loops."""
    Py, Px = f.shape
    out = np.zeros((Ny, Nx // 2), complex)
    for j, my in enumerate(fourier.mode_index(Ny)):
        if j == Ny // 2:
            continue
        for mx in range(Nx // 2):
            s = 0j
            for iy in range(Py):
                for ix in range(Px):
                    x = ix * Lx / Px
                    y = iy * Ly / Py
                    s += f[iy, ix] * complex(math.cos(-(2 * math.pi * mx / Lx * x + 2 * math.pi * my / Ly * y)),
                                             math.sin(-(2 * math.pi * mx / Lx * x + 2 * math.pi * my / Ly * y)))
            out[j, mx] = s / (Px * Py)
    return out


@pytest.mark.parametrize("Py,Px", [(8, 8), (12, 12), (12, 6)])
def test_fourier_forward_matches_brute_force(Py, Px):
    Nx, Ny = (8, 8) if Px >= 8 else (4, 8)
    Lx, Ly = 4 * math.pi, 2 * math.pi
    rng = np.random.default_rng(4)
    f = rng.standard_normal((Py, Px))
    got = fourier.to_modes(f, Nx, Ny)
    ref = brute_dft2(f, Lx, Ly, Nx, Ny)
    assert np.max(np.abs(got - ref)) < 1e-14 * Px * Py


def test_fourier_backward_matches_brute_synthesis():
    Nx, Ny, Py, Px = 8, 8, 12, 12
    Lx, Ly = 4 * math.pi, 2 * math.pi
    rng = np.random.default_rng(5)
    s = rng.standard_normal((Ny, Nx // 2)) + 1j * rng.standard_normal((Ny, Nx // 2))
    s[Ny // 2] = 0
    # Hermitian completion at mx = 0 so the field is real
    for j, my in enumerate(fourier.mode_index(Ny)):
        if 0 < my < Ny // 2:
            s[(-my) % Ny, 0] = np.conj(s[j, 0])
    s[0, 0] = s[0, 0].real
    got = fourier.from_modes(s, Py, Px)
    ref = np.zeros((Py, Px))
    for iy in range(Py):
        for ix in range(Px):
            x, y = ix * Lx / Px, iy * Ly / Py
            acc = 0.0
            for j, my in enumerate(fourier.mode_index(Ny)):
                if j == Ny // 2:
                    continue
                for mx in range(Nx // 2):
                    e = s[j, mx] * np.exp(1j * (2 * math.pi * mx / Lx * x + 2 * math.pi * my / Ly * y))
                    acc += e.real if mx == 0 else 2 * e.real
            ref[iy, ix] = acc
    assert np.max(np.abs(got - ref)) < 1e-12


def test_three_dimensional_transform_matches_brute_force_8x8x9():
    p = Params(nx=8, ny=8, nz=9)
    ch = Channel(p)
    rng = np.random.default_rng(6)
    f = rng.standard_normal((9, 8, 8))
    got = ch.physical_to_spectral(f)
    N = 8
    z = cheb.points(N)
    T = cheb_recurrence(N, z)                    # T[n, j]
    cb = np.ones(N + 1)
    cb[0] = cb[N] = 2
    ref = np.zeros_like(got)
    for k in range(9):
        ref_k = brute_dft2(f[k], p.lx, p.ly, 8, 8)
        for n in range(N + 1):
            ref[n] += 2.0 / (cb[n] * N) * T[n, k] / cb[k] * ref_k
    assert np.max(np.abs(got - ref)) < 1e-13


def test_spectral_derivatives_of_analytic_fields():
    p = Params(nx=16, ny=12, nz=17)
    ch = Channel(p)
    x = np.arange(p.nx) * p.lx / p.nx
    y = np.arange(p.ny) * p.ly / p.ny
    z = cheb.points(16)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    f = np.sin(3 * 2 * math.pi / p.lx * X) * np.cos(2 * 2 * math.pi / p.ly * Y) * np.exp(Z)
    a = ch.physical_to_spectral(f)
    fx = ch.spectral_to_physical(ch.ikx * a)
    fy = ch.spectral_to_physical(ch.iky * a)
    fz = ch.spectral_to_physical(ch.dz(a))
    kx, ky = 3 * 2 * math.pi / p.lx, 2 * 2 * math.pi / p.ly
    assert np.max(np.abs(fx - kx * np.cos(kx * X) * np.cos(ky * Y) * np.exp(Z))) < 1e-13
    assert np.max(np.abs(fy + ky * np.sin(kx * X) * np.sin(ky * Y) * np.exp(Z))) < 1e-13
    assert np.max(np.abs(fz - f)) < 4 * 16 ** 2 * np.finfo(float).eps * np.e
