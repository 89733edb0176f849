"""Fourier building blocks of the oracle (periodic x and y directions).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 2.2 (Fourier series along the periodic x and y directions on equally spaced points;
non-linear terms formed in physical space) and Sec. 3.2.1 (real-to-complex transform in x, complex
transform in y).  numpy.fft is the library primitive for the DFT itself.

Conventions (one fixed reading, the paper gives none):

* spectral arrays hold modes mx = 0..Nx/2-1 (the x Nyquist mode is dropped) and the Ny y-modes in
  FFT order, index j <-> my = j for j < Ny/2 and my = j - Ny for j > Ny/2; the y Nyquist row
  j = Ny/2 is identically zero;
* forward: fhat = (1 / (Px Py)) * sum over the (Py, Px) grid of f exp(-i (kx x + ky y));
* backward: f = sum over modes of fhat exp(+i (kx x + ky y)) (negative mx by Hermitian symmetry);
* the 3/2 rule: products are formed on a grid of Px = 3 Nx / 2 by Py = 3 Ny / 2 points and only
  the kept modes are transformed back (zero padding / truncation).
"""
import numpy as np


def mode_index(Ny):
    """my for each stored y index j (FFT order); the Nyquist index Ny/2 maps to -Ny/2."""
    j = np.arange(Ny)
    return np.where(j < Ny // 2, j, j - Ny)


def wavenumbers(Nx, Ny, Lx, Ly):
    """kx (Mx,), ky (Ny,) with kx = 2 pi mx / Lx and ky = 2 pi my / Ly."""
    mx = np.arange(Nx // 2)
    my = mode_index(Ny)
    return 2.0 * np.pi * mx / Lx, 2.0 * np.pi * my / Ly


def to_modes(f, Nx, Ny):
    """Physical (..., Py, Px) -> kept modes (..., Ny, Nx/2).  Any Py >= Ny, Px >= Nx."""
    Py, Px = f.shape[-2:]
    F = np.fft.rfft2(f, axes=(-2, -1)) / (Px * Py)
    out = np.zeros(f.shape[:-2] + (Ny, Nx // 2), dtype=complex)
    for j, my in enumerate(mode_index(Ny)):
        if j == Ny // 2:
            continue
        out[..., j, :] = F[..., my % Py, : Nx // 2]
    return out


def from_modes(s, Py, Px):
    """Kept modes (..., Ny, Mx) -> physical (..., Py, Px), zero padding the missing modes."""
    Ny, Mx = s.shape[-2:]
    F = np.zeros(s.shape[:-2] + (Py, Px // 2 + 1), dtype=complex)
    for j, my in enumerate(mode_index(Ny)):
        if j == Ny // 2:
            continue
        F[..., my % Py, :Mx] = s[..., j, :]
    return np.fft.irfft2(F, s=(Py, Px), axes=(-2, -1)) * (Px * Py)
