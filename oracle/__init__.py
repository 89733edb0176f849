"""Plain FP64 CPU oracle of the pseudo-spectral Navier-Stokes + Cahn-Hilliard channel step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path (the C-ABI library in
``paper_2406_01322_gb300``) never imports, links or calls anything in here, and this package never
imports the product path.

Sources of truth (section / equation numbers of Roccon, "A GPU-ready pseudo-spectral method for
direct numerical simulations of multiphase turbulence", arXiv:2406.01322):

* Sec. 2.1.1, Eq. (CHE), chemical potential, Eq. (width): Cahn-Hilliard equation.
* Sec. 2.1.2, Eqs. (cont), (NSE), (kort): Navier-Stokes with Korteweg capillary stress.
* Sec. 2.2, Eqs. (omegaz), (ww), (omegadef), (phisplit): wall-normal velocity-vorticity form,
  split Cahn-Hilliard operator, Fourier x Fourier x Chebyshev discretisation, IMEX scheme and the
  step sequence i)-v).
* Sec. 3.2.1: Chebyshev transform as a DCT-I of the Chebyshev-Gauss-Lobatto samples.
* Sec. 3.2.2: tridiagonal (Chebyshev-tau) Helmholtz solves per (x, y) wavenumber pair.

Where the paper is silent the oracle takes one fixed reading; every reading is listed in the
module docstring of ``oracle.channel``.

Module map:

* ``oracle.chebyshev``  Chebyshev points, transforms, derivative, tau (Gottlieb-Orszag) solves.
* ``oracle.fourier``    x/y Fourier transforms with 3/2-rule padding (numpy.fft as the primitive).
* ``oracle.channel``    the full time step, set/get fields, diagnostics.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed forms, library
routines (numpy.polynomial.chebyshev, brute-force DFT sums) or exact discrete recurrences.
"""
