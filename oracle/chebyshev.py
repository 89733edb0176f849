"""Chebyshev building blocks of the oracle (wall-normal direction z in [-1, 1]).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. 2.2 (Chebyshev polynomials along the wall-normal direction on stretched collocation
points, series of 1-D Helmholtz problems per (x, y) wavenumber pair) and Sec. 3.2.1 (the Chebyshev
transform is a DCT-I of the samples).  Everything is written as dense matrices taken straight from
the definitions, in FP64.

Notation: N = Nz - 1 is the polynomial degree, z_j = cos(pi j / N) for j = 0..N (j = 0 is the top
wall z = +1), c_0 = 2 and c_n = 1 otherwise, cbar_0 = cbar_N = 2 and cbar_n = 1 otherwise.
"""
import functools

import numpy as np


def points(N):
    """Chebyshev-Gauss-Lobatto points z_j = cos(pi j / N), j = 0..N (Sec. 2.2)."""
    j = np.arange(N + 1)
    return np.cos(np.pi * j / N)


def c_weights(N):
    """c_n of the Chebyshev derivative/integral relations: c_0 = 2, c_n = 1 for n >= 1."""
    c = np.ones(N + 1)
    c[0] = 2.0
    return c


def cbar_weights(N):
    """cbar_n of the discrete transform: cbar_0 = cbar_N = 2, 1 otherwise."""
    c = np.ones(N + 1)
    c[0] = 2.0
    c[N] = 2.0
    return c


def backward_matrix(N):
    """B[j, n] = T_n(z_j) = cos(pi n j / N): coefficient -> sample map (Sec. 3.2.1, DCT-I)."""
    j = np.arange(N + 1)[:, None]
    n = np.arange(N + 1)[None, :]
    # reduce n*j modulo 2N first so the cosine argument stays in [0, 2 pi)
    return np.cos(np.pi * ((n * j) % (2 * N)) / N)


def forward_matrix(N):
    """F[n, j] = 2 / (cbar_n N) cos(pi n j / N) / cbar_j: sample -> coefficient map.

    This is the inverse of ``backward_matrix`` on the N+1 CGL samples (discrete Chebyshev
    interpolation, a DCT-I up to the cbar weights; Sec. 3.2.1)."""
    cb = cbar_weights(N)
    return 2.0 / (cb[:, None] * N) * backward_matrix(N).T / cb[None, :]


def deriv_matrix(N):
    """D[n, p] = 2 p / c_n for p > n with p + n odd: Chebyshev coefficients of d/dz.

    Standard coefficient-space differentiation of a degree-N Chebyshev series (Sec. 2.2 uses the
    Chebyshev representation in z; the derivative follows from 2 n T_n = T'_{n+1}/(n+1) ...)."""
    c = c_weights(N)
    D = np.zeros((N + 1, N + 1))
    for n in range(N + 1):
        for p in range(n + 1, N + 1):
            if (p + n) % 2 == 1:
                D[n, p] = 2.0 * p / c[n]
    return D


def integral_weights(N):
    """q[n] = integral_{-1}^{1} T_n(z) dz = 2 / (1 - n^2) for even n, 0 for odd n."""
    q = np.zeros(N + 1)
    for n in range(0, N + 1, 2):
        q[n] = 2.0 / (1.0 - n * n)
    return q


def clenshaw_curtis_weights(N):
    """Quadrature weights on the CGL points that integrate every degree-N polynomial exactly.

    w_j = sum_n q_n F[n, j]: integrate the interpolating Chebyshev series term by term."""
    return integral_weights(N) @ forward_matrix(N)


@functools.lru_cache(maxsize=16)
def go_matrix(N):
    """Gottlieb-Orszag second-integral matrix G, rows n = 2..N (rows 0, 1 are zero).

    If D^2 a = b with b a Chebyshev series of degree <= N-2, then for n >= 2
        a_n = c_{n-2} b_{n-2} / (4 n (n-1)) - b_n / (2 (n^2-1)) + b_{n+2} / (4 n (n+1)),
    where b_m is taken as 0 for m > N-2 (tau truncation).  This is the standard row
    transformation of the Chebyshev-tau equations that makes the solve quasi-tridiagonal
    (Sec. 3.2.2: tridiagonal Gauss elimination per (x, y) position)."""
    c = c_weights(N)
    G = np.zeros((N + 1, N + 1))
    for n in range(2, N + 1):
        G[n, n - 2] = c[n - 2] / (4.0 * n * (n - 1))
        if n <= N - 2:
            G[n, n] = -1.0 / (2.0 * (n * n - 1))
        if n + 2 <= N - 2:
            G[n, n + 2] = 1.0 / (4.0 * n * (n + 1))
    G.setflags(write=False)          # cached: shared by every caller, never modified
    return G


def bc_rows(N, bc):
    """Two boundary rows: values at z = +1 and z = -1 (bc='dirichlet'), of d/dz (bc='neumann')
    or of d2/dz2 (bc='second').

    T_n(+1) = 1, T_n(-1) = (-1)^n, T_n'(+1) = n^2, T_n'(-1) = (-1)^(n+1) n^2,
    T_n''(+1) = n^2 (n^2 - 1) / 3, T_n''(-1) = (-1)^n n^2 (n^2 - 1) / 3."""
    n = np.arange(N + 1, dtype=float)
    sgn = (-1.0) ** np.arange(N + 1)
    if bc == "dirichlet":
        return np.stack([np.ones(N + 1), sgn])
    if bc == "neumann":
        return np.stack([n * n, -sgn * n * n])
    if bc == "second":
        t2 = n * n * (n * n - 1.0) / 3.0
        return np.stack([t2, sgn * t2])
    raise ValueError(bc)


def wall_rows(N, top, bottom):
    """Row 0: condition `top` at z = +1; row 1: condition `bottom` at z = -1; each one of
    'dirichlet', 'neumann', 'second' (value, first or second derivative), as in ``bc_rows``."""
    return np.stack([bc_rows(N, top)[0], bc_rows(N, bottom)[1]])


def helmholtz_matrix(N, alpha, bc):
    """Dense tau matrix of (D^2 - alpha) a = f in Gottlieb-Orszag form.

    Rows 0, 1: boundary conditions (bc: one kind for both walls, or a (top, bottom) pair).
    Rows n = 2..N: a_n - alpha (G a)_n = (G f)_n."""
    M = np.eye(N + 1) - alpha * go_matrix(N)
    M[0:2, :] = wall_rows(N, *bc) if isinstance(bc, tuple) else bc_rows(N, bc)
    return M


def helmholtz_rhs(N, f, g_plus=0.0, g_minus=0.0):
    """Right-hand side matching ``helmholtz_matrix``: BC values, then (G f)_n for n >= 2.

    f may hold several right-hand sides as columns (shape (N+1, L))."""
    r = go_matrix(N) @ f
    r = r.astype(np.result_type(r, g_plus, g_minus))
    r[0] = g_plus
    r[1] = g_minus
    return r


def solve_helmholtz(f, alpha, bc, g_plus=0.0, g_minus=0.0):
    """Solve (D^2 - alpha) a = f (tau rows 0..N-2) with two boundary conditions; dense LU.

    f: (N+1,) or (N+1, L) (L right-hand sides sharing alpha, one factorisation)."""
    N = len(f) - 1
    M = helmholtz_matrix(N, alpha, bc)
    r = helmholtz_rhs(N, f, g_plus, g_minus)
    return _solve_real(M, r)


def coupled_w_matrix(N, k2, beta, walls="no-slip"):
    """Dense matrix of the influence-matrix pair for (theta, w), 2(N+1) unknowns.

    (D^2 - k^2 - beta) theta = r   (tau rows 0..N-2)
    (D^2 - k^2) w = theta          (tau rows 0..N-2)
    no-slip:   w(+1) = w(-1) = 0, w'(+1) = w'(-1) = 0 (all four wall rows on w, Eq. (ww));
    free-slip: w(+1) = w(-1) = 0, w''(+1) = w''(-1) = 0 (again all four on w);
    (top, bottom) pair of 'no-slip' / 'free-slip': w(+-1) = 0 and, at each wall, w' = 0
    (no-slip) or w'' = 0 (free-slip).
    Both second-order problems are written in Gottlieb-Orszag form.  The walls are those of
    Sec. 2.1 (no-slip or free-slip).  Unknown vector = [theta_0..N, w_0..N]."""
    G = go_matrix(N)
    n1 = N + 1
    M = np.zeros((2 * n1, 2 * n1))
    I = np.eye(n1)
    rows = slice(2, n1)
    # theta rows n = 2..N
    M[2:n1, 0:n1] = (I - (k2 + beta) * G)[rows]
    # w rows n = 2..N:  w_n - k^2 (G w)_n - (G theta)_n = 0
    M[n1 + 2:2 * n1, n1:2 * n1] = (I - k2 * G)[rows]
    M[n1 + 2:2 * n1, 0:n1] = -G[rows]
    kind = {"no-slip": "neumann", "free-slip": "second"}
    top, bottom = walls if isinstance(walls, tuple) else (walls, walls)
    M[0:2, n1:2 * n1] = bc_rows(N, "dirichlet")                 # w = 0 at both walls
    M[n1:n1 + 2, n1:2 * n1] = wall_rows(N, kind[top], kind[bottom])
    return M


def solve_coupled_w(r, k2, beta, walls="no-slip"):
    """Solve the (theta, w) problem of ``coupled_w_matrix`` for a right-hand side r of shape
    (N+1,) or for the columns of r (N+1, L) (one factorisation).

    Returns (theta, w)."""
    N = len(r) - 1
    n1 = N + 1
    M = coupled_w_matrix(N, k2, beta, walls)
    rhs = np.zeros((2 * n1,) + r.shape[1:], dtype=np.result_type(r, float))
    rhs[0:n1] = go_matrix(N) @ r
    rhs[0:2] = 0.0
    x = _solve_real(M, rhs)
    return x[:n1], x[n1:]


def _solve_real(M, r):
    """Dense LU solve (numpy.linalg.solve: LAPACK gesv, partial pivoting) of a real matrix
    against a real or complex right-hand side r of shape (n,) or (n, L): the real and imaginary
    parts are solved as columns of one real system."""
    if np.iscomplexobj(r):
        cols = r.reshape(r.shape[0], -1)
        L = cols.shape[1]
        sol = np.linalg.solve(M, np.concatenate([cols.real, cols.imag], axis=1))
        return (sol[:, :L] + 1j * sol[:, L:]).reshape(r.shape)
    return np.linalg.solve(M, r)
