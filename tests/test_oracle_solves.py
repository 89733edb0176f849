"""Pins of the oracle's Chebyshev-tau Helmholtz and influence-matrix solves (Sec. 3.2.2: series of
tridiagonal Helmholtz problems along z per (x, y) wavenumber pair; Eq. (ww): no-slip 4th-order
problem for w solved as a pair of Helmholtz problems).

Manufactured polynomial solutions of degree <= N are reproduced exactly (to rounding) by the tau
method, so they pin the matrices; right-hand sides are built with numpy.polynomial.chebyshev
(a library routine independent of the oracle's own derivative matrix).
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import chebyshev as cheb


def pad(c, N):
    out = np.zeros(N + 1)
    out[: len(c)] = c
    return out


def one_minus_z2():
    return npc.poly2cheb([1.0, 0.0, -1.0])


@pytest.mark.parametrize("N,alpha", [(16, 0.0), (32, 7.5), (64, 3.0e6), (128, 6.0e6), (256, 1.5e7)])
def test_dirichlet_manufactured(N, alpha):
    rng = np.random.default_rng(N)
    q = rng.standard_normal(N - 1) / np.arange(1, N) ** 2          # degree N-2
    a = pad(npc.chebmul(one_minus_z2(), q), N)                      # a(+-1) = 0, degree N
    f = pad(npc.chebder(a, 2), N) - alpha * a
    got = cheb.solve_helmholtz(f, alpha, "dirichlet")
    assert np.max(np.abs(got - a)) < 1e-12 * np.max(np.abs(a)) * max(1, N / 64)


@pytest.mark.parametrize("N,alpha", [(16, 2.0), (64, 8944.27), (128, 5.0e4), (256, 2.236e5)])
def test_neumann_manufactured(N, alpha):
    rng = np.random.default_rng(N + 1)
    q = rng.standard_normal(N - 2) / np.arange(1, N - 1) ** 2       # degree N-3
    a = pad(npc.chebint(npc.chebmul(one_minus_z2(), q)), N)         # a'(+-1) = 0, degree N
    a[0] += 0.3
    f = pad(npc.chebder(a, 2), N) - alpha * a
    got = cheb.solve_helmholtz(f, alpha, "neumann")
    assert np.max(np.abs(got - a)) < 1e-12 * np.max(np.abs(a)) * max(1, N / 64)


def test_dirichlet_inhomogeneous_closed_form():
    # (D^2 - alpha) a = 1, a(+-1) = 0 has a = (cosh(sqrt(alpha) z) / cosh(sqrt(alpha)) - 1) / alpha
    N, alpha = 40, 4.0
    f = np.zeros(N + 1)
    f[0] = 1.0
    a = cheb.solve_helmholtz(f, alpha, "dirichlet")
    z = cheb.points(N)
    s = math.sqrt(alpha)
    exact = (np.cosh(s * z) / math.cosh(s) - 1.0) / alpha
    assert np.max(np.abs(cheb.backward_matrix(N) @ a - exact)) < 1e-14


def test_dirichlet_boundary_values():
    N = 24
    f = np.zeros(N + 1)
    a = cheb.solve_helmholtz(f, 9.0, "dirichlet", g_plus=2.0, g_minus=-1.0)
    z = cheb.points(N)
    # a'' = 9 a, a(+1) = 2, a(-1) = -1
    exact = (2.0 * np.sinh(3 * (z + 1)) + (-1.0) * np.sinh(3 * (1 - z))) / math.sinh(6)
    assert np.max(np.abs(cheb.backward_matrix(N) @ a - exact)) < 1e-13


@pytest.mark.parametrize("N", [10, 16])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_gottlieb_orszag_rows_equal_literal_tau_rows(N, bc):
    # Literal tau method: rows 0..N-2 of (D^2 - alpha) a = f, plus two boundary rows.  The
    # Gottlieb-Orszag rows are a row transformation of it: same solution.
    alpha = 5.0
    rng = np.random.default_rng(7)
    f = rng.standard_normal(N + 1)
    D = cheb.deriv_matrix(N)
    L = D @ D - alpha * np.eye(N + 1)
    M = np.zeros((N + 1, N + 1))
    M[: N - 1] = L[: N - 1]
    M[N - 1:] = cheb.bc_rows(N, bc)
    r = np.concatenate([f[: N - 1], [0.0, 0.0]])
    literal = np.linalg.solve(M, r)
    assert np.max(np.abs(cheb.solve_helmholtz(f, alpha, bc) - literal)) < 1e-12


@pytest.mark.parametrize("N,k2,beta", [(16, 0.25, 10.0), (32, 1.25, 3.0e6), (128, 4.0, 6.0e6),
                                      (256, 100.0, 1.5e7)])
def test_influence_pair_manufactured(N, k2, beta):
    rng = np.random.default_rng(N + 2)
    q = rng.standard_normal(N - 3) / np.arange(1, N - 2) ** 2       # degree N-4
    w = pad(npc.chebmul(npc.chebpow(one_minus_z2(), 2), q), N)      # w = w' = 0 at the walls
    theta = pad(npc.chebder(w, 2), N) - k2 * w
    r = pad(npc.chebder(theta, 2), N) - (k2 + beta) * theta
    th_got, w_got = cheb.solve_coupled_w(r, k2, beta)
    assert np.max(np.abs(w_got - w)) < 1e-13 * np.max(np.abs(w)) * max(1, N / 64)
    # theta is fixed only through the wall slopes of the thin homogeneous solutions
    # (width 1/sqrt(beta)): its rounding error is O(eps N^2 sqrt(beta)) while w stays exact.
    bound = 4 * np.finfo(float).eps * N * N * math.sqrt(beta) * np.max(np.abs(theta))
    assert np.max(np.abs(th_got - theta)) < max(bound, 1e-13 * np.max(np.abs(theta)))


def test_influence_pair_wall_conditions():
    # Arbitrary forcing: the solution must satisfy w(+-1) = w'(+-1) = 0.
    N = 48
    rng = np.random.default_rng(9)
    r = rng.standard_normal(N + 1)
    _, w = cheb.solve_coupled_w(r, 2.0, 1.0e4)
    n = np.arange(N + 1)
    sgn = (-1.0) ** n
    scale = np.max(np.abs(w))
    assert abs(np.sum(w)) < 1e-13 * scale and abs(np.sum(sgn * w)) < 1e-13 * scale
    assert abs(np.sum(n * n * w)) < 1e-11 * scale and abs(np.sum(sgn * n * n * w)) < 1e-11 * scale


@pytest.mark.parametrize("N,k2,beta", [(16, 0.25, 10.0), (32, 1.25, 3.0e6), (128, 4.0, 6.0e6)])
def test_free_slip_pair_manufactured(N, k2, beta):
    """Free-slip walls (Sec. 2.1): w = (1 - z^2)^3 q has w = w'' = 0 at both walls; the
    (theta, w) solve must return it exactly."""
    rng = np.random.default_rng(N + 5)
    q = rng.standard_normal(N - 5) / np.arange(1, N - 4) ** 2       # degree N-6
    w = pad(npc.chebmul(npc.chebpow(one_minus_z2(), 3), q), N)
    theta = pad(npc.chebder(w, 2), N) - k2 * w
    r = pad(npc.chebder(theta, 2), N) - (k2 + beta) * theta
    th_got, w_got = cheb.solve_coupled_w(r, k2, beta, "free-slip")
    # the w'' wall rows carry entries up to N^4 / 3 (the no-slip w' rows: N^2), a factor ~N^2
    # more rounding in the dense solve
    assert np.max(np.abs(w_got - w)) < 1e-13 * np.max(np.abs(w)) * max(1, N * N / 64)
    # theta is fixed only through the wall curvature of the thin homogeneous solutions (width
    # 1/sqrt(beta)), seen through rows of size N^4/3: rounding O(eps N^4 sqrt(beta)); w stays exact
    bound = 4 * np.finfo(float).eps * N ** 4 / 3 * math.sqrt(beta) * np.max(np.abs(theta))
    assert np.max(np.abs(th_got - theta)) < max(bound, 1e-12 * np.max(np.abs(theta)))


def test_free_slip_pair_wall_conditions():
    # Arbitrary forcing: w(+-1) = 0 and w''(+-1) = 0 (T_n''(+-1) = (+-1)^n n^2 (n^2 - 1) / 3).
    N = 48
    r = np.random.default_rng(19).standard_normal(N + 1)
    _, w = cheb.solve_coupled_w(r, 2.0, 1.0e4, "free-slip")
    n = np.arange(N + 1, dtype=float)
    sgn = (-1.0) ** n
    t2 = n * n * (n * n - 1) / 3
    scale = np.max(np.abs(w))
    assert abs(np.sum(w)) < 1e-13 * scale and abs(np.sum(sgn * w)) < 1e-13 * scale
    assert abs(np.sum(t2 * w)) < 1e-9 * scale and abs(np.sum(sgn * t2 * w)) < 1e-9 * scale
    # the second derivative at the walls from the coefficients directly (numpy.polynomial)
    d2 = npc.chebder(w, 2)
    assert abs(npc.chebval(1.0, d2)) < 1e-9 * scale and abs(npc.chebval(-1.0, d2)) < 1e-9 * scale
    # the no-slip rows would leave w' nonzero here: the two wall sets differ
    assert abs(np.sum(n * n * w)) > 1e-6 * scale


@pytest.mark.parametrize("walls", [("neumann", "dirichlet"), ("dirichlet", "neumann")])
def test_mixed_wall_helmholtz_manufactured(walls):
    """Different rows on each wall (Sec. 2.1 allows a combination of no-slip and free-slip):
    any polynomial a solves (D^2 - alpha) a = f with its own wall values."""
    N, alpha = 32, 7.5e3
    a = np.random.default_rng(4).standard_normal(N + 1) / np.arange(1, N + 2) ** 2
    f = pad(npc.chebder(a, 2), N) - alpha * a
    val = {"dirichlet": lambda z: npc.chebval(z, a),
           "neumann": lambda z: npc.chebval(z, npc.chebder(a))}
    got = cheb.solve_helmholtz(f, alpha, walls, val[walls[0]](1.0), val[walls[1]](-1.0))
    assert np.max(np.abs(got - a)) < 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("N", [16, 64])
def test_mixed_wall_pair_manufactured(N):
    """Free-slip at z = +1, no-slip at z = -1: w = (1+z)^2 (1-z)^3 q has w(+-1) = 0, w'(-1) = 0
    and w''(+1) = 0; the mirrored case uses w(-z)."""
    rng = np.random.default_rng(N + 7)
    q = rng.standard_normal(N - 4) / np.arange(1, N - 3) ** 2          # degree N-5
    base = npc.chebmul(npc.chebpow(npc.poly2cheb([1.0, 1.0]), 2), npc.chebpow(npc.poly2cheb([1.0, -1.0]), 3))
    w = pad(npc.chebmul(base, q), N)
    k2, beta = 1.5, 4.0e4
    for walls, ww in ((("free-slip", "no-slip"), w), (("no-slip", "free-slip"), w * (-1.0) ** np.arange(N + 1))):
        theta = pad(npc.chebder(ww, 2), N) - k2 * ww
        r = pad(npc.chebder(theta, 2), N) - (k2 + beta) * theta
        _, w_got = cheb.solve_coupled_w(r, k2, beta, walls)
        # one w'' row (entries up to N^4 / 3): rounding grows like N^2 as for free-slip walls
        tol = 1e-13 * max(1, N * N / 64)
        assert np.max(np.abs(w_got - ww)) < tol * np.max(np.abs(ww)), walls


def test_lines_sharing_k2_solve_as_one_factorisation():
    """The oracle's step solves every line with the same k^2 against one matrix (the columns of
    one system); each column must equal the single-line solve of that line."""
    from oracle.channel import Channel, Params
    c = Channel(Params(nx=8, ny=8, nz=17, dt=1e-3))
    rng = np.random.default_rng(5)
    shape = c.omega.shape
    r = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(3)]
    lines = [(1, 1), (7, 1), (0, 2), (1, 0), (7, 0), (0, 0), (3, 2)]   # (1,1)/(7,1) share k^2
    got = c.solve_lines(lines, *r)
    for (j, m) in lines:
        one = c.solve_line(j, m, r[0][:, j, m], r[1][:, j, m], r[2][:, j, m])
        for a, b in zip(got[(j, m)], one):
            assert np.max(np.abs(a - b)) <= 1e-13 * max(np.max(np.abs(b)), 1e-300)
