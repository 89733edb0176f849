"""Seeded synthetic initial conditions shaped like the paper's channel workloads.

This module only draws seeded random numbers and evaluates closed-form fields on the collocation
grid; it contains none of the solver's arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from it.

Recipe (the paper's demo starts from a pre-computed turbulent field that is not available, so a
seeded stand-in is used; Sec. 4 describes drops released in a channel at Re_tau = 300):

* velocity = laminar Poiseuille profile (Re/2)(1 - z^2) in x plus a divergence-free, no-slip
  perturbation built from Fourier modes 1 <= |(mx, my)| <= 4: a wall-normal mode
  w = Re[A e^{i theta}] (1-z^2)^2 with (u, v) from continuity, and a vortical mode
  (u, v) = Re[i (ky, -kx) B e^{i theta}] (1-z^2) / |k|; A, B have real and imaginary parts drawn
  uniformly from (-1, 1) by numpy's PCG64(seed); the perturbation is rescaled so that its largest
  pointwise magnitude on the grid is ``amp``;
* phi = tanh((R - d) / (sqrt 2 Ch)), d = distance (periodic in x, y) to the nearest drop centre
  (the equilibrium profile of Sec. 2.1.1, Eq. (width)); one drop sits at the box centre, several
  drops are rejection-sampled with |z_c| <= 1 - R - 0.1 and centre separation >= 2R + 0.1.

All arrays are C-ordered (Nz, Ny, Nx) float64 with x_i = i Lx / Nx, y_j = j Ly / Ny,
z_k = cos(pi k / (Nz - 1)).
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi

# Workloads: name -> parameters.  The sizes and physical numbers are those of the five channel
# workloads of this project (tiny, medium, large channel; uneven ensemble; adjoint case).
WORKLOADS = {
    "channel_32x32x33": dict(nx=32, ny=32, nz=33, re_tau=150.0, ch=0.05, pe=20.0, we=1.0,
                             dt=1e-4, steps=10, ndrops=1, radius=0.4, seed=1, precision=0),
    "channel_128x128x129": dict(nx=128, ny=128, nz=129, re_tau=150.0, ch=0.02, pe=50.0, we=1.0,
                                dt=5e-5, steps=100, ndrops=8, radius=0.3, seed=2, precision=0),
    "channel_512x256x257_mixed": dict(nx=512, ny=256, nz=257, re_tau=300.0, ch=0.01, pe=100.0,
                                      we=3.0, dt=2e-5, steps=200, ndrops=64, radius=0.2, seed=3,
                                      precision=1),
    "channel_128x128x129_adjoint": dict(nx=128, ny=128, nz=129, re_tau=150.0, ch=0.02, pe=50.0,
                                        we=1.0, dt=5e-5, steps=50, ndrops=4, radius=0.3, seed=5,
                                        precision=0),
}


def ensemble_members(n=32, seed=4):
    """Uneven ensemble: n channels with seeded sizes nx in {64, 96, 128}, ny in {64, 128},
    nz in {65, 97, 129}; Re_tau = 150, one drop R = 0.3, Ch = 0.03, Pe = 1/Ch, We = 1, dt = 5e-5;
    member m's initial field uses seed 1000 + m.  Transforms in float32, solves in float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(n):
        out.append(dict(nx=int(rng.choice([64, 96, 128])), ny=int(rng.choice([64, 128])),
                        nz=int(rng.choice([65, 97, 129])), re_tau=150.0, ch=0.03,
                        pe=1.0 / 0.03, we=1.0, dt=5e-5, steps=100, ndrops=1, radius=0.3,
                        seed=1000 + m, precision=1))
    return out


def grid(nx, ny, nz, lx=4.0 * math.pi, ly=2.0 * math.pi):
    """Collocation coordinates x (nx,), y (ny,), z (nz,)."""
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny)
    z = np.cos(np.pi * np.arange(nz) / (nz - 1))
    return x, y, z


def wall_profiles(bc):
    """(w profile f, vortical profile g) as polynomials in z meeting the wall conditions exactly:
    w = 0 at both walls and w' = 0 at a no-slip wall, w'' = 0 at a free-slip wall (then u, v from
    continuity, proportional to f', vanish at a no-slip wall and have zero slope at a free-slip
    one); g = 0 at a no-slip wall, g' = 0 at a free-slip wall.  bc: 0 no-slip, 1 free-slip,
    2 no-slip at z = -1 and free-slip at z = +1, 3 the mirror."""
    P = np.polynomial.Polynomial
    one_m, one_p = P([1.0, -1.0]), P([1.0, 1.0])       # 1 - z, 1 + z
    if bc == 0:
        return (one_m * one_p) ** 2, one_m * one_p
    if bc == 1:
        return (one_m * one_p) ** 3, (one_m * one_p) ** 2
    if bc == 2:
        return one_p ** 2 * one_m ** 3, one_p * P([3.0, -1.0])
    if bc == 3:
        return one_m ** 2 * one_p ** 3, one_m * P([3.0, 1.0])
    raise ValueError(bc)


def mean_profile(bc):
    """Laminar-like mean profile with max 1: zero at no-slip walls, zero slope at free-slip ones."""
    P = np.polynomial.Polynomial
    return {0: P([1.0, 0.0, -1.0]), 1: P([1.0, 0.0, -2.0, 0.0, 1.0]),
            2: P([3.0, 2.0, -1.0]) / 4.0, 3: P([3.0, -2.0, -1.0]) / 4.0}[bc]


def perturbation(nx, ny, nz, seed, amp=0.1, kmax=4, lx=4.0 * math.pi, ly=2.0 * math.pi, bc=0):
    """Divergence-free velocity perturbation (u, v, w), each (nz, ny, nx), meeting the wall
    conditions of `bc` (see wall_profiles)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y, z = grid(nx, ny, nz, lx, ly)
    Z = z[:, None, None]
    fpoly, gpoly = wall_profiles(bc)
    f = fpoly(Z)                        # w profile
    fp = fpoly.deriv()(Z)               # f'
    g = gpoly(Z)                        # vortical (u, v) profile
    u = np.zeros((nz, ny, nx))
    v = np.zeros((nz, ny, nx))
    w = np.zeros((nz, ny, nx))
    for mx in range(0, kmax + 1):
        for my in range(-kmax, kmax + 1):
            if mx == 0 and my <= 0:
                continue
            if mx * mx + my * my > kmax * kmax:
                continue
            A = complex(rng.uniform(-1, 1), rng.uniform(-1, 1))
            B = complex(rng.uniform(-1, 1), rng.uniform(-1, 1))
            kx = TWO_PI * mx / lx
            ky = TWO_PI * my / ly
            k2 = kx * kx + ky * ky
            e = np.exp(1j * (kx * x[None, None, :] + ky * y[None, :, None]))
            w += np.real(A * e) * f
            u += np.real(1j * kx / k2 * A * e) * fp
            v += np.real(1j * ky / k2 * A * e) * fp
            kk = math.sqrt(k2)
            u += np.real(1j * ky / kk * B * e) * g
            v += np.real(-1j * kx / kk * B * e) * g
    mag = np.sqrt(u * u + v * v + w * w).max()
    s = amp / mag if mag > 0 else 0.0
    return u * s, v * s, w * s


def drop_centres(ndrops, radius, seed, lx=4.0 * math.pi, ly=2.0 * math.pi):
    """Drop centres: one at the box centre, or rejection-sampled non-overlapping centres."""
    if ndrops == 1:
        return np.array([[lx / 2, ly / 2, 0.0]])
    rng = np.random.Generator(np.random.PCG64(seed + 10_000))
    zmax = 1.0 - radius - 0.1
    out = []
    tries = 0
    while len(out) < ndrops:
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("could not place drops")
        c = np.array([rng.uniform(0, lx), rng.uniform(0, ly), rng.uniform(-zmax, zmax)])
        ok = True
        for o in out:
            d = _periodic_dist(c, o, lx, ly)
            if d < 2 * radius + 0.1:
                ok = False
                break
        if ok:
            out.append(c)
    return np.array(out)


def _periodic_dist(a, b, lx, ly):
    dx = abs(a[0] - b[0])
    dx = min(dx, lx - dx)
    dy = abs(a[1] - b[1])
    dy = min(dy, ly - dy)
    return math.sqrt(dx * dx + dy * dy + (a[2] - b[2]) ** 2)


def drops(nx, ny, nz, ndrops, radius, ch, seed, lx=4.0 * math.pi, ly=2.0 * math.pi):
    """phi = tanh((R - d) / (sqrt 2 Ch)) with d the distance to the nearest drop centre."""
    x, y, z = grid(nx, ny, nz, lx, ly)
    X = x[None, None, :]
    Y = y[None, :, None]
    Z = z[:, None, None]
    d = np.full((nz, ny, nx), np.inf)
    for c in drop_centres(ndrops, radius, seed, lx, ly):
        dx = np.abs(X - c[0])
        dx = np.minimum(dx, lx - dx)
        dy = np.abs(Y - c[1])
        dy = np.minimum(dy, ly - dy)
        d = np.minimum(d, np.sqrt(dx * dx + dy * dy + (Z - c[2]) ** 2))
    return np.tanh((radius - d) / (math.sqrt(2.0) * ch))


def initial_fields(nx, ny, nz, re_tau, ch, ndrops, radius, seed, amp=0.1,
                   lx=4.0 * math.pi, ly=2.0 * math.pi, bc=0, **_):
    """(u, v, w, phi) initial condition of the recipe above, each (nz, ny, nx) float64.  Other
    walls than no-slip (bc = 1, 2, 3) take the profiles of wall_profiles and mean_profile."""
    _, _, z = grid(nx, ny, nz, lx, ly)
    u, v, w = perturbation(nx, ny, nz, seed, amp=amp, lx=lx, ly=ly, bc=bc)
    u = u + (0.5 * re_tau * mean_profile(bc)(z))[:, None, None]
    phi = drops(nx, ny, nz, ndrops, radius, ch, seed, lx, ly)
    return u, v, w, phi


def workload_fields(name, **overrides):
    """Initial fields of a named workload (overrides replace entries of the table)."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return initial_fields(**w)
