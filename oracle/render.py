"""Oracle of the headless interface image (test infrastructure: only tests, the smoke check and the
benchmark's CPU baseline use this package).

The image is of the surface phi = 0 that the paper's Sec. 4 shows for its drop simulation,
rendered for visual checks: for each pixel a perspective ray crosses the box
[0, lx] x [0, ly] x [-1, 1]; phi, interpolated trilinearly from its values on the collocation
grid (periodic in x and y, linearly between Gauss-Lobatto nodes in z), is sampled every `step`
along the ray; the first sign change is refined by 40 bisections; the hit is shaded with a
headlight, 0.25 + 0.75 |n . d| times the drop colour, n the unit gradient of phi (its spectral
derivatives, interpolated the same way).  Written with numpy, all rays marched together.
"""
import math

import numpy as np

BISECT = 40
BACKGROUND = np.array([0.08, 0.08, 0.12])
DROP = np.array([0.90, 0.45, 0.15])


def fields(c):
    """phi, phi_x, phi_y, phi_z of an oracle Channel on its unpadded grid, each (nz, ny, nx)."""
    ph = c.phi
    return [c.spectral_to_physical(a) for a in (ph, c.ikx * ph, c.iky * ph, c.dz(ph))]


def sample(f, p, x, y, z):
    """Trilinear value of the (nz, ny, nx) grid field f at points (x, y, z) (arrays)."""
    nz, ny, nx = f.shape
    N = nz - 1
    xs = x / (p.lx / nx)
    ys = y / (p.ly / ny)
    xf, yf = np.floor(xs), np.floor(ys)
    tx, ty = xs - xf, ys - yf
    i0 = np.mod(xf.astype(np.int64), nx)
    j0 = np.mod(yf.astype(np.int64), ny)
    i1, j1 = (i0 + 1) % nx, (j0 + 1) % ny
    zc = np.clip(z, -1.0, 1.0)
    k0 = np.clip((np.arccos(zc) * N / math.pi).astype(np.int64), 0, N - 1)
    k1 = k0 + 1
    z0, z1 = np.cos(math.pi * k0 / N), np.cos(math.pi * k1 / N)
    tz = (z0 - zc) / (z0 - z1)

    def plane(k):
        v00, v01 = f[k, j0, i0], f[k, j0, i1]
        v10, v11 = f[k, j1, i0], f[k, j1, i1]
        w0 = v00 + tx * (v01 - v00)
        w1 = v10 + tx * (v11 - v10)
        return w0 + ty * (w1 - w0)

    va, vb = plane(k0), plane(k1)
    return va + tz * (vb - va)


def camera_rays(width, height, eye, target, up, fov_deg):
    """Unit ray directions (height, width, 3) of a perspective camera."""
    eye, target, up = (np.asarray(v, dtype=float) for v in (eye, target, up))
    f = (target - eye) / np.linalg.norm(target - eye)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(0.5 * math.radians(fov_deg))
    px = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * th * (width / height)
    py = (1.0 - 2.0 * (np.arange(height) + 0.5) / height) * th
    d = f[None, None, :] + px[None, :, None] * r[None, None, :] + py[:, None, None] * u[None, None, :]
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def render(c, width, height, eye, target, up=(0.0, 0.0, 1.0), fov_deg=40.0, step=0.0):
    """(rgb uint8 (height, width, 3), depth (height, width); -1 where the ray misses)."""
    p = c.p
    phi, fx, fy, fz = fields(c)
    if not step > 0.0:
        step = 0.5 * min(p.lx / p.nx, p.ly / p.ny, math.pi / (p.nz - 1))
    e = np.asarray(eye, dtype=float)
    d = camera_rays(width, height, eye, target, up, fov_deg).reshape(-1, 3)
    n = d.shape[0]
    lo, hi = np.array([0.0, 0.0, -1.0]), np.array([p.lx, p.ly, 1.0])
    t0, t1 = np.zeros(n), np.full(n, np.inf)
    miss = np.zeros(n, dtype=bool)
    for a in range(3):
        par = np.abs(d[:, a]) < 1e-300
        miss |= par & ((e[a] < lo[a]) | (e[a] > hi[a]))
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[a] - e[a]) / d[:, a]
            tb = (hi[a] - e[a]) / d[:, a]
        tmin, tmax = np.minimum(ta, tb), np.maximum(ta, tb)
        t0 = np.where(par, t0, np.maximum(t0, tmin))
        t1 = np.where(par, t1, np.minimum(t1, tmax))
    live = ~miss & (t1 > t0)
    nmax = np.where(live, np.ceil((t1 - t0) / step), 0).astype(np.int64)
    pts = lambda t, idx: (e[0] + t * d[idx, 0], e[1] + t * d[idx, 1], e[2] + t * d[idx, 2])
    hit = np.full(n, -1.0)
    ta = t0.copy()
    fa = np.zeros(n)
    idx = np.nonzero(live)[0]
    fa[idx] = sample(phi, p, *pts(ta[idx], idx))
    active = live.copy()
    s = 0
    while active.any():
        s += 1
        idx = np.nonzero(active & (s <= nmax))[0]
        active[np.nonzero(active & (s > nmax))[0]] = False
        if idx.size == 0:
            break
        tb = np.minimum(t0[idx] + s * step, t1[idx])
        fb = sample(phi, p, *pts(tb, idx))
        cross = (fa[idx] > 0.0) != (fb > 0.0)
        if cross.any():
            ci = idx[cross]
            a, b, fl = ta[ci].copy(), tb[cross].copy(), fa[ci].copy()
            for _ in range(BISECT):
                m = 0.5 * (a + b)
                fm = sample(phi, p, *pts(m, ci))
                same = (fm > 0.0) == (fl > 0.0)
                a = np.where(same, m, a)
                fl = np.where(same, fm, fl)
                b = np.where(same, b, m)
            hit[ci] = 0.5 * (a + b)
            active[ci] = False
        keep = idx[~cross]
        ta[keep] = tb[~cross]
        fa[keep] = fb[~cross]
    col = np.tile(BACKGROUND, (n, 1))
    hi_idx = np.nonzero(hit >= 0.0)[0]
    if hi_idx.size:
        x, y, z = pts(hit[hi_idx], hi_idx)
        g = np.stack([sample(q, p, x, y, z) for q in (fx, fy, fz)], axis=-1)
        gn = np.linalg.norm(g, axis=-1)
        lam = np.where(gn > 0, np.abs(np.sum(g * d[hi_idx], axis=-1)) / np.where(gn > 0, gn, 1), 0)
        col[hi_idx] = DROP[None, :] * (0.25 + 0.75 * lam)[:, None]
    rgb = np.clip(np.floor(255.0 * col + 0.5), 0, 255).astype(np.uint8)
    return rgb.reshape(height, width, 3), hit.reshape(height, width)
