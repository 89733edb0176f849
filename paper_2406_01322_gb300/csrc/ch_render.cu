// Headless rendering of the interface phi = 0 (the surface the paper's Sec. 4 shows for its drop
// simulation): one thread per pixel casts a perspective ray through the box
// [0, lx] x [0, ly] x [-1, 1], marches phi with a fixed step, refines the first sign change by
// bisection and shades the hit with a headlight on the spectral gradient of phi.  phi and its
// gradient are the state's fields on the unpadded collocation grid, interpolated trilinearly
// (periodic in x and y, between Gauss-Lobatto nodes in z).  No graphics API: the image is an
// RGB8 device buffer (and optionally a depth buffer) for the caller to write out.
#include <math.h>

#include "../../include/ch_flow.h"
#include "ch_grid.h"
#include "ch_internal.h"

using chf::GridDev;

namespace {

struct Cam {
  double e[3];     // eye
  double f[3];     // forward (unit)
  double r[3];     // right (unit)
  double u[3];     // up (unit)
  double th;       // tan(fov / 2)
  double aspect;   // width / height
};

constexpr int kBisect = 40;
constexpr double kPi = 3.141592653589793238462643383279;

// trilinear sample of a (nz, ny, nx) field at (x, y, z)
__device__ double sample(const double* __restrict__ f, const GridDev& g, double x, double y,
                         double z) {
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  const double xs = x / dx, ys = y / dy;
  const double xf = floor(xs), yf = floor(ys);
  const double tx = xs - xf, ty = ys - yf;
  int i0 = (int)xf % g.nx;
  if (i0 < 0) i0 += g.nx;
  int j0 = (int)yf % g.ny;
  if (j0 < 0) j0 += g.ny;
  const int i1 = (i0 + 1) % g.nx, j1 = (j0 + 1) % g.ny;
  const int N = g.N;
  const double zc = fmin(1.0, fmax(-1.0, z));
  int k0 = (int)(acos(zc) * N / kPi);
  if (k0 > N - 1) k0 = N - 1;
  if (k0 < 0) k0 = 0;
  const int k1 = k0 + 1;
  const double z0 = cos(kPi * k0 / N), z1 = cos(kPi * k1 / N);
  const double tz = (z0 - zc) / (z0 - z1);
  const size_t sk = (size_t)g.ny * g.nx;
  const double* a = f + (size_t)k0 * sk;
  const double* b = f + (size_t)k1 * sk;
  auto bil = [&](const double* p) {
    const double v00 = p[(size_t)j0 * g.nx + i0], v01 = p[(size_t)j0 * g.nx + i1];
    const double v10 = p[(size_t)j1 * g.nx + i0], v11 = p[(size_t)j1 * g.nx + i1];
    const double w0 = v00 + tx * (v01 - v00), w1 = v10 + tx * (v11 - v10);
    return w0 + ty * (w1 - w0);
  };
  const double va = bil(a), vb = bil(b);
  return va + tz * (vb - va);
}

__global__ void render_kernel(GridDev g, const double* __restrict__ phys, long long fsp, Cam c,
                              int W, int H, double step, unsigned char* __restrict__ rgb,
                              double* __restrict__ depth) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y * blockDim.y + threadIdx.y;
  if (px >= W || py >= H) return;
  const double* phi = phys + 3 * fsp;
  const double sx = (2.0 * (px + 0.5) / W - 1.0) * c.th * c.aspect;
  const double sy = (1.0 - 2.0 * (py + 0.5) / H) * c.th;
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = c.f[a] + sx * c.r[a] + sy * c.u[a];
  const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int a = 0; a < 3; ++a) d[a] /= dn;
  // ray against the box (slabs)
  const double lo[3] = {0.0, 0.0, -1.0}, hi[3] = {g.lx, g.ly, 1.0};
  double t0 = 0.0, t1 = 1e300;
  bool miss = false;
  for (int a = 0; a < 3; ++a) {
    if (fabs(d[a]) < 1e-300) {
      if (c.e[a] < lo[a] || c.e[a] > hi[a]) miss = true;
      continue;
    }
    double ta = (lo[a] - c.e[a]) / d[a], tb = (hi[a] - c.e[a]) / d[a];
    if (ta > tb) {
      const double tt = ta;
      ta = tb;
      tb = tt;
    }
    t0 = fmax(t0, ta);
    t1 = fmin(t1, tb);
  }
  double hit = -1.0;
  if (!miss && t1 > t0) {
    // fixed-step march (at most ceil((t1 - t0) / step) samples), then bisection
    double ta = t0;
    double fa = sample(phi, g, c.e[0] + ta * d[0], c.e[1] + ta * d[1], c.e[2] + ta * d[2]);
    const int nmax = (int)ceil((t1 - t0) / step);
    for (int s = 1; s <= nmax; ++s) {
      const double tb = fmin(t0 + s * step, t1);
      const double fb = sample(phi, g, c.e[0] + tb * d[0], c.e[1] + tb * d[1], c.e[2] + tb * d[2]);
      if ((fa > 0.0) != (fb > 0.0)) {
        double a = ta, b = tb, fl = fa;
        for (int it = 0; it < kBisect; ++it) {
          const double m = 0.5 * (a + b);
          const double fm = sample(phi, g, c.e[0] + m * d[0], c.e[1] + m * d[1], c.e[2] + m * d[2]);
          if ((fm > 0.0) == (fl > 0.0)) {
            a = m;
            fl = fm;
          } else {
            b = m;
          }
        }
        hit = 0.5 * (a + b);
        break;
      }
      ta = tb;
      fa = fb;
    }
  }
  double col[3] = {0.08, 0.08, 0.12};   // background
  if (hit >= 0.0) {
    const double x = c.e[0] + hit * d[0], y = c.e[1] + hit * d[1], z = c.e[2] + hit * d[2];
    const double gx = sample(phys + 4 * fsp, g, x, y, z);
    const double gy = sample(phys + 5 * fsp, g, x, y, z);
    const double gz = sample(phys + 6 * fsp, g, x, y, z);
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    const double lam = gn > 0.0 ? fabs(gx * d[0] + gy * d[1] + gz * d[2]) / gn : 0.0;
    const double base[3] = {0.90, 0.45, 0.15};
    for (int a = 0; a < 3; ++a) col[a] = base[a] * (0.25 + 0.75 * lam);
  }
  const size_t o = ((size_t)py * W + px);
  for (int a = 0; a < 3; ++a) {
    const double v = floor(255.0 * col[a] + 0.5);
    rgb[3 * o + a] = (unsigned char)fmin(255.0, fmax(0.0, v));
  }
  if (depth) depth[o] = hit;
}

}  // namespace

extern "C" {

int ch_render_interface(ch_grid* G, unsigned char* rgb, double* depth, int width, int height,
                        const double* camera, double fov_deg, double step) {
  if (!G || !rgb || !camera || width < 1 || height < 1 || !(fov_deg > 0.0 && fov_deg < 180.0))
    return CH_ERR_ARG;
  if (!G->fields_set) return CH_ERR_STATE;
  const GridDev& g = G->g;
  Cam c;
  double f[3], up[3];
  for (int a = 0; a < 3; ++a) {
    c.e[a] = camera[a];
    f[a] = camera[3 + a] - camera[a];
    up[a] = camera[6 + a];
  }
  const double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fn > 0.0)) return CH_ERR_ARG;
  for (int a = 0; a < 3; ++a) c.f[a] = f[a] / fn;
  // right = f x up, true up = right x f
  double r[3] = {c.f[1] * up[2] - c.f[2] * up[1], c.f[2] * up[0] - c.f[0] * up[2],
                 c.f[0] * up[1] - c.f[1] * up[0]};
  const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(rn > 0.0)) return CH_ERR_ARG;
  for (int a = 0; a < 3; ++a) c.r[a] = r[a] / rn;
  c.u[0] = c.r[1] * c.f[2] - c.r[2] * c.f[1];
  c.u[1] = c.r[2] * c.f[0] - c.r[0] * c.f[2];
  c.u[2] = c.r[0] * c.f[1] - c.r[1] * c.f[0];
  c.th = tan(0.5 * fov_deg * kPi / 180.0);
  c.aspect = (double)width / (double)height;
  if (!(step > 0.0)) step = 0.5 * fmin(fmin(g.lx / g.nx, g.ly / g.ny), kPi / g.N);
  int r7 = ch_state_phys7(G);
  if (r7 != CH_OK) return r7;
  dim3 blk(16, 8), grd((width + 15) / 16, (height + 7) / 8);
  render_kernel<<<grd, blk, 0, G->stream>>>(g, G->phys7, G->fsp, c, width, height, step, rgb,
                                            depth);
  if (cudaGetLastError() != cudaSuccess) return CH_ERR_CUDA;
  return CH_OK;
}

}  // extern "C"
