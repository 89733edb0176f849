// C-ABI of the channel solver (declared in include/ch_flow.h): validation, plans, twiddle
// tables, internal buffers, the per-step launch schedule and its CUDA-graph replay.
//
// One time step (paper Sec. 2.2, steps i)-v)) is six launches on the handle's stream (eight with
// the tensor-core Chebyshev method: the forward transform of the nine products before zrhs and
// the backward transform of the five fields after zbwd, zrhs and zbwd then skipping their DCTs):
//   zrhs    : Chebyshev DCT-I of the nine non-linear fields (as seven combinations), assembly,
//             AB2 / CN / IE right-hand sides;
//   zsolve  : the Chebyshev-tau solves of every wavenumber line;
//   zbwd    : state update, velocity from continuity, backward DCT-I of the five fields the next
//             products need;
//   ybwd    : ky -> y with 3/2 zero padding (i ky phi formed here: six fields);
//   xline   : kx -> x (padded), the nine products, x -> kx (truncated);
//   yfwd    : y -> ky, truncation and the 1/(Px Py) normalisation.
// The non-linear buffer therefore always holds the products of the current state.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ch_flow.h"
#include "ch_grid.h"
#include "ch_internal.h"

using chf::kBw;
using chf::kMaxSmem;
using chf::kNl;
using chf::kYa;
using chf::Tw;

using chf::FftPlan;
using chf::GridDev;

namespace chf {

bool smooth23(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

bool make_radices(int n, FftPlan* pl) { return make_radices_style(n, 0, pl); }

std::mutex& smem_limit_mutex() {
  static std::mutex m;
  return m;
}

bool make_radices_style(int n, int style, FftPlan* pl) {
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  if (m != 1) return false;
  int k = 0;
  pl->prune = 0;
  if (style == 3) {   // one radix 3 first (the pruned pass), then as for style 2
    if (b < 1) return false;
    pl->rad[k++] = 3;
    --b;
    pl->prune = 1;
  }
  if (style == 1)
    while (b > 0) { pl->rad[k++] = 3; --b; }
  if (style == 2 || style == 3) {
    while (a >= 3 && a != 4) { pl->rad[k++] = 8; a -= 3; }
  } else if (a % 2 == 1 && a >= 3) {
    pl->rad[k++] = 8;
    a -= 3;
  }
  while (a >= 2) { pl->rad[k++] = 4; a -= 2; }
  if (a == 1) { pl->rad[k++] = 2; a = 0; }
  while (b > 0) { pl->rad[k++] = 3; --b; }
  if (k > CHF_MAX_STAGES) return false;
  if (k == 0) { pl->rad[k++] = 2; }  // n == 1 never used
  pl->nst = k;
  pl->n = n;
  return true;
}

// size rules of ch_params (see include/ch_flow.h): CH_OK or CH_ERR_SIZE
int check_sizes(int nx, int ny, int nz) {
  if (nx < 4 || ny < 4 || nz < 5 || nx % 2 || ny % 2) return CH_ERR_SIZE;
  if (!smooth23(nx) || !smooth23(ny) || !smooth23(3 * nx / 2) || !smooth23(3 * ny / 2) ||
      (nz - 1) % 2 || !smooth23(2 * (nz - 1)))
    return CH_ERR_SIZE;
  if (3 * nx / 2 > 8192 || 3 * ny / 2 > 8192 || nz > 4097) return CH_ERR_SIZE;
  return CH_OK;
}

}  // namespace chf

using chf::make_radices;
using chf::smooth23;


namespace {

void* galloc(ch_grid* G, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (G->af) {
    p = G->af(bytes, G->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) G->allocs.push_back(p);
  return p;
}

void release_all(ch_grid* G) {
  for (void* p : G->allocs) {
    if (G->ff) G->ff(p, G->actx);
    else if (!G->af) cudaFree(p);
  }
  G->allocs.clear();
}

// twiddles exp(-2 pi i t / n) in extended precision, rounded once
int make_plan(ch_grid* G, int n, int prec, FftPlan* pl, int style = 0) {
  if (!chf::make_radices_style(n, style, pl)) return CH_ERR_SIZE;
  std::vector<double2> h64(n);
  std::vector<float2> h32(n);
  std::vector<float> hdf(4 * (size_t)n);  // double-float pairs (h, l) of re and im
  const long double pi2 = 6.283185307179586476925286766559L;
  for (int t = 0; t < n; ++t) {
    const long double a = pi2 * (long double)t / (long double)n;
    const long double c = cosl(a), s = -sinl(a);
    h64[t] = make_double2((double)c, (double)s);
    h32[t] = make_float2((float)c, (float)s);
    const float ch = (float)c, sh = (float)s;
    hdf[4 * (size_t)t + 0] = ch;
    hdf[4 * (size_t)t + 1] = (float)(c - (long double)ch);
    hdf[4 * (size_t)t + 2] = sh;
    hdf[4 * (size_t)t + 3] = (float)(s - (long double)sh);
  }
  Tw tw;
  tw.d64 = galloc(G, n * sizeof(double2));
  tw.d32 = galloc(G, n * sizeof(float2));
  tw.ddf = galloc(G, 4 * (size_t)n * sizeof(float));
  if (!tw.d64 || !tw.d32 || !tw.ddf) return CH_ERR_ALLOC;
  if (cudaMemcpy(tw.d64, h64.data(), n * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(tw.d32, h32.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(tw.ddf, hdf.data(), 4 * (size_t)n * sizeof(float), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return CH_ERR_CUDA;
  G->tws.push_back(tw);
  pl->tw = prec == 0 ? tw.d64 : prec == 1 ? tw.d32 : tw.ddf;
  return CH_OK;
}

}  // namespace

chf::YMap chf::step_ymap() {
  chf::YMap m;
  const int src[kYa] = {0, 1, 2, 3, 3, 4};  // u v w phi (phi -> i ky phi) Dphi
  for (int f = 0; f < chf::YMap::kMax; ++f) m.src[f] = f < kYa ? src[f] : 0;
  m.dy_mask = 1u << 4;
  m.kys = 0.0;
  return m;
}

using chf::step_ymap;

namespace {

// the CUDA error behind the last CH_ERR_CUDA of this thread (ch_last_cuda_error)
thread_local cudaError_t t_last_cuda = cudaSuccess;

#define CK(x)                                       \
  do {                                              \
    cudaError_t e__ = (x);                          \
    if (e__ != cudaSuccess) {                       \
      t_last_cuda = e__;                            \
      cudaGetLastError();                           \
      return CH_ERR_CUDA;                           \
    }                                               \
  } while (0)

// the nine products of the current state on the y-padded grid: bw <- 5 fields; ya <- y
// backward; yb <- x line
int eval_products(ch_grid* G) {
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  const chf::YMap ym = step_ymap();
  CK(chf::launch_zbwd(0, G->prec, kBw, g, G->R, G->om, G->w, G->phi, G->bw, G->fs, G->pz, s));
  CK(chf::launch_ypass(1, G->prec, g, g.Py, G->bw, G->ya, kYa, G->fs, G->fsy, 1.0, G->py[G->prec], s, &ym));
  CK(chf::launch_xline(G->prec, g, G->ya, G->yb, G->fsy, 1.0, G->px[G->prec], s));
  return CH_OK;
}

// non-linear terms of the current state: the products, then nl <- the seven combined lines of
// the forward y pass (normalised)
int eval_nonlinear_impl(ch_grid* G) {
  const GridDev& g = G->g;
  const int r = eval_products(G);
  if (r != CH_OK) return r;
  CK(chf::launch_ycomb(G->prec, g, G->yb, G->nl, G->fsy, G->fs,
                       1.0 / ((double)g.Px * (double)g.Py), G->py[G->prec], G->stream));
  return CH_OK;
}

// The step's launch schedule (the only copy).  Launch positions: 0 Chebyshev forward transform
// on the tensor cores (CH_CHEB_TC only), 1 zrhs, 2 zsolve, 3 zbwd, 4 Chebyshev backward
// transform (CH_CHEB_TC only), 5 y backward, 6 x line, 7 y forward.  ev, when given, holds
// CH_STEP_KERNELS events: ev[p] is recorded after position p (right away for an empty position).
int launch_step(ch_grid* G, int first, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  const GridDev& g = G->g;
  const chf::YMap ym = step_ymap();
  const bool tc = G->cheb == CH_CHEB_TC;
  const int nlines = g.Mx * g.ny;
  cudaError_t e[CH_STEP_KERNELS];
  for (int k = 0; k < CH_STEP_KERNELS; ++k) e[k] = cudaSuccess;
  // NVTX ranges (host side, for profilers) around the stages
  nvtxRangePushA("ch step");
  if (tc) {
    nvtxRangePushA("cheb fwd (tensor cores)");
    e[6] = chf::launch_cheb_tc(G->prec, 0, G->nl, G->fs, G->cf, G->fs, chf::kNc, nlines,
                               g.nz, G->tcf, G->tc_err, s);
    nvtxRangePop();
  }
  if (ev) cudaEventRecord(ev[0], s);
  nvtxRangePushA("zrhs");
  e[0] = tc ? chf::launch_zrhs_coef(g, G->cf, G->fs, G->om, G->w, G->phi, G->hom, G->hw,
                                    G->hphi, G->R, first, G->pz, s)
            : chf::launch_zrhs(G->prec, g, G->nl, G->fs, G->om, G->w, G->phi, G->hom, G->hw,
                               G->hphi, G->R, first, G->pz, s);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[1], s);
  nvtxRangePushA("zsolve");
  e[1] = chf::launch_zsolve(g, G->R, G->fs, s);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[2], s);
  nvtxRangePushA("zbwd");
  e[2] = tc ? chf::launch_zbwd_coef(g, G->R, G->om, G->w, G->phi, G->cf, G->fs, G->pz, s)
            : chf::launch_zbwd(1, G->prec, kBw, g, G->R, G->om, G->w, G->phi, G->bw, G->fs,
                               G->pz, s);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[3], s);
  if (tc) {
    nvtxRangePushA("cheb bwd (tensor cores)");
    e[7] = chf::launch_cheb_tc(0, G->prec, G->cf, G->fs, G->bw, G->fs, kBw, nlines,
                               g.nz, G->tcb, G->tc_err, s);
    nvtxRangePop();
  }
  if (ev) cudaEventRecord(ev[4], s);
  nvtxRangePushA("ybwd");
  e[3] = chf::launch_ypass(1, G->prec, g, g.Py, G->bw, G->ya, kYa, G->fs, G->fsy, 1.0,
                           G->py[G->prec], s, &ym);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[5], s);
  nvtxRangePushA("xline");
  e[4] = chf::launch_xline(G->prec, g, G->ya, G->yb, G->fsy, 1.0, G->px[G->prec], s);
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[6], s);
  nvtxRangePushA("yfwd");
  e[5] = chf::launch_ycomb(G->prec, g, G->yb, G->nl, G->fsy, G->fs,
                           1.0 / ((double)g.Px * (double)g.Py), G->py[G->prec], s);
  nvtxRangePop();
  nvtxRangePop();
  if (ev) cudaEventRecord(ev[7], s);
  for (int k = 0; k < CH_STEP_KERNELS; ++k)
    if (e[k] != cudaSuccess) {
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
  return CH_OK;
}

// launch position of each entry of ch_step_timed's kernel_ms (zrhs zsolve zbwd ybwd xline yfwd
// cheb_fwd cheb_bwd)
const int kStepPos[CH_STEP_KERNELS] = {1, 2, 3, 5, 6, 7, 0, 4};

// the 7 backward fields of the state, evaluated on the unpadded grid, into phys7
int state_to_phys7(ch_grid* G, int nf) {
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  CK(chf::launch_zbwd(0, 0, 7, g, G->R, G->om, G->w, G->phi, G->auxA, G->fs, G->pz, s));
  CK(chf::launch_ypass(1, 0, g, g.ny, G->auxA, G->auxB, nf, G->fs, G->fs, 1.0, G->pyu, s));
  CK(chf::launch_x_c2r(g, G->auxB, G->phys7, nf, G->fs, G->fsp, G->pxu, s));
  return CH_OK;
}

// failure exit of ch_init_grid: free what was obtained so far
int bail(ch_grid* G, int code) {
  release_all(G);
  cudaStreamDestroy(G->cap);
  delete G;
  return code;
}

void drop_graph(ch_grid* G) {
  if (G->graph_ok) cudaGraphExecDestroy(G->gexec);
  G->graph_ok = 0;
}

}  // namespace

int ch_launch_step(ch_grid* G, int first, cudaStream_t s, cudaEvent_t* ev) {
  return launch_step(G, first, s, ev);
}
int ch_state_phys7(ch_grid* G) { return state_to_phys7(G, 7); }
int ch_eval_nonlinear(ch_grid* G) { return eval_nonlinear_impl(G); }

extern "C" {

const char* ch_last_cuda_error(void) { return cudaGetErrorString(t_last_cuda); }

const char* ch_status_string(int st) {
  switch (st) {
    case CH_OK: return "ok";
    case CH_ERR_ARG: return "invalid argument";
    case CH_ERR_SIZE: return "unsupported grid size";
    case CH_ERR_ALLOC: return "allocation failed";
    case CH_ERR_CUDA: return "CUDA error";
    case CH_ERR_DIVERGED: return "solution diverged (NaN/Inf)";
    case CH_ERR_TIMEOUT: return "device wait timed out";
    case CH_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

int ch_init_grid(const ch_params* p, ch_alloc_fn alloc, ch_free_fn free_fn, void* alloc_ctx,
                 void* stream, ch_grid** out) {
  if (!p || !out) return CH_ERR_ARG;
  *out = nullptr;
  if (!(p->dt > 0) || !(p->lx > 0) || !(p->ly > 0) || !(p->re_tau > 0) || !(p->we > 0) ||
      !(p->ch > 0) || !(p->pe > 0))
    return CH_ERR_ARG;
  if (p->precision != CH_PREC_FP64 && p->precision != CH_PREC_MIXED &&
      p->precision != CH_PREC_DFLOAT)
    return CH_ERR_ARG;
  if (p->dealias_z != 0 || p->bc < 0 || p->bc > 3) return CH_ERR_ARG;
  if ((alloc == nullptr) != (free_fn == nullptr)) return CH_ERR_ARG;
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  if (chf::check_sizes(nx, ny, nz) != CH_OK) return CH_ERR_SIZE;

  ch_grid* G = new (std::nothrow) ch_grid();
  if (!G) return CH_ERR_ALLOC;
  G->p = *p;
  G->prec = p->precision;
  G->stream = (cudaStream_t)stream;
  G->af = alloc;
  G->ff = free_fn;
  G->actx = alloc_ctx;
  G->gexec = nullptr;
  G->graph_ok = 0;
  if (cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete G;
    return CH_ERR_CUDA;
  }
  GridDev& g = G->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.N = nz - 1;
  g.Mx = nx / 2;
  g.Px = 3 * nx / 2;
  g.Py = 3 * ny / 2;
  g.lx = p->lx;
  g.ly = p->ly;
  g.re = p->re_tau;
  g.we = p->we;
  g.ch = p->ch;
  g.pe = p->pe;
  g.dt = p->dt;
  g.gx = p->gx;
  g.gy = p->gy;
  g.beta = 2.0 * p->re_tau / p->dt;
  g.lam = sqrt(p->pe / (p->ch * p->ch * p->dt));
  g.shat = 2.0 * g.lam * p->ch * p->ch;
  g.kappa = 3.0 / sqrt(8.0) * p->ch / p->we;
  g.bc = p->bc;

  const size_t esz = G->prec == CH_PREC_MIXED ? sizeof(float2) : sizeof(double2);
  G->fs = (long long)g.Mx * ny * nz;
  G->fsy = (long long)g.Mx * g.Py * nz;
  G->fsp = (long long)nx * ny * nz;
  int st = CH_OK;
  auto A = [&](size_t bytes) -> void* {
    void* q = galloc(G, bytes);
    if (!q) st = CH_ERR_ALLOC;
    return q;
  };
  const size_t sb = (size_t)G->fs * sizeof(double2);
  G->om = (double2*)A(sb);
  G->w = (double2*)A(sb);
  G->phi = (double2*)A(sb);
  G->hom = (double2*)A(sb);
  G->hw = (double2*)A(sb);
  G->hphi = (double2*)A(sb);
  G->nl = A((size_t)kNl * G->fs * esz);
  G->bw = A((size_t)kBw * G->fs * esz);
  G->ya = A((size_t)kYa * G->fsy * esz);
  G->yb = A((size_t)kNl * G->fsy * esz);
  G->auxA = (double2*)A((size_t)7 * sb);
  G->auxB = (double2*)A((size_t)7 * sb);
  G->phys7 = (double*)A((size_t)7 * G->fsp * sizeof(double));
  G->tab = (double*)A((size_t)6 * nz * sizeof(double));
  G->zcs = (double2*)A((size_t)(nz - 1) * sizeof(double2));
  G->R = (double2*)A((size_t)3 * sb);
  g.NK = g.Mx * (ny / 2 + 1);
  G->fac = (double*)A(chf::fac_doubles(g) * sizeof(double));
  G->diag_part = (double*)A((size_t)(304 * 6 + 16) * sizeof(double));
  G->obj_part = (double*)A(((size_t)g.Mx * ny + 8) * sizeof(double));
  G->diag_out = G->diag_part + 304 * 6;
  if (st != CH_OK) {
    return bail(G, st);
  }
  // plans
  int e = CH_OK;
  // radix schedules (measured on GB300): the float64 and float32 x/y passes run fastest with as
  // many radix-8 passes as possible (style 2: e.g. 192 = 8*8*3 in three passes), the
  // double-float ones with the default schedule (style 0: 192 = 4*4*4*3)
  if (e == CH_OK) e = make_plan(G, g.Px, 0, &G->px[0], 2);
  if (e == CH_OK) {
    G->px[1] = G->px[0];
    G->px[1].tw = G->tws.back().d32;
    G->px[2] = G->px[0];
    G->px[2].tw = G->tws.back().ddf;
    if (!chf::make_radices_style(g.Px, 0, &G->px[2])) e = CH_ERR_SIZE;
  }
  if (e == CH_OK) e = make_plan(G, g.Py, 0, &G->py[0], 2);
  if (e == CH_OK) {
    G->py[1] = G->py[0];
    G->py[1].tw = G->tws.back().d32;
    G->py[2] = G->py[0];
    G->py[2].tw = G->tws.back().ddf;
    if (!chf::make_radices_style(g.Py, 0, &G->py[2])) e = CH_ERR_SIZE;
  }
  if (e == CH_OK) e = make_plan(G, g.N, 0, &G->pz, 2);
  if (e == CH_OK) e = make_plan(G, nx, 0, &G->pxu);
  if (e == CH_OK) e = make_plan(G, ny, 0, &G->pyu);
  if (e != CH_OK) {
    return bail(G, e);
  }
  // tables: Gottlieb-Orszag rows, Clenshaw-Curtis weights, local z spacing, integrals of T_n
  {
    const int N = g.N;
    std::vector<double> h(6 * (size_t)nz, 0.0);
    double* t1 = h.data();
    double* t2 = t1 + nz;
    double* t3 = t2 + nz;
    double* ccw = t3 + nz;
    double* dzl = ccw + nz;
    double* qint = dzl + nz;
    for (int n = 2; n <= N; ++n) {
      const double cnm2 = (n - 2 == 0) ? 2.0 : 1.0;
      t1[n] = cnm2 / (4.0 * n * (n - 1));
      t2[n] = (n <= N - 2) ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0;
      t3[n] = (n + 2 <= N - 2) ? 1.0 / (4.0 * n * (n + 1)) : 0.0;
    }
    for (int n = 0; n <= N; n += 2) qint[n] = 2.0 / (1.0 - (double)n * n);
    // ccw_j = sum_n qint_n * 2/(cbar_n N) cos(pi n j / N) / cbar_j (exact for degree <= N)
    const long double pi = 3.141592653589793238462643383279L;
    for (int j = 0; j <= N; ++j) {
      long double acc = 0.0L;
      for (int n = 0; n <= N; n += 2) {
        const long double cbn = (n == 0 || n == N) ? 2.0L : 1.0L;
        acc += (long double)qint[n] * 2.0L / (cbn * N) * cosl(pi * (long double)((n * j) % (2 * N)) / N);
      }
      const long double cbj = (j == 0 || j == N) ? 2.0L : 1.0L;
      ccw[j] = (double)(acc / cbj);
    }
    std::vector<double> z(nz);
    for (int j = 0; j <= N; ++j) z[j] = cos(3.14159265358979323846 * j / N);
    for (int j = 1; j < N; ++j) dzl[j] = 0.5 * (z[j - 1] - z[j + 1]);
    dzl[0] = z[0] - z[1];
    dzl[N] = z[N - 1] - z[N];
    if (cudaMemcpy(G->tab, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      return bail(G, CH_ERR_CUDA);
    }
    std::vector<double2> cs(N);
    for (int j = 0; j < N; ++j) {
      const long double a = pi * (long double)j / (long double)N;
      cs[j] = make_double2((double)cosl(a), (double)sinl(a));
    }
    if (cudaMemcpy(G->zcs, cs.data(), N * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(G, CH_ERR_CUDA);
    g.zcs = G->zcs;
    g.go1 = G->tab;
    g.go2 = G->tab + nz;
    g.go3 = G->tab + 2 * nz;
    g.fac = G->fac;
    if (chf::build_factor_table(g, G->fac, 0) != cudaSuccess) return bail(G, CH_ERR_CUDA);
  }
  if (chf::zline_smem(g) > (size_t)kMaxSmem || chf::xline_smem(g.Px, sizeof(double2)) > (size_t)kMaxSmem) {
    return bail(G, CH_ERR_SIZE);
  }
  G->first = 1;
  G->fields_set = 0;
  G->nstep = 0;
  G->t = 0.0;
  for (double2* q : {G->om, G->w, G->phi, G->hom, G->hw, G->hphi})
    if (cudaMemset(q, 0, sb) != cudaSuccess) {
      return bail(G, CH_ERR_CUDA);
    }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    return bail(G, CH_ERR_CUDA);
  }
  *out = G;
  return CH_OK;
}

int ch_set_stream(ch_grid* G, void* stream) {
  if (!G) return CH_ERR_ARG;
  G->stream = (cudaStream_t)stream;
  drop_graph(G);
  return CH_OK;
}

static int set_from_phys(ch_grid* G, const double* u, const double* v, const double* w,
                         const double* phi) {
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  const double* f4[4] = {u, v, w, phi};
  for (int f = 0; f < 4; ++f)
    CK(chf::launch_x_r2c(g, f4[f], G->auxA + f * G->fs, 1, G->fsp, G->fs, G->pxu, s));
  CK(chf::launch_ypass(0, 0, g, g.ny, G->auxA, G->auxB, 4, G->fs, G->fs,
                       1.0 / ((double)g.nx * (double)g.ny), G->pyu, s));
  CK(chf::launch_project(g, G->auxB, G->fs, G->om, G->w, G->phi, G->hom, G->hw, G->hphi, G->pz, s));
  G->first = 1;
  G->nstep = 0;
  G->t = 0.0;
  G->fields_set = 1;
  G->nl_stale = 0;
  return eval_nonlinear_impl(G);
}

int ch_set_fields(ch_grid* G, const double* u, const double* v, const double* w,
                  const double* phi) {
  if (!G || !u || !v || !w || !phi) return CH_ERR_ARG;
  return set_from_phys(G, u, v, w, phi);
}

int ch_set_fields_host(ch_grid* G, const double* u, const double* v, const double* w,
                       const double* phi) {
  if (!G || !u || !v || !w || !phi) return CH_ERR_ARG;
  const size_t b = (size_t)G->fsp * sizeof(double);
  const double* f4[4] = {u, v, w, phi};
  for (int f = 0; f < 4; ++f)
    CK(cudaMemcpyAsync(G->phys7 + f * G->fsp, f4[f], b, cudaMemcpyHostToDevice, G->stream));
  return set_from_phys(G, G->phys7, G->phys7 + G->fsp, G->phys7 + 2 * G->fsp,
                       G->phys7 + 3 * G->fsp);
}

int ch_step(ch_grid* G, int nsteps) {
  if (!G || nsteps < 0) return CH_ERR_ARG;
  if (!G->fields_set || G->nl_stale) return CH_ERR_STATE;
  for (int i = 0; i < nsteps; ++i) {
    if (G->first) {
      int r = launch_step(G, 1, G->stream);
      if (r != CH_OK) return r;
      G->first = 0;
    } else {
      if (!G->graph_ok) {
        // capture on the private stream (the caller's stream may be the legacy default
        // stream, which cannot be captured); the graph is then launched on the caller's stream
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal));
        int r = launch_step(G, 0, G->cap);
        cudaError_t e = cudaStreamEndCapture(G->cap, &graph);
        if (r != CH_OK || e != cudaSuccess) {
          cudaGetLastError();
          return CH_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&G->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return CH_ERR_CUDA;
        G->graph_ok = 1;
      }
      nvtxRangePushA("ch step (graph)");
      cudaError_t eg = cudaGraphLaunch(G->gexec, G->stream);
      nvtxRangePop();
      CK(eg);
    }
    G->nstep += 1;
    G->t += G->p.dt;
  }
  return CH_OK;
}

int ch_launches_per_step(const ch_grid* G) {
  return G ? (G->cheb == CH_CHEB_TC ? 8 : 6) : 0;
}

int ch_step_timed(ch_grid* G, int nsteps, double* kernel_ms, double* total_ms) {
  if (!G || nsteps < 0 || !total_ms) return CH_ERR_ARG;
  if (!G->fields_set || G->nl_stale) return CH_ERR_STATE;
  const int NKER = CH_STEP_KERNELS;
  const int nev = NKER * nsteps + 1;
  std::vector<cudaEvent_t> ev(nev);
  for (int i = 0; i < nev; ++i) CK(cudaEventCreate(&ev[i]));
  int st = CH_OK;
  CK(cudaEventRecord(ev[0], G->stream));
  for (int i = 0; i < nsteps && st == CH_OK; ++i) {
    st = launch_step(G, G->first, G->stream, &ev[NKER * i + 1]);
    G->first = 0;
    G->nstep += 1;
    G->t += G->p.dt;
  }
  CK(cudaEventSynchronize(ev[nev - 1]));
  double ks[CH_STEP_KERNELS] = {0};
  for (int i = 0; i < nsteps; ++i)
    for (int k = 0; k < NKER; ++k) {
      const int p = kStepPos[k];
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[NKER * i + p], ev[NKER * i + p + 1]));
      ks[k] += ms;
    }
  float tot = 0.f;
  CK(cudaEventElapsedTime(&tot, ev[0], ev[nev - 1]));
  for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
  if (kernel_ms)
    for (int k = 0; k < NKER; ++k) kernel_ms[k] = ks[k];
  *total_ms = tot;
  return st;
}

int ch_get_fields(ch_grid* G, double* u, double* v, double* w, double* phi) {
  if (!G || !u || !v || !w || !phi) return CH_ERR_ARG;
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  CK(chf::launch_zbwd(0, 0, 7, g, G->R, G->om, G->w, G->phi, G->auxA, G->fs, G->pz, s));
  CK(chf::launch_ypass(1, 0, g, g.ny, G->auxA, G->auxB, 4, G->fs, G->fs, 1.0, G->pyu, s));
  double* f4[4] = {u, v, w, phi};
  for (int f = 0; f < 4; ++f)
    CK(chf::launch_x_c2r(g, G->auxB + f * G->fs, f4[f], 1, G->fs, G->fsp, G->pxu, s));
  return CH_OK;
}

int ch_get_fields_host(ch_grid* G, double* u, double* v, double* w, double* phi) {
  if (!G || !u || !v || !w || !phi) return CH_ERR_ARG;
  int r = ch_get_fields(G, G->phys7, G->phys7 + G->fsp, G->phys7 + 2 * G->fsp,
                        G->phys7 + 3 * G->fsp);
  if (r != CH_OK) return r;
  const size_t b = (size_t)G->fsp * sizeof(double);
  double* f4[4] = {u, v, w, phi};
  for (int f = 0; f < 4; ++f)
    CK(cudaMemcpyAsync(f4[f], G->phys7 + f * G->fsp, b, cudaMemcpyDeviceToHost, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  return CH_OK;
}

int ch_diagnostics(ch_grid* G, ch_diag* out) {
  if (!G || !out) return CH_ERR_ARG;
  int r = state_to_phys7(G, 7);
  if (r != CH_OK) return r;
  const GridDev& g = G->g;
  const int nz = g.nz;
  CK(chf::launch_diag(g, G->phys7, G->fsp, G->phi, G->tab + 3 * nz, G->tab + 4 * nz,
                      G->tab + 5 * nz, G->diag_part, G->diag_out, G->stream));
  double h[8];
  CK(cudaMemcpyAsync(h, G->diag_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  if (G->tc_err) {
    int te = 0;
    CK(cudaMemcpy(&te, G->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (te) return CH_ERR_TIMEOUT;
  }
  out->t = G->t;
  out->step = G->nstep;
  out->mass = h[0];
  out->kinetic = h[1];
  out->grad2 = h[2];
  out->free_energy = h[3];
  out->cfl = h[4];
  out->max_phi = h[5];
  out->nan = h[6] != 0.0 ? 1 : 0;
  if (!isfinite(h[0]) || !isfinite(h[1])) out->nan = 1;
  return out->nan ? CH_ERR_DIVERGED : CH_OK;
}

// checkpoint layout: 64-byte header, then om w phi hom hw hphi
using chf::StateHeader;

size_t ch_state_bytes(const ch_grid* G) {
  if (!G) return 0;
  return sizeof(StateHeader) + (size_t)6 * G->fs * sizeof(double2);
}

int ch_get_state(ch_grid* G, void* buf) {
  if (!G || !buf) return CH_ERR_ARG;
  StateHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = chf::kStateMagic;
  h.nx = G->g.nx;
  h.ny = G->g.ny;
  h.nz = G->g.nz;
  h.first = G->first;
  h.nstep = G->nstep;
  h.t = G->t;
  h.fields_set = G->fields_set;
  char* b = (char*)buf;
  CK(cudaMemcpyAsync(b, &h, sizeof(h), cudaMemcpyHostToDevice, G->stream));
  const size_t sb = (size_t)G->fs * sizeof(double2);
  const double2* src[6] = {G->om, G->w, G->phi, G->hom, G->hw, G->hphi};
  for (int i = 0; i < 6; ++i)
    CK(cudaMemcpyAsync(b + sizeof(h) + i * sb, src[i], sb, cudaMemcpyDeviceToDevice, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  return CH_OK;
}

int ch_set_state(ch_grid* G, const void* buf) {
  if (!G || !buf) return CH_ERR_ARG;
  StateHeader h;
  const char* b = (const char*)buf;
  CK(cudaMemcpyAsync(&h, b, sizeof(h), cudaMemcpyDeviceToHost, G->stream));
  CK(cudaStreamSynchronize(G->stream));
  if (h.magic != chf::kStateMagic || h.nx != G->g.nx || h.ny != G->g.ny || h.nz != G->g.nz)
    return CH_ERR_ARG;
  const size_t sb = (size_t)G->fs * sizeof(double2);
  double2* dst[6] = {G->om, G->w, G->phi, G->hom, G->hw, G->hphi};
  for (int i = 0; i < 6; ++i)
    CK(cudaMemcpyAsync(dst[i], b + sizeof(h) + i * sb, sb, cudaMemcpyDeviceToDevice, G->stream));
  G->first = h.first;
  G->nstep = h.nstep;
  G->t = h.t;
  G->fields_set = h.fields_set;
  G->nl_stale = 0;
  if (!G->fields_set) return CH_OK;
  return eval_nonlinear_impl(G);
}

int ch_get_spectral(ch_grid* G, double* om, double* w, double* phi) {
  if (!G) return CH_ERR_ARG;
  const size_t sb = (size_t)G->fs * sizeof(double2);
  if (om) CK(cudaMemcpyAsync(om, G->om, sb, cudaMemcpyDeviceToDevice, G->stream));
  if (w) CK(cudaMemcpyAsync(w, G->w, sb, cudaMemcpyDeviceToDevice, G->stream));
  if (phi) CK(cudaMemcpyAsync(phi, G->phi, sb, cudaMemcpyDeviceToDevice, G->stream));
  return CH_OK;
}

int ch_set_spectral(ch_grid* G, const double* om, const double* w, const double* phi) {
  if (!G) return CH_ERR_ARG;
  const size_t sb = (size_t)G->fs * sizeof(double2);
  if (om) CK(cudaMemcpyAsync(G->om, om, sb, cudaMemcpyDeviceToDevice, G->stream));
  if (w) CK(cudaMemcpyAsync(G->w, w, sb, cudaMemcpyDeviceToDevice, G->stream));
  if (phi) CK(cudaMemcpyAsync(G->phi, phi, sb, cudaMemcpyDeviceToDevice, G->stream));
  for (double2* q : {G->hom, G->hw, G->hphi}) CK(cudaMemsetAsync(q, 0, sb, G->stream));
  G->first = 1;
  G->nstep = 0;
  G->t = 0.0;
  G->fields_set = 1;
  G->nl_stale = 0;
  return eval_nonlinear_impl(G);
}

int ch_transform_forward(ch_grid* G, const double* phys, double* spec) {
  if (!G || !phys || !spec) return CH_ERR_ARG;
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  CK(chf::launch_x_r2c(g, phys, G->auxA, 1, G->fsp, G->fs, G->pxu, s));
  CK(chf::launch_ypass(0, 0, g, g.ny, G->auxA, G->auxB, 1, G->fs, G->fs,
                       1.0 / ((double)g.nx * (double)g.ny), G->pyu, s));
  CK(chf::launch_dct_lines(0, 0, g, G->auxB, (double2*)spec, 1, G->fs, G->pz, s));
  return CH_OK;
}

int ch_transform_backward(ch_grid* G, const double* spec, double* phys) {
  if (!G || !phys || !spec) return CH_ERR_ARG;
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  CK(chf::launch_dct_lines(1, 0, g, spec, G->auxA, 1, G->fs, G->pz, s));
  CK(chf::launch_ypass(1, 0, g, g.ny, G->auxA, G->auxB, 1, G->fs, G->fs, 1.0, G->pyu, s));
  CK(chf::launch_x_c2r(g, G->auxB, phys, 1, G->fs, G->fsp, G->pxu, s));
  return CH_OK;
}

int ch_nonlinear(ch_grid* G, double* out9) {
  if (!G || !out9) return CH_ERR_ARG;
  if (!G->fields_set || G->nl_stale) return CH_ERR_STATE;
  // The step keeps only the seven combined lines; the nine products are evaluated again from the
  // state into nl (which has room for nine fields), transformed, and nl is restored.
  const GridDev& g = G->g;
  const double scale = 1.0 / ((double)g.Px * (double)g.Py);
  const int r = eval_products(G);
  if (r != CH_OK) return r;
  CK(chf::launch_ypass(0, G->prec, g, g.Py, G->yb, G->nl, kNl, G->fsy, G->fs, scale,
                       G->py[G->prec], G->stream));
  CK(chf::launch_dct_lines(0, G->prec, g, G->nl, (double2*)out9, kNl, G->fs, G->pz, G->stream));
  CK(chf::launch_ycomb(G->prec, g, G->yb, G->nl, G->fsy, G->fs, scale, G->py[G->prec],
                       G->stream));
  return CH_OK;
}

void ch_destroy(ch_grid* G) {
  if (!G) return;
  cudaStreamSynchronize(G->stream);
  drop_graph(G);
  ch_adjoint_release(G);
  release_all(G);
  cudaStreamDestroy(G->cap);
  delete G;
}

int ch_set_chebyshev(ch_grid* G, int method) {
  if (!G || (method != CH_CHEB_FFT && method != CH_CHEB_TC)) return CH_ERR_ARG;
  if (G->adj_block) return CH_ERR_STATE;   // not while a reverse sweep is open
  if (method == CH_CHEB_TC) {
    if (!G->cf) {
      const GridDev& g = G->g;
      std::vector<uint16_t> dig[2];
      std::vector<int> fe[2];
      chf::ChebTc t[2];
      for (int dir = 0; dir < 2; ++dir) {
        int NT, nNt, Kp;
        if (chf::cheb_tc_tables(g.N, dir, dig[dir], fe[dir], NT, nNt, Kp) != 0) return CH_ERR_SIZE;
        t[dir].NT = NT;
        t[dir].nNt = nNt;
        t[dir].Kp = Kp;
        t[dir].dir = dir;
        void* dd = galloc(G, dig[dir].size() * sizeof(uint16_t));
        void* df = galloc(G, fe[dir].size() * sizeof(int));
        if (!dd || !df) return CH_ERR_ALLOC;
        CK(cudaMemcpy(dd, dig[dir].data(), dig[dir].size() * sizeof(uint16_t),
                      cudaMemcpyHostToDevice));
        CK(cudaMemcpy(df, fe[dir].data(), fe[dir].size() * sizeof(int), cudaMemcpyHostToDevice));
        t[dir].dig = (const uint16_t*)dd;
        t[dir].fexp = (const int*)df;
        CK(chf::cheb_tc_prepare(NT));
      }
      CK(chf::zline_coef_prepare(g));
      // one persistent CTA per SM, each with a plane cache for one tile of rows
      int dev = 0, nsm = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      if (nsm < 1) nsm = 1;
      void* cache = galloc(G, (size_t)nsm * chf::cheb_tc_cache_bytes(t[0].Kp));
      if (!cache) return CH_ERR_ALLOC;
      for (int dir = 0; dir < 2; ++dir) {
        t[dir].cache = (uint32_t*)cache;
        t[dir].ctas = nsm;
      }
      int* err = (int*)galloc(G, sizeof(int));
      double2* cf = (double2*)galloc(G, (size_t)chf::kNc * G->fs * sizeof(double2));
      if (!err || !cf) return CH_ERR_ALLOC;
      CK(cudaMemset(err, 0, sizeof(int)));
      G->tcf = t[0];
      G->tcb = t[1];
      G->tc_err = err;
      G->cf = cf;
    }
  }
  drop_graph(G);
  G->cheb = method;
  return CH_OK;
}

int ch_get_chebyshev(const ch_grid* G) { return G ? G->cheb : CH_ERR_ARG; }

int ch_set_fft_pruning(ch_grid* G, int on) {
  if (!G || (on != 0 && on != 1)) return CH_ERR_ARG;
  if (G->adj_block) return CH_ERR_STATE;   // not while a reverse sweep is open
  // pruned: one radix 3 first, then as many radix 8 as possible; default: the measured
  // schedules (maximal radix 8 for float64 and float32, the plain one for double-float)
  const int def[3] = {2, 2, 0};
  for (int p = 0; p < 3; ++p) {
    chf::FftPlan x = G->px[p], y = G->py[p];
    if (!chf::make_radices_style(G->g.Px, on ? 3 : def[p], &x) ||
        !chf::make_radices_style(G->g.Py, on ? 3 : def[p], &y))
      return CH_ERR_SIZE;
    x.tw = G->px[p].tw;
    y.tw = G->py[p].tw;
    G->px[p] = x;
    G->py[p] = y;
  }
  drop_graph(G);
  return CH_OK;
}

int ch_get_fft_pruning(const ch_grid* G) { return G ? G->px[0].prune : CH_ERR_ARG; }

int ch_chebyshev_lines(ch_grid* G, int dir, const double* in, double* out, int nf) {
  if (!G || !in || !out || nf < 1 || (dir != 0 && dir != 1)) return CH_ERR_ARG;
  const GridDev& g = G->g;
  if (G->cheb == CH_CHEB_TC) {
    CK(chf::launch_cheb_tc(0, 0, in, G->fs, out, G->fs, nf, g.Mx * g.ny, g.nz,
                           dir == 0 ? G->tcf : G->tcb, G->tc_err, G->stream));
  } else {
    CK(chf::launch_dct_lines(dir, 0, g, in, (double2*)out, nf, G->fs, G->pz, G->stream));
  }
  return CH_OK;
}

int ch_selftest_bounded_wait(int nwaits, int* spun) {
  if (nwaits < 1) return CH_ERR_ARG;
  int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_ALLOC;
  }
  int h[2] = {0, 0}, st = CH_OK;
  if (cudaMemset(d, 0, 2 * sizeof(int)) != cudaSuccess ||
      chf::launch_wait_selftest(d, nwaits, 0) != cudaSuccess ||
      cudaMemcpy(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    st = CH_ERR_CUDA;
  } else if (h[0]) {
    st = CH_ERR_TIMEOUT;
  }
  if (spun) *spun = h[1];
  cudaFree(d);
  return st;
}

int ch_fp64_fma_rate(double* tflops) {
  if (!tflops) return CH_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  const int blocks = 16 * sms, iters = 4096;
  double* d = nullptr;
  if (cudaMalloc(&d, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_ALLOC;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.0f;
  int st = CH_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      chf::launch_fma_probe(d, blocks, iters, 0) != cudaSuccess ||
      cudaEventRecord(e0, 0) != cudaSuccess ||
      chf::launch_fma_probe(d, blocks, iters, 0) != cudaSuccess ||
      cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) {
    cudaGetLastError();
    st = CH_ERR_CUDA;
  } else {
    *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  return st;
}

int ch_device_status(ch_grid* G) {
  if (!G) return CH_ERR_ARG;
  CK(cudaStreamSynchronize(G->stream));
  if (G->tc_err) {
    int te = 0;
    CK(cudaMemcpy(&te, G->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (te) {
      CK(cudaMemset(G->tc_err, 0, sizeof(int)));
      return CH_ERR_TIMEOUT;
    }
  }
  return CH_OK;
}

}  // extern "C"
