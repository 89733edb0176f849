// Discrete adjoint of the time step (float64 grids): the reverse sweep of reverse-mode
// differentiation through the discrete step map of paper Sec. 2.2 (steps i)-v)), with the
// objective J = 1/2 int |u|^2 dV + int |grad phi|^2 dV of the final state.
//
// Forward step n (state s_n = (omega, w, phi) coefficients, history h_{n-1}):
//   N_n = Yf X Yb Zb(s_n)                 non-linear fields (zbwd, y backward, x line, y forward)
//   (R, h_n) = Zr(s_n, N_n, h_{n-1})       assembly, AB2, right-hand sides (linear in s_n, N_n, h)
//   s_{n+1} = U(Sol(R), s_n)               tau solves and the sum-form update
// Reverse step n, given lambda_{n+1} = dJ/ds_{n+1} and mu_n = dJ/dh_n:
//   Rb = Sol^T lambda_{n+1};  (lam, mu_{n-1}, Nb) = Zr^T(Rb, lambda_{n+1}, mu_n);
//   lambda_n = lam + Zb^T Yb^T X_{s_n}^T Yf^T Nb,
// where X_{s_n}^T is the transposed Jacobian of the x line at s_n: the forward fields of s_n are
// recomputed (zbwd + y backward) from the state saved before step n.  Every transpose is taken
// under the real inner product sum Re(conj(a) b) of the stored coefficients.
// The map differentiated is the literal Crank-Nicolson step (wall conditions imposed on
// q^{n+1}); the forward kernels' sum form agrees with it on every state that meets the wall
// conditions, which the trajectory from admissible initial fields always does, and the adjoint
// also carries the derivative with respect to wall values of q^n (see adj_zsolve).
#include <string.h>

#include <new>
#include <vector>

#include "../../include/ch_flow.h"
#include "ch_grid.h"
#include "ch_internal.h"

using chf::FftPlan;
using chf::GridDev;
using chf::kBw;
using chf::kNl;
using chf::kYa;

namespace {

#define CK(x)                                       \
  do {                                              \
    cudaError_t e__ = (x);                          \
    if (e__ != cudaSuccess) {                       \
      cudaGetLastError();                           \
      return CH_ERR_CUDA;                           \
    }                                               \
  } while (0)

// objective of the current state; lam receives dJ/ds (3 fields)
int objective_impl(ch_grid* G, double2* lam, double* J) {
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  const int nlines = g.Mx * g.ny;
  CK(chf::launch_objective(g, G->om, G->w, G->phi, lam, G->fs, G->obj_part, s));
  CK(chf::launch_sum(G->obj_part, nlines, G->obj_part + nlines, s));
  if (J) {
    CK(cudaMemcpyAsync(J, G->obj_part + nlines, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return CH_OK;
}

}  // namespace

void ch_adjoint_release(ch_grid* G) {
  if (!G || !G->adj_block) return;
  cudaStreamSynchronize(G->stream);
  if (G->ff) G->ff(G->adj_block, G->actx);
  else if (!G->af) cudaFree(G->adj_block);
  G->adj_block = nullptr;
  G->a_lam = G->a_L = G->a_Rb = G->a_mu = G->a_mu2 = G->a_nlb = G->a_x6 = G->a_bb = nullptr;
  if (G->seg_block) {
    if (G->ff) G->ff(G->seg_block, G->actx);
    else if (!G->af) cudaFree(G->seg_block);
    G->seg_block = nullptr;
    G->seg_cap = 0;
  }
}

extern "C" {

int ch_objective(ch_grid* G, double* J) {
  if (!G || !J) return CH_ERR_ARG;
  if (!G->fields_set) return CH_ERR_STATE;
  if (G->prec != CH_PREC_FP64) return CH_ERR_ARG;
  return objective_impl(G, G->auxA, J);
}

int ch_adjoint_begin(ch_grid* G, double* J) {
  if (!G) return CH_ERR_ARG;
  if (!G->fields_set) return CH_ERR_STATE;
  // float64, no-slip walls, FFT Chebyshev transforms only
  if (G->prec != CH_PREC_FP64 || G->g.bc != 0 || G->cheb != CH_CHEB_FFT) return CH_ERR_ARG;
  if (chf::adj_xline_smem(G->g.Px) > (size_t)chf::kMaxSmem) return CH_ERR_SIZE;
  if (!G->adj_block) {
    const size_t sb = (size_t)G->fs * sizeof(double2);
    const size_t nb = (size_t)G->g.Mx * G->g.ny * 6;  // wall-value adjoints
    const size_t bytes = 24 * sb + (size_t)6 * G->fsy * sizeof(double2) + nb * sizeof(double2);
    void* p = nullptr;
    if (G->af) p = G->af(bytes, G->actx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
    if (!p) return CH_ERR_ALLOC;
    G->adj_block = p;
    double2* b = (double2*)p;
    const long long fs = G->fs;
    G->a_lam = b;
    G->a_L = b + 3 * fs;
    G->a_Rb = b + 6 * fs;
    G->a_mu = b + 9 * fs;
    G->a_mu2 = b + 12 * fs;
    G->a_nlb = b + 15 * fs;
    G->a_x6 = b + 24 * fs;
    G->a_bb = G->a_x6 + 6 * G->fsy;
  }
  // lambda_K = dJ/ds_K, mu_{K-1} = 0 (the last history is not used by J)
  int r = objective_impl(G, G->a_L, J);
  if (r != CH_OK) return r;
  CK(cudaMemsetAsync(G->a_mu, 0, (size_t)3 * G->fs * sizeof(double2), G->stream));
  return CH_OK;
}

}  // extern "C"

namespace {

// the linear part of one reverse step, given the forward y-padded fields ya of s_n (the x line's
// linearisation point) and whether step n started Adams-Bashforth; ev (optional): 8 events,
// ev[0] already recorded before, ev[k + 1] recorded after launch k of the 7 launches
int reverse_core(ch_grid* G, const double2* ya, int first, cudaEvent_t* ev) {
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  cudaError_t e[7];
  e[0] = chf::launch_adj_zsolve(g, G->a_L, G->a_Rb, G->fs, G->a_bb, s);
  if (ev) cudaEventRecord(ev[1], s);
  e[1] = chf::launch_adj_zrhs(g, G->a_Rb, G->a_L, G->a_mu, G->a_lam, G->a_mu2, G->a_nlb, G->fs,
                              first, G->a_bb, G->pz, s);
  if (ev) cudaEventRecord(ev[2], s);
  e[2] = chf::launch_ypass(1, 0, g, g.Py, G->a_nlb, G->yb, kNl, G->fs, G->fsy, 1.0, G->py[0], s);
  if (ev) cudaEventRecord(ev[3], s);
  e[3] = chf::launch_adj_xline(g, ya, (const double2*)G->yb, G->a_x6, G->fsy, G->px[0], s);
  if (ev) cudaEventRecord(ev[4], s);
  e[4] = chf::launch_ypass(0, 0, g, g.Py, G->a_x6, G->auxA, kYa, G->fsy, G->fs, 1.0, G->py[0], s);
  if (ev) cudaEventRecord(ev[5], s);
  e[5] = chf::launch_fold_dy(g, G->auxA, G->fs, s);
  if (ev) cudaEventRecord(ev[6], s);
  e[6] = chf::launch_adj_zbwd(g, G->auxA, G->fs, G->a_lam, G->fs, G->pz, s);
  if (ev) cudaEventRecord(ev[7], s);
  for (int k = 0; k < 7; ++k)
    if (e[k] != cudaSuccess) {
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
  double2* t = G->a_L;
  G->a_L = G->a_lam;
  G->a_lam = t;
  t = G->a_mu;
  G->a_mu = G->a_mu2;
  G->a_mu2 = t;
  return CH_OK;
}

// one reverse step from a saved state; ev (optional) holds CH_ADJ_KERNELS + 1 events: ev[0]
// before the first launch, ev[k + 1] after launch k
int adjoint_step_impl(ch_grid* G, const void* state, cudaEvent_t* ev) {
  if (!G || !state) return CH_ERR_ARG;
  if (!G->adj_block) return CH_ERR_STATE;
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  chf::StateHeader h;
  const char* b = (const char*)state;
  CK(cudaMemcpyAsync(&h, b, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h.magic != chf::kStateMagic || h.nx != g.nx || h.ny != g.ny || h.nz != g.nz ||
      !h.fields_set)
    return CH_ERR_ARG;
  const size_t sb = (size_t)G->fs * sizeof(double2);
  double2* dst[3] = {G->om, G->w, G->phi};
  for (int i = 0; i < 3; ++i)
    CK(cudaMemcpyAsync(dst[i], b + sizeof(h) + i * sb, sb, cudaMemcpyDeviceToDevice, s));
  G->first = h.first;
  G->nstep = h.nstep;
  G->t = h.t;
  G->nl_stale = 1;
  const chf::YMap ym = chf::step_ymap();
  if (ev) cudaEventRecord(ev[0], s);
  // forward fields of s_n on the y-padded grid (the x line's linearisation point)
  cudaError_t e0 = chf::launch_zbwd(0, 0, kBw, g, G->R, G->om, G->w, G->phi, G->bw, G->fs, G->pz, s);
  if (ev) cudaEventRecord(ev[1], s);
  cudaError_t e1 = chf::launch_ypass(1, 0, g, g.Py, G->bw, G->ya, kYa, G->fs, G->fsy, 1.0,
                                     G->py[0], s, &ym);
  if (ev) cudaEventRecord(ev[2], s);
  if (e0 != cudaSuccess || e1 != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  return reverse_core(G, (const double2*)G->ya, h.first, ev ? ev + 2 : nullptr);
}

}  // namespace

extern "C" {

int ch_adjoint_step(ch_grid* G, const void* state) { return adjoint_step_impl(G, state, nullptr); }

int ch_adjoint_step_timed(ch_grid* G, const void* state, double* kernel_ms) {
  if (!kernel_ms) return CH_ERR_ARG;
  cudaEvent_t ev[CH_ADJ_KERNELS + 1];
  for (int i = 0; i <= CH_ADJ_KERNELS; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
  int st = adjoint_step_impl(G, state, ev);
  if (st == CH_OK && cudaEventSynchronize(ev[CH_ADJ_KERNELS]) != cudaSuccess) st = CH_ERR_CUDA;
  for (int k = 0; k < CH_ADJ_KERNELS && st == CH_OK; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) st = CH_ERR_CUDA;
    kernel_ms[k] = ms;
  }
  for (int i = 0; i <= CH_ADJ_KERNELS; ++i) cudaEventDestroy(ev[i]);
  if (st == CH_ERR_CUDA) cudaGetLastError();
  return st;
}

int ch_adjoint_segment(ch_grid* G, const void* checkpoint, int nsteps) {
  if (!G || !checkpoint || nsteps < 1) return CH_ERR_ARG;
  if (!G->adj_block) return CH_ERR_STATE;
  cudaStream_t s = G->stream;
  const size_t yab = (size_t)kYa * G->fsy * sizeof(double2);
  if (G->seg_cap < nsteps) {                 // storage for the y-padded fields of the segment
    if (G->seg_block) {
      cudaStreamSynchronize(s);
      if (G->ff) G->ff(G->seg_block, G->actx);
      else if (!G->af) cudaFree(G->seg_block);
      G->seg_block = nullptr;
      G->seg_cap = 0;
    }
    void* p = nullptr;
    if (G->af) p = G->af((size_t)nsteps * yab, G->actx);
    else if (cudaMalloc(&p, (size_t)nsteps * yab) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
    if (!p) return CH_ERR_ALLOC;
    G->seg_block = p;
    G->seg_cap = nsteps;
  }
  char* seg = (char*)G->seg_block;
  // recompute the segment from its checkpoint, keeping each state's y-padded fields
  int r = ch_set_state(G, checkpoint);       // also evaluates the fields of the first state
  if (r != CH_OK) return r;
  std::vector<int> first((size_t)nsteps);
  for (int k = 0; k < nsteps; ++k) {
    first[k] = G->first;
    CK(cudaMemcpyAsync(seg + (size_t)k * yab, G->ya, yab, cudaMemcpyDeviceToDevice, s));
    if (k + 1 < nsteps) {
      r = ch_step(G, 1);                     // ends with the y-padded fields of the next state
      if (r != CH_OK) return r;
    }
  }
  for (int k = nsteps - 1; k >= 0; --k) {
    r = reverse_core(G, (const double2*)(seg + (size_t)k * yab), first[k], nullptr);
    if (r != CH_OK) return r;
  }
  return CH_OK;
}

int ch_adjoint_gradient(ch_grid* G, double* gu, double* gv, double* gw, double* gphi) {
  if (!G || !gu || !gv || !gw || !gphi) return CH_ERR_ARG;
  if (!G->adj_block) return CH_ERR_STATE;
  const GridDev& g = G->g;
  cudaStream_t s = G->stream;
  CK(chf::launch_adj_project(g, G->a_L, G->fs, G->auxA, G->pz, s));
  CK(chf::launch_ypass(1, 0, g, g.ny, G->auxA, G->auxB, 4, G->fs, G->fs, 1.0, G->pyu, s));
  double* out[4] = {gu, gv, gw, gphi};
  for (int f = 0; f < 4; ++f)
    CK(chf::launch_x_c2r(g, G->auxB + f * G->fs, out[f], 1, G->fs, G->fsp, G->pxu, s));
  return CH_OK;
}

int ch_adjoint_end(ch_grid* G) {
  if (!G) return CH_ERR_ARG;
  ch_adjoint_release(G);
  return CH_OK;
}

}  // extern "C"
