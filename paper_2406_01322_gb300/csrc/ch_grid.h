// Host-side state of one channel handle (internal to libchflow).
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/ch_flow.h"
#include "ch_internal.h"

namespace chf {

const int kMaxSmem = 227 * 1024 - 1024;  // opt-in limit less room for static shared memory

struct Tw {
  void* d64 = nullptr;  // double2[n]
  void* d32 = nullptr;  // float2[n]
  void* ddf = nullptr;  // df2[n] (double-float pairs)
};

// fields through the step: 5 backward (u v w phi Dphi) -> 6 y-padded (phi_y added by the y
// pass) -> 9 products (Sxx-Szz Syy-Szz Sxy Sxz Syz phi^3 u phi v phi w phi)
constexpr int kBw = 5, kYa = 6, kNl = 9;

// backward y-pass map of the step: u v w phi (phi -> i ky phi) Dphi
YMap step_ymap();

// header of a ch_get_state buffer (followed by om, w, phi, h_om, h_w, h_phi)
struct StateHeader {
  uint64_t magic;
  int32_t nx, ny, nz, first;
  int64_t nstep;
  double t;
  int32_t fields_set, pad0;
  uint64_t pad[2];
};
static_assert(sizeof(StateHeader) == 64, "header size");
const uint64_t kStateMagic = 0x3130333234303632ULL;

}  // namespace chf

struct ch_grid {
  ch_params p;
  chf::GridDev g;
  int prec;
  cudaStream_t stream;
  ch_alloc_fn af;
  ch_free_fn ff;
  void* actx;
  std::vector<void*> allocs;

  // state and Adams-Bashforth history, (Mx, Ny, Nz) complex float64
  double2 *om, *w, *phi, *hom, *hw, *hphi;
  // step buffers in working precision
  void *nl, *bw, *ya, *yb;
  // auxiliary float64 buffers for set/get/diagnostics/stage entry points
  double2 *auxA, *auxB;
  double* phys7;
  // right-hand sides / solved sums of the three implicit problems (3 fields), operator table
  double2* R;
  double* fac;
  // small tables and diagnostics scratch
  double* tab;  // go1 go2 go3 ccw dzl qint, nz each
  double2* zcs; // cos(pi j / N), sin(pi j / N), j < N
  double* diag_part;
  double* diag_out;

  chf::FftPlan px[3], py[3], pz, pxu, pyu;  // px, py indexed by precision
  std::vector<chf::Tw> tws;

  long long fs;      // elements per (Mx, Ny, Nz) field
  long long fsy;     // elements per (Mx, Py, Nz) field
  long long fsp;     // elements per physical (Nz, Ny, Nx) field
  int first;         // next step starts Adams-Bashforth
  int fields_set;
  long long nstep;
  double t;
  cudaGraphExec_t gexec;
  int graph_ok;
  cudaStream_t cap;  // private non-blocking stream used only to capture the step graph

  // discrete adjoint: per-line objective partial sums and the reduced value (allocated with the
  // grid), the reverse-sweep workspace (one block, ch_adjoint_begin .. ch_adjoint_end)
  double* obj_part = nullptr;
  void* adj_block = nullptr;
  double2 *a_lam = nullptr, *a_L = nullptr, *a_Rb = nullptr, *a_mu = nullptr, *a_mu2 = nullptr;
  double2 *a_nlb = nullptr, *a_x6 = nullptr, *a_bb = nullptr;
  void* seg_block = nullptr;  // y-padded fields of the states of one recomputed segment
  int seg_cap = 0;            // states that seg_block holds
  int nl_stale = 0;  // 1: the state was replaced by a reverse step; products not recomputed

  // Chebyshev transform of the step: CH_CHEB_FFT (inside zrhs / zbwd) or CH_CHEB_TC (tensor
  // cores, two extra launches); the tables, the coefficient buffer (9 fields) and the error flag
  // of the bounded device waits exist once CH_CHEB_TC was selected
  int cheb = 0;
  chf::ChebTc tcf, tcb;
  double2* cf = nullptr;
  int* tc_err = nullptr;
};

// launch schedule of one step on stream s (events optional) and the non-linear evaluation
int ch_launch_step(ch_grid* G, int first, cudaStream_t s, cudaEvent_t* ev);
int ch_eval_nonlinear(ch_grid* G);
// u v w phi phi_x phi_y phi_z of the state on the unpadded grid into phys7 ((nz, ny, nx) each)
int ch_state_phys7(ch_grid* G);
// frees the reverse-sweep workspace if allocated
void ch_adjoint_release(ch_grid* G);
