// Ensemble of independent channels of uneven sizes advanced together.
//
// Each member is an ordinary ch_grid (its own buffers, plans and operator tables).  A step of
// the ensemble is six grouped persistent launches, one per stage (z right-hand sides, tau
// solves, z backward, y backward, x line, y forward): the CTAs of a launch walk a flat work list
// that numbers every member's tiles, so small members share the GPU instead of each leaving it
// mostly idle.  With the tensor-core Chebyshev method each member adds its two z-transform
// launches (its own persistent grid over its tiles of rows) before zrhs and after zbwd, and the
// grouped zrhs / zbwd work on coefficients.  The launches are captured once into a CUDA graph
// and replayed per step.
//
// Autotuner: for the ensemble's sizes it times, on the live ensemble (state saved and restored
// bit for bit), the radix schedules of the x, y and z transforms (three styles each, and for x and
// y a fourth: the pruned transforms of the 3/2-rule padding; chosen per transform kind from the
// stage times that use it) and the number of persistent CTAs per SM of
// each stage, and keeps the fastest.  The choice is cached per size signature for the process.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ch_flow.h"
#include "ch_grid.h"
#include "ch_internal.h"

namespace chf {
size_t zsolve_tile_smem(const GridDev& g);
int zsolve_tile_lines();
int zsolve_threads();
cudaError_t launch_grouped_z(int stage, int prec, const Member* mem, const int* begin, int nmem,
                             int grid, size_t smem, int zsolve_tile, int coef, cudaStream_t s);
cudaError_t launch_grouped_xy(int stage, int prec, const Member* mem, const int* begin, int nmem,
                              int grid, size_t smem, int ywq, cudaStream_t s);
int occupancy_z(int stage, int prec, size_t smem, int zsolve_tile, int coef);
int occupancy_xy(int stage, int prec, size_t smem, int ywq);

int stage_items(int stage, const Member& m, int prec) {
  (void)prec;
  const GridDev& g = m.g;
  const int lines = g.Mx * g.ny;
  switch (stage) {
    case 0:
    case 2: return lines;
    case 1:
      return m.zsolve_tile ? (lines + zsolve_tile_lines() - 1) / zsolve_tile_lines()
                           : (2 * lines + zsolve_threads() - 1) / zsolve_threads();
    case 3: return ((g.nz + m.tzb - 1) / m.tzb) * g.Mx * kYa;
    case 4: return ((g.nz + 1) / 2) * g.Py;
    default: return chf::ycomb_items(g.Mx, g.nz, m.tzf);
  }
}

size_t stage_smem(int stage, const Member& m, int prec, int coef) {
  const size_t elem = prec == 1 ? sizeof(float2) : sizeof(double2);   // df2 is 16 bytes too
  switch (stage) {
    case 0:
    case 2: return coef ? zline_coef_stage_smem(m.g, stage) : zline_smem(m.g);
    case 1: return m.zsolve_tile ? zsolve_tile_smem(m.g) : 0;
    case 3: return ysmem_bytes(m.g.Py, m.tzb, elem);
    case 4: return xline_smem(m.g.Px, elem);
    default: return ycomb_smem(m.g.Py, m.tzf, elem);
  }
}

int stage_occupancy(int stage, int prec, size_t smem, int zsolve_tile, int coef, int ywq) {
  return stage <= 2 ? occupancy_z(stage, prec, smem, zsolve_tile, coef)
                    : occupancy_xy(stage, prec, smem, ywq);
}

cudaError_t launch_grouped(int stage, int prec, const Member* mem, const int* begin, int nmem,
                           int grid, size_t smem, int zsolve_tile, int coef, int ywq,
                           cudaStream_t s) {
  if (stage <= 2)
    return launch_grouped_z(stage, prec, mem, begin, nmem, grid, smem, zsolve_tile, coef, s);
  return launch_grouped_xy(stage, prec, mem, begin, nmem, grid, smem, ywq, s);
}

// the grouped y-pass kernels' warp-FFT level for the members' padded y lengths (float32): 0, 2
// or 8, the largest warp-FFT q among them rounded up to an instantiated level
int ensemble_ywq(const std::vector<int>& py, int prec) {
  if (prec != 1) return 0;
  int q = 0;
  for (int P : py) q = std::max(q, warp_fft_q(P));
  return q == 0 ? 0 : (q <= 2 ? 2 : 8);
}

}  // namespace chf

using chf::Member;

namespace {

constexpr int kStages = CH_ENSEMBLE_STAGES;

struct Tuning {
  int style[3] = {0, 0, 0};        // radix style of x, y, z transforms
  int ctas_per_sm[kStages] = {0, 0, 0, 0, 0, 0};  // 0 = occupancy limit
  int tuned = 0;
};

std::mutex g_tune_mutex;
std::map<std::string, Tuning> g_tune_cache;

}  // namespace

struct ch_ensemble {
  std::vector<ch_grid*> members;
  int prec;
  int cheb;                     // Chebyshev method of the grouped step (CH_CHEB_FFT / CH_CHEB_TC)
  int nsm;
  cudaStream_t stream;
  cudaStream_t cap;
  ch_alloc_fn af;
  ch_free_fn ff;
  void* actx;
  std::vector<void*> allocs;
  Member* dmem;                 // device descriptors
  int* dbegin;                  // device work lists, kStages x (n + 1)
  std::vector<Member> hmem;
  std::vector<int> hbegin;
  size_t smem[kStages];
  int occ[kStages];
  int zsolve_tile;
  int ywq;                      // warp-FFT level of the grouped y passes (ensemble_ywq)
  int xwq;                      // the same for the grouped x line (padded x lengths)
  Tuning tune;
  std::string signature;
  cudaGraphExec_t gexec;
  int graph_ok;
};

namespace {

void* ealloc(ch_ensemble* E, size_t bytes) {
  void* p = nullptr;
  if (E->af) {
    p = E->af(bytes, E->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) E->allocs.push_back(p);
  return p;
}

void efree(ch_ensemble* E, void* p) {
  for (size_t i = 0; i < E->allocs.size(); ++i)
    if (E->allocs[i] == p) {
      if (E->ff) E->ff(p, E->actx);
      else if (!E->af) cudaFree(p);
      E->allocs.erase(E->allocs.begin() + i);
      return;
    }
}

void efree_all(ch_ensemble* E) {
  for (void* p : E->allocs) {
    if (E->ff) E->ff(p, E->actx);
    else if (!E->af) cudaFree(p);
  }
  E->allocs.clear();
}

void apply_style(chf::FftPlan* pl, int style) {
  chf::FftPlan t = *pl;
  if (chf::make_radices_style(pl->n, style, &t)) {
    t.tw = pl->tw;
    *pl = t;
  }
}

// host descriptors, work lists, per-stage shared memory and occupancy from the members
int build_descriptors(ch_ensemble* E) {
  const int n = (int)E->members.size();
  const size_t elem = E->prec == 1 ? sizeof(float2) : sizeof(double2);   // df2 is 16 bytes too
  E->hmem.resize(n);
  E->zsolve_tile = 1;
  for (int i = 0; i < n; ++i) {
    ch_grid* G = E->members[i];
    if (chf::zsolve_tile_smem(G->g) > 72 * 1024) E->zsolve_tile = 0;
  }
  for (int i = 0; i < n; ++i) {
    ch_grid* G = E->members[i];
    Member& M = E->hmem[i];
    memset(&M, 0, sizeof(M));
    M.g = G->g;
    M.px = G->px[E->prec];
    M.py = G->py[E->prec];
    M.pz = G->pz;
    apply_style(&M.px, E->tune.style[0]);
    apply_style(&M.py, E->tune.style[1]);
    apply_style(&M.pz, E->tune.style[2] == 3 ? 2 : E->tune.style[2]);
    M.nl = G->nl;
    M.bw = G->bw;
    M.ya = G->ya;
    M.yb = G->yb;
    M.om = G->om;
    M.w = G->w;
    M.phi = G->phi;
    M.hom = G->hom;
    M.hw = G->hw;
    M.hphi = G->hphi;
    M.R = G->R;
    M.cf = G->cf;
    M.fs = G->fs;
    M.fsy = G->fsy;
    M.first = G->first;
    M.tzb = chf::ytile_for(G->g.Py, elem);
    M.tzf = M.tzb;
    M.zsolve_tile = E->zsolve_tile;
    M.ym = chf::step_ymap();
    M.ym.kys = 6.283185307179586476925 / G->g.ly;
    for (int f = 0; f < chf::YMap::kMax; ++f) M.yf.src[f] = f;
    M.yf.dy_mask = 0;
    M.yf.kys = M.ym.kys;
    M.yscale = 1.0 / ((double)G->g.Px * (double)G->g.Py);
    M.kxs = 6.283185307179586476925 / G->g.lx;
  }
  E->hbegin.assign((size_t)kStages * (n + 1), 0);
  for (int s = 0; s < kStages; ++s) {
    size_t mx = 0;
    int* b = &E->hbegin[(size_t)s * (n + 1)];
    for (int i = 0; i < n; ++i) {
      b[i + 1] = b[i] + chf::stage_items(s, E->hmem[i], E->prec);
      const size_t sm = chf::stage_smem(s, E->hmem[i], E->prec, E->cheb == CH_CHEB_TC);
      if (sm > mx) mx = sm;
    }
    E->smem[s] = mx;
    if (mx > (size_t)chf::kMaxSmem) return CH_ERR_SIZE;
  }
  return CH_OK;
}

int upload(ch_ensemble* E) {
  const int n = (int)E->members.size();
  if (cudaMemcpyAsync(E->dmem, E->hmem.data(), n * sizeof(Member), cudaMemcpyHostToDevice,
                      E->stream) != cudaSuccess ||
      cudaMemcpyAsync(E->dbegin, E->hbegin.data(), E->hbegin.size() * sizeof(int),
                      cudaMemcpyHostToDevice, E->stream) != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  return CH_OK;
}

int grid_of(ch_ensemble* E, int s) {
  const int n = (int)E->members.size();
  const int total = E->hbegin[(size_t)s * (n + 1) + n];
  int per = E->tune.ctas_per_sm[s];
  if (per <= 0 || per > E->occ[s]) per = E->occ[s];
  if (per <= 0) per = 1;
  long long g = (long long)per * E->nsm;
  if (g > total) g = total;
  return g < 1 ? 1 : (int)g;
}

// tensor-core Chebyshev method: one transform launch per member around the grouped z stages,
// dir 0 (before zrhs) the nine products' samples -> coefficients, dir 1 (after zbwd) the five
// backward fields' coefficients -> samples.  Each launch is a persistent grid over that member's
// tiles of rows.
cudaError_t member_transforms(ch_ensemble* E, int dir, cudaStream_t s) {
  for (ch_grid* G : E->members) {
    const int nlines = G->g.Mx * G->g.ny;
    const cudaError_t e =
        dir == 0 ? chf::launch_cheb_tc(E->prec, 0, G->nl, G->fs, G->cf, G->fs, chf::kNc, nlines,
                                       G->g.nz, G->tcf, G->tc_err, s)
                 : chf::launch_cheb_tc(0, E->prec, G->cf, G->fs, G->bw, G->fs, chf::kBw, nlines,
                                       G->g.nz, G->tcb, G->tc_err, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one ensemble step: the six grouped stages; with the tensor-core method the member transforms
// run before stage 0 and after stage 2 and are timed with those stages
int launch_all(ch_ensemble* E, cudaStream_t s, cudaEvent_t* ev) {
  const int n = (int)E->members.size();
  const int tc = E->cheb == CH_CHEB_TC;
  for (int st = 0; st < kStages; ++st) {
    cudaError_t e = cudaSuccess;
    if (tc && st == 0) e = member_transforms(E, 0, s);
    if (e == cudaSuccess)
      e = chf::launch_grouped(st, E->prec, E->dmem, E->dbegin + (size_t)st * (n + 1), n,
                              grid_of(E, st), E->smem[st], E->zsolve_tile, tc,
                              st == 4 ? E->xwq : E->ywq, s);
    if (e == cudaSuccess && tc && st == 2) e = member_transforms(E, 1, s);
    if (ev) cudaEventRecord(ev[st], s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
  }
  return CH_OK;
}

void compute_occupancy(ch_ensemble* E) {
  std::vector<int> py, px;
  for (ch_grid* G : E->members) {
    py.push_back(G->g.Py);
    px.push_back(G->g.Px);
  }
  E->ywq = chf::ensemble_ywq(py, E->prec);
  E->xwq = chf::ensemble_ywq(px, E->prec);
  for (int s = 0; s < kStages; ++s)
    E->occ[s] = chf::stage_occupancy(s, E->prec, E->smem[s], E->zsolve_tile,
                                     E->cheb == CH_CHEB_TC, s == 4 ? E->xwq : E->ywq);
}

// tuning cache key: member sizes, precision and Chebyshev method
std::string signature_of(const ch_ensemble* E) {
  std::string sig;
  char b[64];
  // sizes and wall conditions of the members (the walls select the solve's code path)
  for (const ch_grid* G : E->members) {
    snprintf(b, sizeof(b), "%dx%dx%d:%d/", G->g.nx, G->g.ny, G->g.nz, G->g.bc);
    sig += b;
  }
  snprintf(b, sizeof(b), "p%d/c%d", E->prec, E->cheb);
  return sig + b;
}

void drop_graph(ch_ensemble* E) {
  if (E->graph_ok) cudaGraphExecDestroy(E->gexec);
  E->graph_ok = 0;
}

// brings the device descriptors' start flags in line with the members
int sync_first_flags(ch_ensemble* E) {
  bool changed = false;
  for (size_t i = 0; i < E->members.size(); ++i)
    if (E->hmem[i].first != E->members[i]->first) {
      E->hmem[i].first = E->members[i]->first;
      changed = true;
    }
  return changed ? upload(E) : CH_OK;
}

void after_step(ch_ensemble* E) {
  for (ch_grid* G : E->members) {
    G->first = 0;
    G->nstep += 1;
    G->t += G->p.dt;
  }
}

int timed_steps(ch_ensemble* E, int nsteps, double* stage_ms, double* total_ms) {
  const int nev = kStages * nsteps + 1;
  std::vector<cudaEvent_t> ev(nev);
  for (int i = 0; i < nev; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return CH_ERR_CUDA;
  int st = CH_OK;
  cudaEventRecord(ev[0], E->stream);
  for (int i = 0; i < nsteps && st == CH_OK; ++i) {
    st = sync_first_flags(E);
    if (st == CH_OK) st = launch_all(E, E->stream, &ev[kStages * i + 1]);
    after_step(E);
  }
  if (cudaEventSynchronize(ev[nev - 1]) != cudaSuccess) st = CH_ERR_CUDA;
  double ks[kStages] = {0};
  for (int i = 0; i < nsteps && st == CH_OK; ++i)
    for (int k = 0; k < kStages; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[kStages * i + k], ev[kStages * i + k + 1]);
      ks[k] += ms;
    }
  float tot = 0.f;
  cudaEventElapsedTime(&tot, ev[0], ev[nev - 1]);
  for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
  if (stage_ms)
    for (int k = 0; k < kStages; ++k) stage_ms[k] = ks[k];
  if (total_ms) *total_ms = tot;
  cudaGetLastError();
  return st;
}

}  // namespace

extern "C" {

int ch_ensemble_init(const ch_params* members, int n, ch_alloc_fn alloc, ch_free_fn free_fn,
                     void* alloc_ctx, void* stream, ch_ensemble** out) {
  if (!members || n < 1 || !out) return CH_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (members[i].precision != members[0].precision) return CH_ERR_ARG;
  ch_ensemble* E = new (std::nothrow) ch_ensemble();
  if (!E) return CH_ERR_ALLOC;
  E->prec = members[0].precision;
  E->cheb = CH_CHEB_FFT;
  E->stream = (cudaStream_t)stream;
  E->af = alloc;
  E->ff = free_fn;
  E->actx = alloc_ctx;
  E->graph_ok = 0;
  E->gexec = nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&E->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete E;
    return CH_ERR_CUDA;
  }
  int st = CH_OK;
  for (int i = 0; i < n && st == CH_OK; ++i) {
    ch_grid* G = nullptr;
    st = ch_init_grid(&members[i], alloc, free_fn, alloc_ctx, stream, &G);
    if (st == CH_OK) E->members.push_back(G);
  }
  if (st == CH_OK) E->signature = signature_of(E);
  if (st == CH_OK) {
    E->dmem = (Member*)ealloc(E, n * sizeof(Member));
    E->dbegin = (int*)ealloc(E, (size_t)kStages * (n + 1) * sizeof(int));
    if (!E->dmem || !E->dbegin) st = CH_ERR_ALLOC;
  }
  if (st == CH_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(E->signature);
    if (it != g_tune_cache.end()) E->tune = it->second;
  }
  if (st == CH_OK) st = build_descriptors(E);
  if (st == CH_OK) {
    compute_occupancy(E);
    st = upload(E);
  }
  if (st == CH_OK && cudaStreamSynchronize(E->stream) != cudaSuccess) st = CH_ERR_CUDA;
  if (st != CH_OK) {
    for (ch_grid* G : E->members) ch_destroy(G);
    efree_all(E);
    cudaStreamDestroy(E->cap);
    delete E;
    return st;
  }
  *out = E;
  return CH_OK;
}

int ch_ensemble_size(const ch_ensemble* E) { return E ? (int)E->members.size() : 0; }

int ch_ensemble_member(ch_ensemble* E, int i, ch_grid** out) {
  if (!E || !out || i < 0 || i >= (int)E->members.size()) return CH_ERR_ARG;
  *out = E->members[i];
  return CH_OK;
}

int ch_ensemble_set_chebyshev(ch_ensemble* E, int method) {
  if (!E || (method != CH_CHEB_FFT && method != CH_CHEB_TC)) return CH_ERR_ARG;
  if (method == E->cheb) return CH_OK;
  // every member takes the method (its tables and coefficient buffer stay allocated for the
  // member's lifetime once made, so a later change of a member's own method leaves the
  // ensemble's step intact)
  for (size_t i = 0; i < E->members.size(); ++i) {
    const int st = ch_set_chebyshev(E->members[i], method);
    if (st != CH_OK) {
      for (size_t j = 0; j < i; ++j) ch_set_chebyshev(E->members[j], E->cheb);
      return st;
    }
  }
  if (cudaStreamSynchronize(E->stream) != cudaSuccess) {
    cudaGetLastError();
    return CH_ERR_CUDA;
  }
  E->cheb = method;
  E->signature = signature_of(E);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(E->signature);
    E->tune = it != g_tune_cache.end() ? it->second : Tuning();
  }
  int st = build_descriptors(E);
  if (st == CH_OK) {
    compute_occupancy(E);
    st = upload(E);
  }
  drop_graph(E);
  if (st == CH_OK && cudaStreamSynchronize(E->stream) != cudaSuccess) {
    cudaGetLastError();
    st = CH_ERR_CUDA;
  }
  return st;
}

int ch_ensemble_get_chebyshev(const ch_ensemble* E) { return E ? E->cheb : CH_ERR_ARG; }

int ch_ensemble_step(ch_ensemble* E, int nsteps) {
  if (!E || nsteps < 0) return CH_ERR_ARG;
  for (ch_grid* G : E->members)
    if (!G->fields_set) return CH_ERR_STATE;
  for (int i = 0; i < nsteps; ++i) {
    int st = sync_first_flags(E);
    if (st != CH_OK) return st;
    if (!E->graph_ok) {
      cudaGraph_t graph;
      if (cudaStreamBeginCapture(E->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return CH_ERR_CUDA;
      }
      int r = launch_all(E, E->cap, nullptr);
      cudaError_t e = cudaStreamEndCapture(E->cap, &graph);
      if (r != CH_OK || e != cudaSuccess) {
        cudaGetLastError();
        return CH_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&E->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return CH_ERR_CUDA;
      }
      E->graph_ok = 1;
    }
    if (cudaGraphLaunch(E->gexec, E->stream) != cudaSuccess) {
      cudaGetLastError();
      return CH_ERR_CUDA;
    }
    after_step(E);
  }
  return CH_OK;
}

int ch_ensemble_step_timed(ch_ensemble* E, int nsteps, double* stage_ms, double* total_ms) {
  if (!E || nsteps < 0 || !total_ms) return CH_ERR_ARG;
  for (ch_grid* G : E->members)
    if (!G->fields_set) return CH_ERR_STATE;
  return timed_steps(E, nsteps, stage_ms, total_ms);
}

int ch_ensemble_autotune(ch_ensemble* E, int reps) {
  if (!E || reps < 1) return CH_ERR_ARG;
  for (ch_grid* G : E->members)
    if (!G->fields_set) return CH_ERR_STATE;
  const int n = (int)E->members.size();
  // save every member's state (restored bit for bit afterwards)
  std::vector<void*> saved(n, nullptr);
  int st = CH_OK;
  for (int i = 0; i < n && st == CH_OK; ++i) {
    saved[i] = ealloc(E, ch_state_bytes(E->members[i]));
    if (!saved[i]) st = CH_ERR_ALLOC;
    else st = ch_get_state(E->members[i], saved[i]);
  }
  Tuning best = E->tune;
  double stage_ms[kStages];
  double tot;
  // 1) radix styles, chosen per transform kind from the stages that use it (style 3, the pruned
  // transforms of the 3/2-rule padding, only for x and y: the z lines are not padded)
  double cost[3][4];
  for (int style = 0; style < 4 && st == CH_OK; ++style) {
    E->tune.style[0] = E->tune.style[1] = E->tune.style[2] = style;
    for (int s = 0; s < kStages; ++s) E->tune.ctas_per_sm[s] = 0;
    st = build_descriptors(E);
    if (st == CH_OK) st = upload(E);
    if (st == CH_OK) st = timed_steps(E, 1, stage_ms, &tot);  // warm
    if (st == CH_OK) st = timed_steps(E, reps, stage_ms, &tot);
    cost[0][style] = stage_ms[4];
    cost[1][style] = stage_ms[3] + stage_ms[5];
    cost[2][style] = stage_ms[0] + stage_ms[2];
  }
  for (int k = 0; k < 3 && st == CH_OK; ++k) {
    int b = 0;
    for (int style = 1; style < (k < 2 ? 4 : 3); ++style)
      if (cost[k][style] < cost[k][b]) b = style;
    best.style[k] = b;
  }
  // 2) persistent CTAs per SM of each stage
  const int cand[4] = {1, 2, 4, 0};
  double bestms[kStages];
  for (int s = 0; s < kStages; ++s) bestms[s] = 1e300;
  for (int c = 0; c < 4 && st == CH_OK; ++c) {
    E->tune = best;
    for (int s = 0; s < kStages; ++s) E->tune.ctas_per_sm[s] = cand[c];
    st = build_descriptors(E);
    if (st == CH_OK) st = upload(E);
    if (st == CH_OK) st = timed_steps(E, reps, stage_ms, &tot);
    for (int s = 0; s < kStages && st == CH_OK; ++s)
      if (stage_ms[s] < bestms[s]) {
        bestms[s] = stage_ms[s];
        best.ctas_per_sm[s] = cand[c];
      }
  }
  best.tuned = 1;
  E->tune = best;
  if (st == CH_OK) st = build_descriptors(E);
  // restore the states (this also restores the start flags and step counts)
  for (int i = 0; i < n && st == CH_OK; ++i) st = ch_set_state(E->members[i], saved[i]);
  if (st == CH_OK) {
    for (int i = 0; i < n; ++i) E->hmem[i].first = E->members[i]->first;
    st = upload(E);
  }
  if (cudaStreamSynchronize(E->stream) != cudaSuccess) {
    cudaGetLastError();
    if (st == CH_OK) st = CH_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i)
    if (saved[i]) efree(E, saved[i]);
  drop_graph(E);
  if (st == CH_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[E->signature] = best;
  }
  return st;
}

int ch_ensemble_tuning(const ch_ensemble* E, char* buf, size_t n) {
  if (!E || !buf || n == 0) return CH_ERR_ARG;
  snprintf(buf, n,
           "{\"tuned\": %d, \"radix_style\": {\"x\": %d, \"y\": %d, \"z\": %d}, "
           "\"ctas_per_sm\": [%d, %d, %d, %d, %d, %d], \"occupancy\": [%d, %d, %d, %d, %d, %d], "
           "\"zsolve_tile\": %d, \"chebyshev\": %d}",
           E->tune.tuned, E->tune.style[0], E->tune.style[1], E->tune.style[2],
           E->tune.ctas_per_sm[0], E->tune.ctas_per_sm[1], E->tune.ctas_per_sm[2],
           E->tune.ctas_per_sm[3], E->tune.ctas_per_sm[4], E->tune.ctas_per_sm[5], E->occ[0],
           E->occ[1], E->occ[2], E->occ[3], E->occ[4], E->occ[5], E->zsolve_tile, E->cheb);
  return CH_OK;
}

void ch_ensemble_destroy(ch_ensemble* E) {
  if (!E) return;
  cudaStreamSynchronize(E->stream);
  drop_graph(E);
  for (ch_grid* G : E->members) ch_destroy(G);
  efree_all(E);
  cudaStreamDestroy(E->cap);
  delete E;
}

}  // extern "C"
