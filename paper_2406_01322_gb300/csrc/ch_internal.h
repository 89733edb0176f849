// Host-side launchers of the solver kernels (internal to libchflow; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ch_common.cuh"

namespace chf {

// n = 2^a 3^b?
bool smooth23(int n);
// radix schedule (8 once for an odd power of two >= 3, then 4s, a 2, then 3s); false if n is
// not {2,3}-smooth or needs too many passes.  Sets pl->n, pl->nst, pl->rad (not pl->tw).
bool make_radices(int n, FftPlan* pl);
// radix schedule with a style: 0 one radix-8 for an odd power of two then 4s, 2, 3s (as
// make_radices); 1 the same with the radix-3 passes first; 2 as many radix-8 passes as possible;
// 3 one radix 3 first, then as style 2, marked for pruning (FftPlan::prune; n must be a
// multiple of 3)
bool make_radices_style(int n, int style, FftPlan* pl);
// the grid-size rules of the C ABI: 0 or a negative CH_ERR_* code
int check_sizes(int nx, int ny, int nz);

// The dynamic shared-memory limit a kernel was raised to, per device (the attribute set by
// cudaFuncSetAttribute belongs to the current device).  Zero-initialised as a static object.
// shared memory of one SM (the CTAs resident on it share it)
constexpr size_t kMaxSmemPerSm = 228 * 1024;

constexpr int kMaxSmemDevices = 64;
struct SmemLimit {
  std::atomic<int> v[kMaxSmemDevices];
};
std::mutex& smem_limit_mutex();

// Raise a kernel's dynamic shared-memory limit on the current device to `bytes` if it is below
// that; *lim remembers, per device, what was set.  Safe to call from several host threads.
// Never called while a stream is being captured (the first, uncaptured launch of every size
// comes first).
template <typename K>
inline cudaError_t ensure_smem(K* kernel, size_t bytes, SmemLimit* lim) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  const bool cached = dev >= 0 && dev < kMaxSmemDevices;
  if (cached && (int)bytes <= lim->v[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(smem_limit_mutex());
  const int have = cached ? lim->v[dev].load(std::memory_order_relaxed) : 0;
  if ((int)bytes <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // do not leave a non-sticky error behind
    return e;
  }
  if (cached) lim->v[dev].store((int)bytes, std::memory_order_release);
  return cudaSuccess;
}

// z-line kernels (one CTA per (mx, j) wavenumber line unless stated).
// zrhs: forward DCT of the 10 non-linear fields (working precision `prec`, 0 fp64 / 1 fp32),
//   assembly, AB2 (history h_* updated), right-hand sides R = [omega | theta-w | phi] (3 fields).
// zsolve: tau solves of every line (tiles of lines, one thread per elimination chain), in place
//   on R: sums omega^{n+1}+omega^n, w^{n+1}+w^n and phi^{n+1}.
// zbwd: update = 1: new state from R; then the fields for the non-linear terms, backward DCT
//   into bw (precision prec).  update = 0: from the state as is.  nout = 5: u v w phi D phi
//   (the step); nout = 7: u v w phi i kx phi, i ky phi, D phi (fp64, update = 0 only).
// Fields are (Mx, Ny, Nz) complex with field stride fs elements.
cudaError_t launch_zrhs(int prec, const GridDev& g, const void* nl, long long fs,
                        const double2* st_om, const double2* st_w, const double2* st_phi,
                        double2* h_om, double2* h_w, double2* h_phi, double2* R, int first,
                        const FftPlan& pz, cudaStream_t s);
cudaError_t launch_zsolve(const GridDev& g, double2* R, long long fs, cudaStream_t s);
cudaError_t launch_zbwd(int update, int prec, int nout, const GridDev& g, const double2* R,
                        double2* st_om, double2* st_w, double2* st_phi, void* bw, long long fs,
                        const FftPlan& pz, cudaStream_t s);
size_t zline_smem(const GridDev& g);
// the same two kernels around the tensor-core Chebyshev transform: zrhs reading the nine
// products' coefficients cf (float64), zbwd (update, 5 outputs) writing coefficients to cf
cudaError_t launch_zrhs_coef(const GridDev& g, const double2* cf, long long fs,
                             const double2* st_om, const double2* st_w, const double2* st_phi,
                             double2* h_om, double2* h_w, double2* h_phi, double2* R, int first,
                             const FftPlan& pz, cudaStream_t s);
cudaError_t zline_coef_prepare(const GridDev& g);   // shared-memory limits of the two, eagerly
cudaError_t launch_zbwd_coef(const GridDev& g, const double2* R, double2* st_om, double2* st_w,
                             double2* st_phi, double2* cf, long long fs, const FftPlan& pz,
                             cudaStream_t s);
// time-independent tau-operator table (g.fac, fac_doubles(g) doubles), built once
size_t fac_doubles(const GridDev& g);
cudaError_t build_factor_table(const GridDev& g, double* fac, cudaStream_t s);

// Projection of four physical-z fields (u, v, w, phi as (Mx, Ny, Nz) complex, already
// Fourier-transformed in x, y) onto the state (omega_z / mean flow, w, phi); zeroes history.
cudaError_t launch_project(const GridDev& g, const double2* uvwp, long long fs, double2* st_om,
                           double2* st_w, double2* st_phi, double2* h_om, double2* h_w,
                           double2* h_phi, const FftPlan& pz, cudaStream_t s);

// DCT-I of nf fields of (Mx, Ny, Nz) lines: dir 0 = samples -> coefficients (input precision
// prec), dir 1 = coefficients -> samples (fp64 in and out).
cudaError_t launch_dct_lines(int dir, int prec, const GridDev& g, const void* in, double2* out,
                             int nf, long long fs, const FftPlan& pz, cudaStream_t s);

// y pass field map: output field f reads input field src[f]; bit f of dy_mask makes the
// backward pass output i ky times the input (d/dy); kys = 2 pi / ly (set by the launcher).
struct YMap {
  static const int kMax = 16;
  int src[kMax];
  unsigned dy_mask;
  double kys;
};

// y-direction pass.  dir 1: (Mx, Ny, Nz) modes -> (Mx, P, Nz) samples (zero padding);
// dir 0: (Mx, P, Nz) samples -> (Mx, Ny, Nz) modes (truncation, Nyquist row zeroed), times scale.
// nf output fields; map == nullptr is the identity map.
cudaError_t launch_ypass(int dir, int prec, const GridDev& g, int P, const void* in, void* out,
                         int nf, long long fs_in, long long fs_out, double scale,
                         const FftPlan& py, cudaStream_t s, const YMap* map = nullptr);

// Forward y pass of the nine products with the spectral assembly's z-independent combinations
// (Eqs. (omegaz), (ww), (phisplit)) formed on the way out, so that the z stage reads and
// transforms seven lines instead of nine:
//   A = i kx Sxx' + i ky Sxy, B = i kx Sxy + i ky Syy'  (Sxx' = Sxx - Szz, Syy' = Syy - Szz)
//   0: P = i kx B - i ky A      (on the kx = ky = 0 line: Sxz)
//   1: Q = i kx Syz - i ky Sxz  (on the kx = ky = 0 line: Syz)
//   2: C = i kx Sxz + i ky Syz  3: R = i kx A + i ky B
//   4: F = -(i kx u phi + i ky v phi)   5: w phi   6: phi^3
// so that S_x = A + D Sxz, S_y = B + D Syz, h_omega = P + D Q, S_z = C,
// i kx S_x + i ky S_y = R + D C.  Work items are (input group, mx, z tile): group 0 transforms
// Sxx', Syy', Sxy (outputs 0, 3), group 1 Sxz, Syz (0 on the mean line, 1, 2), group 2 u phi,
// v phi (4), groups 3 and 4 w phi and phi^3; each group's z tile is the y pass's tile L divided
// so that a CTA holds at most max(L, 3) lines.
// q of the float32 warp-FFT path for a line of P = 96 q points (q = 1, 2, 4, 8), 0 otherwise:
// such lines are transformed by one warp each with the line in registers (32 lanes x 3 q)
__host__ __device__ __forceinline__ int warp_fft_q(int P) {
  if (P % 96 != 0) return 0;
  const int q = P / 96;
  return (q == 1 || q == 2 || q == 4 || q == 8) ? q : 0;
}
constexpr int kNc = 7;            // combined non-linear lines
constexpr int kYcGroups = 5;
__host__ __device__ __forceinline__ int ycomb_nin(int grp) {
  return grp == 0 ? 3 : (grp <= 2 ? 2 : 1);
}
// log2 of a group's z tile for a y-pass tile L (a power of two)
__host__ __device__ __forceinline__ int ycomb_tzs(int grp, int L) {
  int l = 0;
  while ((1 << (l + 1)) <= L) ++l;
  const int d = grp == 0 ? 2 : (grp <= 2 ? 1 : 0);
  return l > d ? l - d : 0;
}
__host__ __device__ __forceinline__ int ycomb_group_items(int grp, int Mx, int Nz, int L) {
  const int tzs = ycomb_tzs(grp, L);
  return ((Nz + (1 << tzs) - 1) >> tzs) * Mx;
}
inline int ycomb_items(int Mx, int Nz, int L) {
  int n = 0;
  for (int grp = 0; grp < kYcGroups; ++grp) n += ycomb_group_items(grp, Mx, Nz, L);
  return n;
}
// lines one CTA holds at most, and its shared memory (two buffers of those lines)
inline int ycomb_lines(int L) {
  int m = 0;
  for (int grp = 0; grp < kYcGroups; ++grp) {
    const int v = ycomb_nin(grp) << ycomb_tzs(grp, L);
    if (v > m) m = v;
  }
  return m;
}
inline size_t ycomb_smem(int P, int L, size_t elem) {
  return (size_t)2 * ycomb_lines(L) * yline_stride(P) * elem;
}
// in: the nine products on the y-padded grid (field stride fs_in); out: the seven combined
// lines (Mx, Ny, Nz) times `scale` (field stride fs_out); y tile from ytile_for
cudaError_t launch_ycomb(int prec, const GridDev& g, const void* in, void* out, long long fs_in,
                         long long fs_out, double scale, const FftPlan& py, cudaStream_t s);

// ---- ensemble: one member's everything the six step kernels need (device-resident array) ----
struct Member {
  GridDev g;
  FftPlan px, py, pz;             // x (Px), y (Py), z (N) plans in the working precision
  const void* nl;                 // 9 non-linear fields (Mx, Ny, Nz)
  void* bw;                       // 5 backward fields (Mx, Ny, Nz)
  void* ya;                       // 6 y-padded fields (Mx, Py, Nz)
  void* yb;                       // 9 y-padded product fields (Mx, Py, Nz)
  double2 *om, *w, *phi, *hom, *hw, *hphi, *R;
  double2* cf;                    // 9 Chebyshev coefficient fields (tensor-core method), or null
  long long fs, fsy;
  int first;                      // 1: this step starts Adams-Bashforth
  int tzb, tzf;                   // y-pass z tiles (backward, forward)
  int zsolve_tile;                // 1: shared-memory tile variant of the tau sweeps
  YMap ym;                        // backward y-pass field map of the step
  YMap yf;                        // forward y-pass field map (identity)
  double yscale;                  // 1 / (Px Py)
  double kxs;                     // 2 pi / lx
};

// Grouped persistent launches over all members: stage work items are numbered member by member,
// begin[m] = first item of member m, begin[nmem] = total; `grid` CTAs loop over the items.
// stage: 0 zrhs, 1 zsolve, 2 zbwd, 3 y backward, 4 x line, 5 y forward.  coef = 1: zrhs reads
// and zbwd writes Chebyshev coefficients in Member::cf (the tensor-core transforms run around
// them) instead of transforming along z themselves.
cudaError_t launch_grouped(int stage, int prec, const Member* mem, const int* begin, int nmem,
                           int grid, size_t smem, int zsolve_tile, int coef, int ywq,
                           cudaStream_t s);
// ywq: the y stages' warp-FFT level for the members' padded y lengths (ensemble_ywq)
int ensemble_ywq(const std::vector<int>& py, int prec);
// work items of one member for a stage, and the dynamic shared memory one item needs
int stage_items(int stage, const Member& m, int prec);
size_t stage_smem(int stage, const Member& m, int prec, int coef);
// shared memory of the coefficient-space zrhs (stage 0) or zbwd (stage 2) of a grid
size_t zline_coef_stage_smem(const GridDev& g, int stage);
// CTAs per SM that the stage kernel can hold with `smem` bytes (occupancy API)
int stage_occupancy(int stage, int prec, size_t smem, int zsolve_tile, int coef, int ywq);
// y-pass z tile for a padded length P (shared by single-grid and grouped launches)
int ytile_for(int P, size_t elem);
// shared memory of a y-pass CTA: two tiles of tz lines of yline_stride(P) elements
inline size_t ysmem_bytes(int P, int tz, size_t elem) {
  return (size_t)2 * tz * yline_stride(P) * elem;
}
// x-line shared memory for a padded length Px
size_t xline_smem(int Px, size_t elem);

// fused x-line kernel: 6 fields u v w phi phi_y phi_z (Mx, Py, Nz) -> 7 c2r (Px, with
// phi_x = i kx phi) -> 9 products -> r2c -> 9 fields.
cudaError_t launch_xline(int prec, const GridDev& g, const void* in7, void* out10, long long fs,
                         double scale, const FftPlan& px, cudaStream_t s);

// plain x transforms on the unpadded grid (fp64): physical (Nz, Ny, Nx) <-> (Mx, Ny, Nz).
cudaError_t launch_x_r2c(const GridDev& g, const double* phys, double2* out, int nf,
                         long long fs_phys, long long fs_spec, const FftPlan& px,
                         cudaStream_t s);
cudaError_t launch_x_c2r(const GridDev& g, const double2* in, double* phys, int nf,
                         long long fs_spec, long long fs_phys, const FftPlan& px,
                         cudaStream_t s);

// ---- discrete adjoint of the step (float64; transposes under the real inner product) ----
// adj_zsolve: Rb = transposed tau solves of L (adjoint of the new state, 3 fields); bb receives
//   per (line, parity) the adjoints of the omega, w and D w wall values of s_n (3 complex).
// adj_zrhs: from Rb, L, bb and mu (adjoint of this step's AB2 history h_n): lam = adjoint of the
//   state s_n except its non-linear dependence, mu_prev = adjoint of h_{n-1}, nlb = adjoint of
//   the 9 spectral non-linear fields times 1/(Px Py).
// adj_xline: transposed x-line (in6 = the forward y-padded fields of s_n, pb9 = adjoints of the
//   9 products after the transposed forward y pass) -> out6 adjoints of u v w phi phi_y phi_z.
// fold_dy: f6[3] += -i ky f6[4]; f6[4] = f6[5].
// adj_zbwd: transposed backward fields (5 inputs u v w phi D phi) accumulated into lam.
// objective: J = 1/2 int |u|^2 + int |grad phi|^2 per line into part[Mx*Ny], lam = dJ/ds.
// adj_project: transposed set_fields projection -> 4 fields scaled for the x/y transposes.
cudaError_t launch_adj_zsolve(const GridDev& g, const double2* L, double2* Rb, long long fs,
                              double2* bb, cudaStream_t s);
cudaError_t launch_adj_zrhs(const GridDev& g, const double2* Rb, const double2* L,
                            const double2* mu, double2* lam, double2* mu_prev, double2* nlb,
                            long long fs, int first, const double2* bb, const FftPlan& pz,
                            cudaStream_t s);
cudaError_t launch_adj_zbwd(const GridDev& g, const double2* in5, long long fs_in, double2* lam,
                            long long fs, const FftPlan& pz, cudaStream_t s);
cudaError_t launch_objective(const GridDev& g, const double2* om, const double2* w,
                             const double2* phi, double2* lam, long long fs, double* part,
                             cudaStream_t s);
cudaError_t launch_adj_project(const GridDev& g, const double2* lam, long long fs, double2* out4,
                               const FftPlan& pz, cudaStream_t s);
cudaError_t launch_fold_dy(const GridDev& g, double2* f6, long long fs, cudaStream_t s);
cudaError_t launch_sum(const double* a, int n, double* out, cudaStream_t s);
size_t adj_xline_smem(int Px);
cudaError_t launch_adj_xline(const GridDev& g, const double2* in6, const double2* pb9,
                             double2* out6, long long fs, const FftPlan& px, cudaStream_t s);

// diagnostics reduction over the 7 physical unpadded fields u v w phi phix phiy phiz
// (each (Nz, Ny, Nx)); out[0..8] as in ch_diag (t and step filled by the host).
cudaError_t launch_diag(const GridDev& g, const double* phys7, long long fs,
                        const double2* st_phi, const double* ccw, const double* dzl,
                        const double* qint, double* part, double* out, cudaStream_t s);

// Chebyshev transform along z as an exact-split (Ozaki) bf16 matrix product on the tensor cores
// (ch_tc.cu).  Tables of one direction (dir 0 forward: samples -> coefficients; 1 backward):
// nNt output slices of NT columns covering the outputs n < N (the kernel sums n = N exactly),
// K padded to Kp (a multiple of 16, < 512).
struct ChebTc {
  const uint16_t* dig = nullptr;   // device: per slice, per K chunk, eight NT x KC digit planes
  const int* fexp = nullptr;       // device: output-row scale exponents F_n (nNt NT entries)
  uint32_t* cache = nullptr;       // device: A digit planes of one tile per persistent CTA
  int NT = 0, nNt = 0, Kp = 0;
  int dir = 0;                     // 0 forward (samples -> coefficients), 1 backward
  int ctas = 0;                    // persistent CTAs (the cache holds ctas cheb_tc_cache_bytes)
};
// bytes of plane cache one persistent CTA needs for rows of padded length Kp
size_t cheb_tc_cache_bytes(int Kp);
// host tables; 0 or -1 (size not supported)
int cheb_tc_tables(int N, int dir, std::vector<uint16_t>& dig, std::vector<int>& fexp, int& NT,
                   int& nNt, int& Kp);
size_t cheb_tc_smem(int NT);
// raise the shared-memory limit of every instantiation for slice width NT (before any capture)
cudaError_t cheb_tc_prepare(int NT);
// nf fields of complex lines, element type tin / tout (0 float64, 1 float32, 2 double-float; the
// pairs float64 -> float64, float32 -> float64, double-float -> float64 and float64 -> float32 /
// double-float), field strides
// fsi / fso (complex elements), nlines lines of Nz; *err |= 1 if a bounded wait gave up
cudaError_t launch_cheb_tc(int tin, int tout, const void* in, long long fsi, void* out,
                           long long fso, int nf, int nlines, int Nz, const ChebTc& t, int* err,
                           cudaStream_t s);
// one bounded mbarrier wait that runs out on purpose (sets *err |= 1 after the wait bound)
cudaError_t launch_wait_selftest(int* err, int nwaits, cudaStream_t s);
// float64 FMA-rate probe: `blocks` CTAs of 256 threads, `iters` iterations of eight independent
// FMA chains per thread; out[blocks * 256] receives each thread's sum
cudaError_t launch_fma_probe(double* out, int blocks, int iters, cudaStream_t s);

}  // namespace chf
