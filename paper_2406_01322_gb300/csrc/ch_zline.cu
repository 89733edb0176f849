// Wall-normal (z-line) kernels: everything that happens along (kx, ky) Chebyshev lines.
//
// Per line (paper Sec. 2.2 steps ii)-v), Sec. 3.2.1-3.2.2):
//   forward DCT-I of the ten non-linear fields (Chebyshev coefficients, Sec. 3.2.1);
//   spectral assembly of h_omega (Eq. (omegaz)), h_w (Eq. (ww)) and S_phi (Eq. (phisplit));
//   Adams-Bashforth 2 on the non-linear terms, Crank-Nicolson on omega_z / lap(w) / mean flow,
//   implicit Euler on the split Cahn-Hilliard operator;
//   Chebyshev-tau solves in Gottlieb-Orszag quasi-tridiagonal form, split by parity and solved
//   by banded elimination (Sec. 3.2.2: tridiagonal Gauss elimination per (x, y) position), with
//   the influence-matrix (homogeneous-solution) correction for the no-slip w problem;
//   velocity from continuity and the omega_z definition (Eqs. (cont), (omegadef));
//   backward DCT-I of the seven fields the next non-linear evaluation needs.
//
// Three step kernels:
//   zrhs   (one CTA per line): DCTs, derivatives, assembly, AB2, right-hand sides -> R buffers;
//   zsolve (one CTA per tile of lines, one thread per (line, parity) elimination chain): the
//          sequential sweeps run on full warps, with operator factors from a table built once;
//   zbwd   (one CTA per line): state update, velocity recovery, backward DCTs.
//
// Crank-Nicolson is applied in "sum form": for q in {omega_z, lap(w), ubar + i vbar},
//   (D^2 - k^2 - beta)(q^{n+1} + q^n) = -2 beta q^n - 2 Re AB2(h),   beta = 2 Re / dt,
// which is the CN equation (D^2-k^2-beta) q^{n+1} = -(D^2-k^2+beta) q^n - 2 Re AB2(h) with
// (D^2-k^2-beta) q^n added to both sides; q^{n+1} + q^n satisfies the same homogeneous
// wall conditions, so the same tau problem gives it and only D^2 (not D^4) of w^n is needed.
//
// Operator table (built once by ch_init_grid; K = mx (ny/2+1) + |my| indexes distinct k^2):
//   for op in {0: D^2-(k^2+beta) Dirichlet, 1: D^2-k^2 Dirichlet, 2: D^2-(k^2+lam) Neumann}
//     Y[op][n][K], RD[op][n][K] (1/pivot), Q[op][n][K]  (n = 0..N, both parities interleaved)
//     rsq[op][p][K] = 1 / (boundary-row sum of Q for parity p)
//   Oh[n][K]  homogeneous Omega_h of the w problem, rsh[p][K] = 1 / sum_n n^2 Oh (parity p);
//   then op 3: D^2-(k^2+beta) Neumann (omega_z and the mean flow between free-slip walls), its
//   Y, RD, Q and rsq, and rsh2[p][K] = 1 / sum_n T_n''(1) Oh (parity p), appended after rsh so
//   that the offsets above do not depend on them.
// Free-slip walls (g.bc = 1): omega_z and the mean flow take Neumann rows (op 3); the w problem
// keeps its influence-matrix form with the wall rows w = w'' = 0 (the correction fixes w''
// instead of w', weights T_n''(1) = n^2 (n^2 - 1) / 3 and rsh2).
//
// All arithmetic in this file is float64.
#include "ch_internal.h"

namespace chf {

namespace {

constexpr int ZT = 128;   // threads of a per-line CTA
// threads of the coefficient-space per-line kernels (tensor-core Chebyshev method): no FFT
// passes, so twice the warps per line keep more float64 work in flight (their shared memory,
// without the DCT scratch, also leaves room for three CTAs per SM at nz = 257)
constexpr int ZTC = 256;
constexpr int NBF = 4;    // DCT lines transformed per FFT call (one warp each for scans)
constexpr int NLINES = 16;

// offsets of the table parts (op 3 sits after the influence-matrix columns)
__host__ __device__ __forceinline__ size_t fac_arr_off(const GridDev& g, int op, int arr) {
  return op < 3 ? (size_t)(op * 3 + arr) * g.nz * g.NK
                : ((size_t)10 * g.nz + 8) * g.NK + (size_t)arr * g.nz * g.NK;
}
__host__ __device__ __forceinline__ size_t fac_rsq_off(const GridDev& g, int op, int p) {
  return op < 3 ? (size_t)9 * g.nz * g.NK + (size_t)(op * 2 + p) * g.NK
                : ((size_t)13 * g.nz + 8) * g.NK + (size_t)p * g.NK;
}
__device__ __forceinline__ const double* fac_ptr(const GridDev& g, int op, int arr, int K) {
  return g.fac + fac_arr_off(g, op, arr) + K;
}
__device__ __forceinline__ double fac_rsq(const GridDev& g, int op, int p, int K) {
  return g.fac[fac_rsq_off(g, op, p) + K];
}
__device__ __forceinline__ const double* fac_oh(const GridDev& g, int K) {
  return g.fac + (size_t)9 * g.nz * g.NK + (size_t)6 * g.NK + K;
}
// 1 / sum_n T_n''(1) Oh_n over parity p (free-slip: the correction fixes w'' at the walls)
__device__ __forceinline__ double fac_rsh2(const GridDev& g, int p, int K) {
  return g.fac[((size_t)13 * g.nz + 10) * g.NK + (size_t)p * g.NK + K];
}
// influence-correction weight of coefficient n: T_n'(1) = n^2 (no-slip), T_n''(1) (free-slip)
__device__ __forceinline__ double infl_weight(int bc, int n) {
  const double n2 = (double)n * (double)n;
  return bc == 1 ? n2 * (n2 - 1.0) * (1.0 / 3.0) : n2;
}
// Different walls (g.bc = 2: no-slip at z = -1, free-slip at z = +1; 3: the mirror).  The wall
// rows no longer split into an even and an odd sum, so each parity chain leaves its lowest
// coefficient a_p free and the two rows (top, bottom) close the line with a 2x2 system in
// (a_0, a_1), exchanged between the two lanes of the line.  Tables per K (after rsh2):
// mo[4] = inverse of [[sum_even top_n Q_n, sum_odd top_n Q_n], [.. bottom ..]] (omega_z and the
// mean flow, op 0 factors), mw[4] = inverse of the same with the w-wall rows and Oh (w problem).
__host__ __device__ __forceinline__ size_t fac_mixed_off(const GridDev& g, int i) {
  return ((size_t)13 * g.nz + 12) * g.NK + (size_t)i * g.NK;
}
// wall rows at z = +1 (top) and z = -1 (bottom) of coefficient n for the mixed cases:
// omega_z rows (value at a no-slip wall, slope at a free-slip wall)
__device__ __forceinline__ double om_row(int bc, bool top, int n) {
  const double n2 = (double)n * (double)n;
  const double sgn = (n & 1) ? -1.0 : 1.0;            // T_n(-1)
  const bool free_wall = top ? (bc == 2) : (bc == 3);
  if (top) return free_wall ? n2 : 1.0;
  return free_wall ? -sgn * n2 : sgn;                 // T_n'(-1) = (-1)^(n+1) n^2
}
// w rows (slope at a no-slip wall, curvature at a free-slip wall; w = 0 is in the sweeps)
__device__ __forceinline__ double w_row(int bc, bool top, int n) {
  const double n2 = (double)n * (double)n;
  const double sgn = (n & 1) ? -1.0 : 1.0;
  const bool free_wall = top ? (bc == 2) : (bc == 3);
  const double d1 = top ? n2 : -sgn * n2;             // T_n'(+-1)
  const double d2 = (top ? 1.0 : sgn) * n2 * (n2 - 1.0) * (1.0 / 3.0);   // T_n''(+-1)
  return free_wall ? d2 : d1;
}
// sum of v over the two lanes (parities) of one line; pm = the pair's lane mask
__device__ __forceinline__ double2 pair_sum(double2 v, unsigned pm) {
  v.x += __shfl_xor_sync(pm, v.x, 1);
  v.y += __shfl_xor_sync(pm, v.y, 1);
  return v;
}
__device__ __forceinline__ double fac_rsh(const GridDev& g, int p, int K) {
  return g.fac[(size_t)10 * g.nz * g.NK + (size_t)6 * g.NK + (size_t)p * g.NK + K];
}

// kx^2 + ky^2 with one explicit fused multiply-add: the same rounding in every kernel that
// inlines it (the grouped ensemble kernels must reproduce the single-grid ones bit for bit, and an
// implicit a*b + c*d leaves the contraction to the compiler, kernel by kernel)
__device__ __forceinline__ double ksq(double kx, double ky) { return fma(kx, kx, ky * ky); }

__device__ __forceinline__ void line_wavenumbers(const GridDev& g, int line, int& mx, int& j,
                                                 double& kx, double& ky) {
  mx = line / g.ny;
  j = line - mx * g.ny;
  const int my = (j < g.ny / 2) ? j : j - g.ny;
  kx = 6.283185307179586476925 * mx / g.lx;
  ky = 6.283185307179586476925 * my / g.ly;
}

__device__ __forceinline__ int line_K(const GridDev& g, int mx, int j) {
  const int h = g.ny / 2;
  const int amy = (j <= h) ? j : g.ny - j;
  return mx * (h + 1) + amy;
}

// ---- d/dz in Chebyshev coefficient space as warp-parallel suffix sums ----------------------
// dst_n = (2 / c_n) sum_{j >= 0} (n + 1 + 2j) src_{n+1+2j} (c_0 = 2, c_n = 1 otherwise; dst_N = 0):
// within each parity class of n, a suffix sum of v_n = 2 (n + 1) src_{n+1}, halved at n = 0.
// One warp per complex line: four 8-lane segments, one per (component, parity of n); a segment's
// N/2 entries are cut into 8 contiguous chunks, each lane sums its chunk from the top (writing
// the partial sums into dst) and a 3-step segmented shuffle scan supplies the chunk offsets.
// The float64 pipe does one fused multiply-add and one addition per entry (weights 2(n+1) are
// built from integer bits; the previous 32-lane layout spent about three times as many float64
// instructions on the same sums, and the float64 rate is what bounds the z kernels).

// a positive int as float64, assembled from its bits with integer instructions only
__device__ __forceinline__ double int_as_f64(int m) {
  const int e = 31 - __clz(m);
  const unsigned long long frac =
      ((unsigned long long)(unsigned)m << (52 - e)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | frac));
}

__device__ void dz_line(const double2* src, double2* dst, int N) {
  const int lane = threadIdx.x & 31;
  const int sl = lane & 7, comp = (lane >> 3) & 1, q = lane >> 4;
  const double* s = reinterpret_cast<const double*>(src) + comp;
  double* d = reinterpret_cast<double*>(dst) + comp;
  const int K = N / 2;                  // entries n = q + 2k, k = 0..K-1
  const int E = (K + 7) >> 3;
  const int k0 = sl * E;
  double acc = 0.0;
  for (int e = E - 1; e >= 0; --e) {
    const int k = k0 + e;
    if (k < K) {
      const int n = q + 2 * k;
      acc = fma(int_as_f64(2 * n + 2), s[2 * n + 2], acc);
      d[2 * n] = acc;
    }
  }
  double v = acc;                       // inclusive suffix scan of the chunk sums in the segment
  for (int off = 1; off < 8; off <<= 1) {
    const double o = __shfl_down_sync(0xffffffffu, v, off, 8);
    if (sl + off < 8) v += o;
  }
  const double nxt = __shfl_down_sync(0xffffffffu, v, 1, 8);
  const double excl = (sl < 7) ? nxt : 0.0;
  for (int e = 0; e < E; ++e) {
    const int k = k0 + e;
    if (k < K) d[2 * (q + 2 * k)] += excl;
  }
  if (q == 0 && sl == 0) {
    d[0] *= 0.5;
    d[2 * N] = 0.0;
  }
  __syncwarp();
}

// several derivatives src[t] -> dst[t] (no aliasing between a source and any destination), one
// warp per line
__device__ void dz_tasks(double2* const* src, double2* const* dst, int ntask, int N) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < ntask; t += nw) dz_line(src[t], dst[t], N);
}

struct ZSmem {
  double2* L;   // NLINES lines of Nz
  double2* FA;  // NBF * N
  double2* FB;
};

__device__ __forceinline__ ZSmem carve(double2* sm, int Nz, int N) {
  ZSmem z;
  z.L = sm;
  z.FA = sm + NLINES * Nz;
  z.FB = z.FA + NBF * N;
  return z;
}

__device__ __forceinline__ double2* LN(const ZSmem& z, int i, int Nz) { return z.L + i * Nz; }

// DCT-I of cnt lines (in place, cnt <= NBF = number of warps):
//   E_k = x_0 + (-1)^k x_N + 2 sum_{j=1}^{N-1} x_j cos(pi j k / N),  k = 0..N,
// i.e. the 2N-point DFT of the even extension (Sec. 3.2.1), computed with ONE complex N-point
// FFT per line: with s_j = x_j + x_{N-j}, d_j = x_j - x_{N-j} (j = 0..N-1) and
// y_j = s_j + sin(pi j/N) d_j, Y = FFT_N(y):  s is even and sin(pi j/N) d_j is odd, so
//   E_{2k}   = (Y_k + Y_{N-k}) / 2,
//   E_{2k+1} = E_1 - 2 i sum_{k'=1}^{k} (Y_{k'} - Y_{N-k'}) / 2   (cos(A+B) - cos(A-B) = -2 sin A sin B),
//   E_1 = sum_j d_j cos(pi j / N).
// mode 0 (forward): x = samples f_j, result a_n = E_n / (cbar_n N).
// mode 1 (backward): x = coefficients with a_0, a_N doubled on input, result f_j = E_j / 2.
// cs[j] = (cos(pi j / N), sin(pi j / N)), j = 0..N-1.
// part 0: the complex lines (real and imaginary parts share one complex FFT); part 1 / 2: the
// real / imaginary parts alone, each as a real line (the other part of the line is neither read
// nor written).
__device__ void dct1_part(const ZSmem& z, int first, int cnt, int Nz, int N, const FftPlan& pz,
                          const double2* __restrict__ cs, int mode, int part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double e0 = (mode == 1) ? 2.0 : 1.0;   // weight of x_0 and x_N
  // the input of this part as a complex value (the other component zero for parts 1 and 2)
  auto in_val = [part](double2 v) {
    return part == 0 ? v : make_double2(part == 1 ? v.x : v.y, 0.0);
  };
  for (int idx = threadIdx.x; idx < cnt * N; idx += blockDim.x) {
    const int f = idx / N, j = idx - f * N;
    const double2* x = LN(z, first + f, Nz);
    double2 y;
    if (j == 0) {
      y = e0 * (in_val(x[0]) + in_val(x[N]));
    } else {
      const double2 a = in_val(x[j]), b = in_val(x[N - j]);
      const double sn = cs[j].y;
      // explicit fused multiply-adds: every kernel that runs this (single-grid and grouped)
      // rounds alike
      y = make_double2(fma(sn, a.x - b.x, a.x + b.x), fma(sn, a.y - b.y, a.y + b.y));
    }
    z.FA[f * N + j] = y;
  }
  // E_1 per line (warp f)
  double2 e1 = make_double2(0.0, 0.0);
  if (warp < cnt) {
    const double2* x = LN(z, first + warp, Nz);
    for (int j = lane; j < N; j += 32) {
      const double2 d = (j == 0) ? e0 * (in_val(x[0]) - in_val(x[N])) : in_val(x[j]) - in_val(x[N - j]);
      const double c = cs[j].x;
      e1.x = fma(c, d.x, e1.x);
      e1.y = fma(c, d.y, e1.y);
    }
    for (int off = 16; off > 0; off >>= 1) {
      e1.x += __shfl_xor_sync(0xffffffffu, e1.x, off);
      e1.y += __shfl_xor_sync(0xffffffffu, e1.y, off);
    }
  }
  __syncthreads();
  const double2* R = block_fft<double, false>(z.FA, z.FB, cnt, N, pz);
  const double sc0 = (mode == 0) ? 0.5 / N : 0.5;   // scale of E_0 and E_N
  const double sc = (mode == 0) ? 1.0 / N : 0.5;    // scale of the others
  // the result of this part into the line (parts 1 and 2: the real part of E into the part's
  // component; its imaginary part is rounding only)
  auto put = [part](double2* dst, double2 v) {
    if (part == 0) *dst = v;
    else if (part == 1) dst->x = v.x;
    else dst->y = v.x;
  };
  // even outputs
  for (int idx = threadIdx.x; idx < cnt * (N / 2 + 1); idx += blockDim.x) {
    const int f = idx / (N / 2 + 1), k = idx - f * (N / 2 + 1);
    const double2 a = R[f * N + k], b = R[f * N + (k == 0 ? 0 : N - k)];
    const double s = (k == 0 || 2 * k == N) ? sc0 : sc;
    put(LN(z, first + f, Nz) + 2 * k, (0.5 * s) * (a + b));
  }
  // odd outputs: prefix sums of Q_k = (Y_k - Y_{N-k}) / 2 over k = 1..N/2-1 (warp f)
  if (warp < cnt) {
    const double2* Y = R + warp * N;
    double2* out = LN(z, first + warp, Nz);
    const int M = N / 2;                    // odd outputs E_1, E_3, .., E_{N-1}: k = 0..M-1
    const int E = (M + 31) / 32;
    const int k0 = lane * E;
    double2 acc = make_double2(0.0, 0.0);
    for (int e = 0; e < E; ++e) {
      const int k = k0 + e;
      if (k >= 1 && k < M) acc = acc + 0.5 * (Y[k] - Y[N - k]);
    }
    double2 v = acc;                        // inclusive scan of chunk sums over lanes
    for (int off = 1; off < 32; off <<= 1) {
      const double ox = __shfl_up_sync(0xffffffffu, v.x, off);
      const double oy = __shfl_up_sync(0xffffffffu, v.y, off);
      if (lane >= off) { v.x += ox; v.y += oy; }
    }
    // exclusive prefix of this lane's chunk = inclusive value of the lane below
    const double px = __shfl_up_sync(0xffffffffu, v.x, 1);
    const double py = __shfl_up_sync(0xffffffffu, v.y, 1);
    double2 T = (lane == 0) ? make_double2(0.0, 0.0) : make_double2(px, py);
    for (int e = 0; e < E; ++e) {
      const int k = k0 + e;
      if (k < M) {
        if (k >= 1) T = T + 0.5 * (Y[k] - Y[N - k]);
        // E_{2k+1} = E_1 - 2 i T
        put(out + 2 * k + 1, sc * make_double2(e1.x + 2.0 * T.y, e1.y - 2.0 * T.x));
      }
    }
  }
  __syncthreads();
}

// DCT-I of cnt lines.  split: transform the real and imaginary parts separately (two real
// transforms) instead of as one complex line.  The complex FFT mixes the rounding of the two
// parts; on the mean line (kx = ky = 0) the imaginary part is the spanwise mean flow, orders of
// magnitude below the streamwise one in the real part, and would otherwise carry the real
// part's rounding.
__device__ void dct1_lines(const ZSmem& z, int first, int cnt, int Nz, int N, const FftPlan& pz,
                           const double2* __restrict__ cs, int mode, bool split = false) {
  if (!split) {
    dct1_part(z, first, cnt, Nz, N, pz, cs, mode, 0);
  } else {
    dct1_part(z, first, cnt, Nz, N, pz, cs, mode, 1);
    dct1_part(z, first, cnt, Nz, N, pz, cs, mode, 2);
  }
}

// forward DCT-I of cnt lines in place (samples -> coefficients), cnt <= NBF
__device__ __forceinline__ void dct_forward_lines(const ZSmem& z, int first, int cnt, int Nz, int N,
                                                  const FftPlan& pz, const double2* cs,
                                                  bool split = false) {
  dct1_lines(z, first, cnt, Nz, N, pz, cs, 0, split);
}

// backward DCT-I of cnt lines (coefficients -> samples), results stored to
// out[(out_first + f) * fs + off + j]
template <typename T2>
__device__ void dct_backward_lines_store(const ZSmem& z, int first, int cnt, int Nz, int N,
                                         const FftPlan& pz, const double2* cs, T2* out,
                                         long long fs, size_t off, int out_first,
                                         bool split = false) {
  dct1_lines(z, first, cnt, Nz, N, pz, cs, 1, split);
  for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
    const int f = idx / Nz, j = idx - f * Nz;
    out[(long long)(out_first + f) * fs + off + j] = from_d2<T2>(LN(z, first + f, Nz)[j]);
  }
  __syncthreads();
}

// ---- zrhs: right-hand sides of the three implicit problems ---------------------------------
// nl: the seven combined non-linear lines (launch_ycomb) as samples on the Gauss-Lobatto points.
// PRE = 1: nl holds their Chebyshev coefficients (float64, transformed by the tensor-core
// kernel), so the forward DCTs are skipped.
template <typename T, int PRE = 0, int GST = PRE>
__device__ __forceinline__ void zrhs_body(const GridDev& g, const typename C2<T>::t* __restrict__ nl,
                                          long long fs, const double2* __restrict__ st_om,
                                          const double2* __restrict__ st_w,
                                          const double2* __restrict__ st_phi,
                                          double2* __restrict__ h_om, double2* __restrict__ h_w,
                                          double2* __restrict__ h_phi, double2* __restrict__ R,
                                          int first, const FftPlan& pz, int line) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const int tid = threadIdx.x;
  double2* Rom = R;
  double2* Rth = R + fs;
  double2* Rps = R + 2 * fs;
  if (j == g.ny / 2) {  // y Nyquist row: identically zero
    for (int n = tid; n < Nz; n += blockDim.x) {
      Rom[off + n] = make_double2(0.0, 0.0);
      Rth[off + n] = make_double2(0.0, 0.0);
      Rps[off + n] = make_double2(0.0, 0.0);
    }
    return;
  }
  const ZSmem z = carve(zsm, Nz, N);
  const bool is00 = (mx == 0 && j == 0);
  const double k2 = ksq(kx, ky);
  // shared lines: 0..6 the combined non-linear lines, 11 w; 7..10 and 12 derivatives, reused as
  // the sweep goes on.  omega and phi: lines 13 and 14 (GST = 0), or read from global memory
  // where they are used (GST = 1, the single-grid coefficient-space variant: thirteen lines,
  // four CTAs per SM at nz = 257); the arithmetic is the same either way
  for (int n = tid; n < Nz; n += blockDim.x) {
    LN(z, 11, Nz)[n] = st_w[off + n];
    if (!GST) {
      LN(z, 13, Nz)[n] = st_om[off + n];
      LN(z, 14, Nz)[n] = st_phi[off + n];
    }
  }
  const double2* phs = GST ? st_phi + off : LN(z, 14, Nz);   // phi^n and omega^n of this line
  const double2* oms = GST ? st_om + off : LN(z, 13, Nz);
  // The seven combined non-linear lines, formed by the forward y pass (the Chebyshev transform
  // commutes with the z-independent factors i kx, i ky):
  //   0: P = i kx B - i ky A   1: Q = i kx Syz - i ky Sxz   (h_omega = P + D Q)
  //   2: C = i kx Sxz + i ky Syz  (S_z = C)   3: R = i kx A + i ky B  (i kx S_x + i ky S_y = R + D C)
  //   4: F = -(i kx u phi + i ky v phi)   5: w phi   6: phi^3
  // with A = i kx Sxx' + i ky Sxy, B = i kx Sxy + i ky Syy' (S_x = A + D Sxz, S_y = B + D Syz).
  // On the (0,0) line lines 0 and 1 carry Sxz and Syz (mean forcing).
  for (int idx = tid; idx < kNc * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    LN(z, f, Nz)[n] = to_d2(nl[(long long)f * fs + off + n]);
  }
  __syncthreads();
  if (!PRE)
    for (int f0 = 0; f0 < 7; f0 += NBF)
      dct_forward_lines(z, f0, (7 - f0 < NBF) ? 7 - f0 : NBF, Nz, N, pz, g.zcs, is00);
  // G = phi^3 - (1 + shat) phi
  for (int n = tid; n < Nz; n += blockDim.x)
    LN(z, 6, Nz)[n] = LN(z, 6, Nz)[n] - (1.0 + g.shat) * phs[n];
  __syncthreads();
  // Seven derivatives (D is linear, so the second derivatives of the assembly are taken of
  // sums): h_w = -k^2 C - D(R + D C), S_phi = F - (k^2 / Pe) G + D(D G / Pe - w phi),
  // theta^n = D^2 w - k^2 w, h_omega = P + D Q.
  {
    double2* src[5] = {LN(z, 1, Nz), LN(z, 2, Nz), LN(z, 6, Nz), LN(z, 11, Nz), LN(z, 0, Nz)};
    double2* dst[5] = {LN(z, 7, Nz), LN(z, 9, Nz), LN(z, 8, Nz), LN(z, 12, Nz), LN(z, 10, Nz)};
    dz_tasks(src, dst, is00 ? 5 : 4, N);   // DQ, DC, DG, Dw (, D Sxz on (0,0))
  }
  __syncthreads();
  const double rpe = 1.0 / g.pe;
  const double k2rpe = k2 * rpe;
  for (int n = tid; n < Nz; n += blockDim.x) {
    const double2 c = LN(z, 3, Nz)[n], dc = LN(z, 9, Nz)[n];
    const double2 wp = LN(z, 5, Nz)[n], dg = LN(z, 8, Nz)[n];
    const double2 f = LN(z, 4, Nz)[n], gg = LN(z, 6, Nz)[n];
    LN(z, 3, Nz)[n] = c + dc;                                                  // R + D C
    LN(z, 5, Nz)[n] = make_double2(fma(rpe, dg.x, -wp.x), fma(rpe, dg.y, -wp.y));  // D G / Pe - w phi
    LN(z, 4, Nz)[n] = make_double2(fma(-k2rpe, gg.x, f.x), fma(-k2rpe, gg.y, f.y));  // F - k^2 G / Pe
  }
  __syncthreads();
  {
    double2* src[3] = {LN(z, 3, Nz), LN(z, 5, Nz), LN(z, 12, Nz)};
    double2* dst[3] = {LN(z, 8, Nz), LN(z, 9, Nz), LN(z, 1, Nz)};
    dz_tasks(src, dst, 3, N);   // D(R + D C), D(D G / Pe - w phi), D^2 w
  }
  __syncthreads();
  // h_omega, h_w, S_phi, theta^n = (D^2 - k^2) w^n; AB2 folded into the right-hand sides:
  //   R_q = -2 beta q^n - 2 Re (a h^n + b h^{n-1}),  R_phi = (Pe / Ch^2)(phi^n / dt + a S^n + b S^{n-1})
  // with (a, b) = (3/2, -1/2), or (1, 0) on the first step
  const double cphi = g.pe / (g.ch * g.ch);
  const double cb = -2.0 * g.beta;
  const double ca = first ? -2.0 * g.re : -3.0 * g.re, cm = g.re;    // -2 Re a, -2 Re b
  const double pa = first ? cphi : 1.5 * cphi, pm = -0.5 * cphi;     // cphi a, cphi b
  const double prd = cphi / g.dt;
  for (int n = tid; n < Nz; n += blockDim.x) {
    double2 hom, hw;
    if (is00) {  // mean flow: Sbar_x + i Sbar_y + (gx + i gy) delta_{n0}
      hom = make_double2(LN(z, 10, Nz)[n].x + (n == 0 ? g.gx : 0.0),
                         LN(z, 7, Nz)[n].x + (n == 0 ? g.gy : 0.0));
      hw = make_double2(0.0, 0.0);
    } else {
      const double2 c = LN(z, 2, Nz)[n], d = LN(z, 8, Nz)[n];
      hom = LN(z, 0, Nz)[n] + LN(z, 7, Nz)[n];                                  // P + D Q
      hw = make_double2(fma(-k2, c.x, -d.x), fma(-k2, c.y, -d.y));             // -k^2 C - D(R + D C)
    }
    const double2 sphi = LN(z, 4, Nz)[n] + LN(z, 9, Nz)[n];
    const double2 w = LN(z, 11, Nz)[n], d2w = LN(z, 1, Nz)[n];
    const double2 th = make_double2(fma(-k2, w.x, d2w.x), fma(-k2, w.y, d2w.y));
    const double2 om = oms[n], ph = phs[n];
    double2 r0 = make_double2(cb * om.x, cb * om.y);
    double2 r1 = make_double2(cb * th.x, cb * th.y);
    double2 r2 = make_double2(prd * ph.x, prd * ph.y);
    if (!first) {
      const double2 o0 = h_om[off + n], o1 = h_w[off + n], o2 = h_phi[off + n];
      r0 = make_double2(fma(cm, o0.x, r0.x), fma(cm, o0.y, r0.y));
      r1 = make_double2(fma(cm, o1.x, r1.x), fma(cm, o1.y, r1.y));
      r2 = make_double2(fma(pm, o2.x, r2.x), fma(pm, o2.y, r2.y));
    }
    h_om[off + n] = hom;
    h_w[off + n] = hw;
    h_phi[off + n] = sphi;
    Rom[off + n] = make_double2(fma(ca, hom.x, r0.x), fma(ca, hom.y, r0.y));
    Rth[off + n] = make_double2(fma(ca, hw.x, r1.x), fma(ca, hw.y, r1.y));
    Rps[off + n] = make_double2(fma(pa, sphi.x, r2.x), fma(pa, sphi.y, r2.y));
  }
}

template <typename T, int PRE = 0>
__global__ void __launch_bounds__(PRE ? ZTC : ZT) zrhs_kernel(GridDev g, const typename C2<T>::t* __restrict__ nl,
                                                  long long fs, const double2* __restrict__ st_om,
                                                  const double2* __restrict__ st_w,
                                                  const double2* __restrict__ st_phi,
                                                  double2* __restrict__ h_om,
                                                  double2* __restrict__ h_w,
                                                  double2* __restrict__ h_phi,
                                                  double2* __restrict__ R, int first, FftPlan pz) {
  zrhs_body<T, PRE>(g, nl, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, R, first, pz, blockIdx.x);
}

// ---- tau elimination with tabulated factors -----------------------------------------------
// Solve (D^2 - alpha) a = f (Gottlieb-Orszag rows n >= 2, homogeneous boundary row) for the
// coefficients of parity p of one complex line, in place (x[n] = f_n on entry, a_n on exit).
// Y, RD, Q point at (op, arr, n = 0, K) with stride NK per n; wb = 1 (Dirichlet) or n^2.
// The table entries come from global memory (L2) and do not depend on the recurrence: each
// sweep fetches them KP at a time into registers ahead of the dependent steps, so one memory
// latency covers KP steps (the arithmetic and its order are unchanged).
constexpr int KP = 8;

// XF: also fetch the chunk's right-hand sides x[n] ahead (x in global memory; the shared-memory
// tile variant reads them in place)
template <bool XF>
__device__ void tau_sweep_c(double2* x, int p, int N, double alpha, bool neumann,
                            const double* t1, const double* t2, const double* t3,
                            const double* __restrict__ Y, const double* __restrict__ RD,
                            const double* __restrict__ Q, int NK, double rsq) {
  const int I = (N - p) / 2;
  double2 xn = make_double2(0.0, 0.0), fnp2 = make_double2(0.0, 0.0);
  for (int i0 = I; i0 >= 1; i0 -= KP) {
    // the chunk's table entries and right-hand sides (x[n] is read before its own step writes
    // it and after no other), fetched ahead of the recurrence
    double f[KP];
    double2 xv[KP + 1];
#pragma unroll
    for (int u = 0; u < KP; ++u)
      f[u] = (i0 - u >= 1) ? __ldg(RD + (size_t)(p + 2 * (i0 - u)) * NK) : 0.0;
#pragma unroll
    for (int u = 0; u <= KP; ++u)
      if (XF) xv[u] = (i0 - u >= 0) ? x[p + 2 * (i0 - u)] : make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 - u;
      if (i >= 1) {
        const int n = p + 2 * i;
        const double2 fn = XF ? xv[u] : x[n];
        const double2 fnm2 = XF ? xv[u + 1] : x[n - 2];
        const double a1 = t1[n], a2 = t2[n], a3 = t3[n];
        const double U = -alpha * a3;
        const double rd = f[u];
        double2 xi;
        xi.x = fma(-U, xn.x, fma(a1, fnm2.x, fma(-a2, fn.x, a3 * fnp2.x))) * rd;
        xi.y = fma(-U, xn.y, fma(a1, fnm2.y, fma(-a2, fn.y, a3 * fnp2.y))) * rd;
        x[n] = xi;
        fnp2 = fn;
        xn = xi;
      }
    }
  }
  double2 P = make_double2(0.0, 0.0), sp = make_double2(0.0, 0.0);
  for (int i0 = 1; i0 <= I; i0 += KP) {
    double f[KP];
    double2 xc[KP];
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      f[u] = (i0 + u <= I) ? __ldg(Y + (size_t)(p + 2 * (i0 + u)) * NK) : 0.0;
      if (XF) xc[u] = (i0 + u <= I) ? x[p + 2 * (i0 + u)] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 + u;
      if (i <= I) {
        const int n = p + 2 * i;
        const double y = f[u];
        const double2 xv = XF ? xc[u] : x[n];
        P.x = fma(y, P.x, xv.x);
        P.y = fma(y, P.y, xv.y);
        x[n] = P;
        const double wb = neumann ? int_as_f64(n * n) : 1.0;
        sp.x = fma(wb, P.x, sp.x);
        sp.y = fma(wb, P.y, sp.y);
      }
    }
  }
  const double2 a0 = make_double2(-sp.x * rsq, -sp.y * rsq);
  x[p] = a0;
  for (int i0 = 1; i0 <= I; i0 += KP) {
    double f[KP];
#pragma unroll
    for (int u = 0; u < KP; ++u)
      f[u] = (i0 + u <= I) ? __ldg(Q + (size_t)(p + 2 * (i0 + u)) * NK) : 0.0;
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 + u;
      if (i <= I) {
        const int n = p + 2 * i;
        double2 v = x[n];
        v.x = fma(f[u], a0.x, v.x);
        v.y = fma(f[u], a0.y, v.y);
        x[n] = v;
      }
    }
  }
}

// Different walls: as tau_sweep_c (Dirichlet/Neumann flag unused) but closed by the two wall
// rows of g.bc together with the partner lane's chain: a_p = -row p of minv . (top, bottom row
// sums of P over both parities); minv points at the four inverse entries (stride NK).
__device__ void tau_sweep_mixed(double2* __restrict__ x, int p, int N, double alpha, int bc,
                                const double* __restrict__ t1, const double* __restrict__ t2,
                                const double* __restrict__ t3, const double* __restrict__ Y,
                                const double* __restrict__ RD, const double* __restrict__ Q,
                                int NK, const double* __restrict__ minv, unsigned pm) {
  const int I = (N - p) / 2;
  double2 xn = make_double2(0.0, 0.0), fnp2 = make_double2(0.0, 0.0);
  for (int i = I; i >= 1; --i) {
    const int n = p + 2 * i;
    const double2 fn = x[n];
    const double2 fnm2 = x[n - 2];
    const double a1 = t1[n], a2 = t2[n], a3 = t3[n];
    const double U = -alpha * a3;
    const double rd = RD[(size_t)n * NK];
    double2 xi;
    xi.x = fma(-U, xn.x, fma(a1, fnm2.x, fma(-a2, fn.x, a3 * fnp2.x))) * rd;
    xi.y = fma(-U, xn.y, fma(a1, fnm2.y, fma(-a2, fn.y, a3 * fnp2.y))) * rd;
    x[n] = xi;
    fnp2 = fn;
    xn = xi;
  }
  double2 P = make_double2(0.0, 0.0), st = P, sb = P;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    const double y = Y[(size_t)n * NK];
    const double2 xv = x[n];
    P.x = fma(y, P.x, xv.x);
    P.y = fma(y, P.y, xv.y);
    x[n] = P;
    const double bt = om_row(bc, true, n), bb = om_row(bc, false, n);
    st.x = fma(bt, P.x, st.x);
    st.y = fma(bt, P.y, st.y);
    sb.x = fma(bb, P.x, sb.x);
    sb.y = fma(bb, P.y, sb.y);
  }
  st = pair_sum(st, pm);
  sb = pair_sum(sb, pm);
  const double m0 = minv[(size_t)(2 * p) * NK], m1 = minv[(size_t)(2 * p + 1) * NK];
  const double2 a0 = make_double2(-fma(m0, st.x, m1 * sb.x), -fma(m0, st.y, m1 * sb.y));
  x[p] = a0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    const double q = Q[(size_t)n * NK];
    double2 v = x[n];
    v.x = fma(q, a0.x, v.x);
    v.y = fma(q, a0.y, v.y);
    x[n] = v;
  }
}

// Different walls, w problem: Omega = Omega_p + c_0 Oh_even + c_1 Oh_odd with the top and bottom
// w-wall rows zero (Omega_p holds w = 0 at both walls already); c from the 2x2 inverse mw.
__device__ void w_correct_mixed(const GridDev& g, double2* __restrict__ row, int p, int K,
                                unsigned pm) {
  const int N = g.N;
  const double* oh = fac_oh(g, K);
  double2 rt = make_double2(0.0, 0.0), rb = rt;
  for (int n = p; n <= N; n += 2) {
    const double bt = w_row(g.bc, true, n), bb = w_row(g.bc, false, n);
    rt.x = fma(bt, row[n].x, rt.x);
    rt.y = fma(bt, row[n].y, rt.y);
    rb.x = fma(bb, row[n].x, rb.x);
    rb.y = fma(bb, row[n].y, rb.y);
  }
  rt = pair_sum(rt, pm);
  rb = pair_sum(rb, pm);
  const double* mw = g.fac + fac_mixed_off(g, 4) + K;
  const double m0 = mw[(size_t)(2 * p) * g.NK], m1 = mw[(size_t)(2 * p + 1) * g.NK];
  const double2 c = make_double2(-fma(m0, rt.x, m1 * rb.x), -fma(m0, rt.y, m1 * rb.y));
  for (int n = p; n <= N; n += 2) {
    const double h = oh[(size_t)n * g.NK];
    double2 v = row[n];
    v.x = fma(c.x, h, v.x);
    v.y = fma(c.y, h, v.y);
    row[n] = v;
  }
}

// zsolve: one thread per (line, parity) elimination chain, sweeping in place on R in global
// memory (line-major like the state).  The two chains of a line sit in adjacent lanes and touch
// adjacent coefficients, so each warp access covers 16 lines x 32 bytes; a chain's half-line is
// re-read by its three passes while still in L1/L2.  No shared memory, so occupancy is set by
// registers.  R holds [omega | theta-w | phi] right-hand sides on entry and the solved sums /
// new phi on exit.
constexpr int ST = 128;   // threads per zsolve CTA
__device__ __forceinline__ void zsolve_body(const GridDev& g, double2* __restrict__ R, long long fs,
                                            int nlines, int t) {
  const int N = g.N, Nz = g.nz;
  const int line = t >> 1, p = t & 1;
  if (line >= nlines) return;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const int K = line_K(g, mx, j);
  const double k2 = ksq(kx, ky);
  const bool is00 = (mx == 0 && j == 0);
  const double* t1 = g.go1;
  const double* t2 = g.go2;
  const double* t3 = g.go3;
  // omega (or the mean flow on the (0,0) line): (D^2 - k^2 - beta) Q = r, Dirichlet rows
  // (no-slip) or Neumann rows (free-slip, op 3)
  const bool fsl = (g.bc == 1);
  const bool mixed = (g.bc >= 2);                 // a different condition on each wall
  const unsigned pm = 0x3u << (threadIdx.x & 30);  // the two lanes (parities) of this line
  const int oo = fsl ? 3 : 0;
  double2* row = R + (size_t)line * Nz;
  if (mixed)
    tau_sweep_mixed(row, p, N, k2 + g.beta, g.bc, t1, t2, t3, fac_ptr(g, 0, 0, K),
                    fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK,
                    g.fac + fac_mixed_off(g, 0) + K, pm);
  else
    tau_sweep_c<true>(row, p, N, k2 + g.beta, fsl, t1, t2, t3, fac_ptr(g, oo, 0, K),
                fac_ptr(g, oo, 1, K), fac_ptr(g, oo, 2, K), g.NK, fac_rsq(g, oo, p, K));
  // w: influence problem (theta, w) with w = w' = 0 at both walls, or (free-slip) theta and w
  // each with Dirichlet rows
  row = R + fs + (size_t)line * Nz;
  if (is00) {
    for (int n = p; n <= N; n += 2) row[n] = make_double2(0.0, 0.0);
  } else {
    tau_sweep_c<true>(row, p, N, k2 + g.beta, false, t1, t2, t3, fac_ptr(g, 0, 0, K),
                fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK, fac_rsq(g, 0, p, K));
    tau_sweep_c<true>(row, p, N, k2, false, t1, t2, t3, fac_ptr(g, 1, 0, K), fac_ptr(g, 1, 1, K),
                fac_ptr(g, 1, 2, K), g.NK, fac_rsq(g, 1, p, K));
  }
  if (!is00 && mixed) {
    w_correct_mixed(g, row, p, K, pm);
  } else if (!is00) {
    // Omega = Omega_p + c Omega_h with D Omega(+-1) = 0 (no-slip) or D^2 Omega(+-1) = 0
    // (free-slip), parity p
    const double* oh = fac_oh(g, K);
    double2 sacc = make_double2(0.0, 0.0);
    for (int n = p; n <= N; n += 2) {
      const double n2 = infl_weight(g.bc, n);
      const double2 v = row[n];
      sacc.x = fma(n2, v.x, sacc.x);
      sacc.y = fma(n2, v.y, sacc.y);
    }
    const double rsh = fsl ? fac_rsh2(g, p, K) : fac_rsh(g, p, K);
    const double2 c = make_double2(-sacc.x * rsh, -sacc.y * rsh);
    for (int n = p; n <= N; n += 2) {
      const double h = oh[(size_t)n * g.NK];
      double2 v = row[n];
      v.x = fma(c.x, h, v.x);
      v.y = fma(c.y, h, v.y);
      row[n] = v;
    }
  }
  // phi: two Neumann problems with the same operator (D^2 - k^2 - lam)
  row = R + 2 * fs + (size_t)line * Nz;
  const double a = k2 + g.lam;
  for (int rep = 0; rep < 2; ++rep)
    tau_sweep_c<true>(row, p, N, a, true, t1, t2, t3, fac_ptr(g, 2, 0, K), fac_ptr(g, 2, 1, K),
                fac_ptr(g, 2, 2, K), g.NK, fac_rsq(g, 2, p, K));
}

__global__ void __launch_bounds__(ST) zsolve_kernel(GridDev g, double2* __restrict__ R,
                                                    long long fs, int nlines) {
  zsolve_body(g, R, fs, nlines, blockIdx.x * blockDim.x + threadIdx.x);
}

constexpr int TL = 32;    // lines per tile-variant CTA (2 TL chains: one per (line, parity))
constexpr int TLT = 256;  // threads of a tile-variant CTA: the first 2 TL solve, all move the tile

// copy of count elements by the whole CTA with eight 16-byte loads in flight per thread (the
// tile's moves between global and shared memory are latency-bound with few threads per SM)
__device__ __forceinline__ void tile_copy(double2* __restrict__ dst,
                                          const double2* __restrict__ src, int count) {
  const int nt = blockDim.x;
  int idx = threadIdx.x;
  for (; idx + 7 * nt < count; idx += 8 * nt) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = src[idx + u * nt];
#pragma unroll
    for (int u = 0; u < 8; ++u) dst[idx + u * nt] = v[u];
  }
  for (; idx < count; idx += nt) dst[idx] = src[idx];
}

// One of the three implicit problems of one line (row = its coefficients in shared memory,
// parity p of the chain): 0 omega (or the mean flow), 1 the w influence problem, 2 phi.
__device__ __forceinline__ void solve_tile_problem(const GridDev& g, double2* __restrict__ row,
                                                   int prob, int p, int K, double k2, bool is00,
                                                   const double* __restrict__ t1,
                                                   const double* __restrict__ t2,
                                                   const double* __restrict__ t3, unsigned pm) {
  const int N = g.N;
  if (prob == 0) {
    const bool fsl = (g.bc == 1);     // free-slip: Neumann rows (op 3)
    const int oo = fsl ? 3 : 0;
    if (g.bc >= 2)                    // a different condition on each wall
      tau_sweep_mixed(row, p, N, k2 + g.beta, g.bc, t1, t2, t3, fac_ptr(g, 0, 0, K),
                      fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK,
                      g.fac + fac_mixed_off(g, 0) + K, pm);
    else
      tau_sweep_c<false>(row, p, N, k2 + g.beta, fsl, t1, t2, t3, fac_ptr(g, oo, 0, K),
                  fac_ptr(g, oo, 1, K), fac_ptr(g, oo, 2, K), g.NK, fac_rsq(g, oo, p, K));
  } else if (prob == 1) {
    if (is00) {
      for (int n = p; n <= N; n += 2) row[n] = make_double2(0.0, 0.0);
    } else {
      tau_sweep_c<false>(row, p, N, k2 + g.beta, false, t1, t2, t3, fac_ptr(g, 0, 0, K),
                  fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK, fac_rsq(g, 0, p, K));
      tau_sweep_c<false>(row, p, N, k2, false, t1, t2, t3, fac_ptr(g, 1, 0, K), fac_ptr(g, 1, 1, K),
                  fac_ptr(g, 1, 2, K), g.NK, fac_rsq(g, 1, p, K));
    }
    if (!is00 && g.bc >= 2) {
      w_correct_mixed(g, row, p, K, pm);
    } else if (!is00) {
      // influence matrix: Omega = Omega_p + c Omega_h with D Omega(+-1) = 0 (no-slip) or
      // D^2 Omega(+-1) = 0 (free-slip), parity p
      const double* oh = fac_oh(g, K);
      double2 sacc = make_double2(0.0, 0.0);
      for (int n = p; n <= N; n += 2) {
        const double n2 = infl_weight(g.bc, n);
        sacc.x = fma(n2, row[n].x, sacc.x);
        sacc.y = fma(n2, row[n].y, sacc.y);
      }
      const double rsh = g.bc == 1 ? fac_rsh2(g, p, K) : fac_rsh(g, p, K);
      const double2 c = make_double2(-sacc.x * rsh, -sacc.y * rsh);
      for (int n = p; n <= N; n += 2) {
        const double h = oh[(size_t)n * g.NK];
        double2 v = row[n];
        v.x = fma(c.x, h, v.x);
        v.y = fma(c.y, h, v.y);
        row[n] = v;
      }
    }
  } else {
    const double a = k2 + g.lam;
    for (int rep = 0; rep < 2; ++rep)
      tau_sweep_c<false>(row, p, N, a, true, t1, t2, t3, fac_ptr(g, 2, 0, K), fac_ptr(g, 2, 1, K),
                  fac_ptr(g, 2, 2, K), g.NK, fac_rsq(g, 2, p, K));
  }
}

// zsolve, tile variant (short lines): TL lines per CTA staged in shared memory, thread = (line,
// parity), the three problems in turn.  R holds [omega | theta-w | phi] right-hand sides on
// entry and the solved sums / new phi on exit (line-major, like the state).
__device__ __forceinline__ void zsolve_tile_body(const GridDev& g, double2* __restrict__ R,
                                                 long long fs, int nlines, int bid) {
  extern __shared__ double2 ssm[];
  const int Nz = g.nz;
  double2* tile = ssm;
  double* t1 = reinterpret_cast<double*>(ssm + TL * Nz);
  double* t2 = t1 + Nz;
  double* t3 = t2 + Nz;
  const int tid = threadIdx.x;
  const int l = tid >> 1, p = tid & 1;
  const int line0 = bid * TL;
  const int line = line0 + l;
  for (int n = tid; n < Nz; n += blockDim.x) {
    t1[n] = g.go1[n];
    t2[n] = g.go2[n];
    t3[n] = g.go3[n];
  }
  int mx = 0, j = 0, K = 0;
  double kx = 0.0, ky = 0.0;
  const bool valid = tid < 2 * TL && line < nlines;
  if (valid) {
    line_wavenumbers(g, line, mx, j, kx, ky);
    K = line_K(g, mx, j);
  }
  const double k2 = ksq(kx, ky);
  const bool is00 = (mx == 0 && j == 0);
  const int ntile = min(TL, nlines - line0);
  const unsigned pm = 0x3u << (threadIdx.x & 30);  // the two lanes of this line
  for (int prob = 0; prob < 3; ++prob) {
    double2* Rp = R + prob * fs + (size_t)line0 * Nz;
    tile_copy(tile, Rp, ntile * Nz);
    __syncthreads();
    if (valid) solve_tile_problem(g, tile + l * Nz, prob, p, K, k2, is00, t1, t2, t3, pm);
    __syncthreads();
    tile_copy(Rp, tile, ntile * Nz);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TLT) zsolve_tile_kernel(GridDev g, double2* __restrict__ R,
                                                        long long fs, int nlines) {
  zsolve_tile_body(g, R, fs, nlines, blockIdx.x);
}

// ---- operator table (init time) -------------------------------------------------------------
__device__ __forceinline__ void K_wavenumbers(const GridDev& g, int K, double& k2) {
  const int h = g.ny / 2;
  const int mx = K / (h + 1), amy = K - mx * (h + 1);
  const double kx = 6.283185307179586476925 * mx / g.lx;
  const double ky = 6.283185307179586476925 * amy / g.ly;
  k2 = ksq(kx, ky);
}

// thread = (K, op, parity): elimination from the top coefficient down; the boundary row
// closes the system at n = p
__global__ void factor_kernel(GridDev g, double* __restrict__ fac) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.NK * 8) return;
  const int K = t / 8, op = (t % 8) >> 1, p = t & 1;
  double k2;
  K_wavenumbers(g, K, k2);
  const double alpha = (op == 0 || op == 3) ? k2 + g.beta : (op == 1) ? k2 : k2 + g.lam;
  const bool neumann = (op >= 2);
  const int N = g.N, NK = g.NK;
  double* Y = fac + fac_arr_off(g, op, 0) + K;
  double* RD = fac + fac_arr_off(g, op, 1) + K;
  double* Q = fac + fac_arr_off(g, op, 2) + K;
  const int I = (N - p) / 2;
  double ynext = 0.0;
  for (int i = I; i >= 1; --i) {
    const int n = p + 2 * i;
    const double L = -alpha * g.go1[n];
    const double Dg = 1.0 + alpha * g.go2[n];
    const double U = -alpha * g.go3[n];
    const double rd = 1.0 / fma(U, ynext, Dg);
    const double y = -L * rd;
    Y[(size_t)n * NK] = y;
    RD[(size_t)n * NK] = rd;
    ynext = y;
  }
  double q = 1.0;
  Y[(size_t)p * NK] = 0.0;
  RD[(size_t)p * NK] = 0.0;
  Q[(size_t)p * NK] = 1.0;
  double sq = neumann ? (double)(p * p) : 1.0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    q *= Y[(size_t)n * NK];
    Q[(size_t)n * NK] = q;
    sq = fma(neumann ? (double)n * (double)n : 1.0, q, sq);
  }
  fac[fac_rsq_off(g, op, p) + K] = 1.0 / sq;
}

// thread = (K, parity): Psi_h = Q_0 / SQ_0 (operator 0 with unit wall value), then
// (D^2 - k^2) Omega_h = Psi_h with Dirichlet walls; also 1 / sum n^2 Omega_h
__global__ void homog_kernel(GridDev g, double* __restrict__ fac) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.NK * 2) return;
  const int K = t >> 1, p = t & 1;
  const int N = g.N, NK = g.NK, Nz = g.nz;
  double k2;
  K_wavenumbers(g, K, k2);
  double* oh = fac + (size_t)9 * Nz * NK + (size_t)6 * NK + K;
  const double* Q0 = fac + ((size_t)(0 * 3 + 2) * Nz) * NK + K;
  const double rsq0 = fac[(size_t)9 * Nz * NK + (size_t)(0 * 2 + p) * NK + K];
  for (int n = p; n <= N; n += 2) oh[(size_t)n * NK] = Q0[(size_t)n * NK] * rsq0;
  // Dirichlet sweep with operator 1 (real, strided)
  const double* Y = fac + ((size_t)(1 * 3 + 0) * Nz) * NK + K;
  const double* RD = fac + ((size_t)(1 * 3 + 1) * Nz) * NK + K;
  const double* Q = fac + ((size_t)(1 * 3 + 2) * Nz) * NK + K;
  const double rsq = fac[(size_t)9 * Nz * NK + (size_t)(1 * 2 + p) * NK + K];
  const int I = (N - p) / 2;
  double xn = 0.0, fnp2 = 0.0;
  for (int i = I; i >= 1; --i) {
    const int n = p + 2 * i;
    const double fn = oh[(size_t)n * NK];
    const double fnm2 = oh[(size_t)(n - 2) * NK];
    const double U = -k2 * g.go3[n];
    const double xi = fma(-U, xn, fma(g.go1[n], fnm2, fma(-g.go2[n], fn, g.go3[n] * fnp2))) *
                      RD[(size_t)n * NK];
    oh[(size_t)n * NK] = xi;
    fnp2 = fn;
    xn = xi;
  }
  double P = 0.0, sp = 0.0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    P = fma(Y[(size_t)n * NK], P, oh[(size_t)n * NK]);
    oh[(size_t)n * NK] = P;
    sp += P;
  }
  const double a0 = -sp * rsq;
  oh[(size_t)p * NK] = a0;
  double sh = 0.0, sh2 = 0.0;
  for (int i = 0; i <= I; ++i) {
    const int n = p + 2 * i;
    double v = oh[(size_t)n * NK];
    if (i > 0) v = fma(Q[(size_t)n * NK], a0, v);
    oh[(size_t)n * NK] = v;
    const double n2 = (double)n * (double)n;
    sh = fma(n2, v, sh);
    sh2 = fma(n2 * (n2 - 1.0) * (1.0 / 3.0), v, sh2);
  }
  fac[(size_t)10 * Nz * NK + (size_t)6 * NK + (size_t)p * NK + K] = (sh != 0.0) ? 1.0 / sh : 0.0;
  fac[((size_t)13 * Nz + 10) * NK + (size_t)p * NK + K] = (sh2 != 0.0) ? 1.0 / sh2 : 0.0;
}

// thread = K: the 2x2 wall closures of the different-walls cases (inverses stored row-major)
__device__ void store_inverse(double* out, size_t NK, double a, double b, double c, double d) {
  const double det = a * d - b * c;
  const double r = (det != 0.0) ? 1.0 / det : 0.0;
  out[0] = d * r;
  out[NK] = -b * r;
  out[2 * NK] = -c * r;
  out[3 * NK] = a * r;
}

__global__ void mixed_kernel(GridDev g, double* __restrict__ fac) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= g.NK) return;
  const int N = g.N;
  const size_t NK = g.NK;
  const double* Q0 = fac + fac_arr_off(g, 0, 2) + K;       // Q_p = 1 at n = p
  const double* oh = fac + (size_t)9 * g.nz * NK + (size_t)6 * NK + K;
  double so[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, sw[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int n = 0; n <= N; ++n) {
    const int c = n & 1;
    const double q = Q0[(size_t)n * NK], h = oh[(size_t)n * NK];
    so[0][c] += om_row(g.bc, true, n) * q;
    so[1][c] += om_row(g.bc, false, n) * q;
    sw[0][c] += w_row(g.bc, true, n) * h;
    sw[1][c] += w_row(g.bc, false, n) * h;
  }
  store_inverse(fac + fac_mixed_off(g, 0) + K, NK, so[0][0], so[0][1], so[1][0], so[1][1]);
  store_inverse(fac + fac_mixed_off(g, 4) + K, NK, sw[0][0], sw[0][1], sw[1][0], sw[1][1]);
}

// ---- zbwd: update + the fields for the non-linear terms ------------------------------------
// UPDATE = 1: new state = (solved sums - old state) for omega, w and phi from R; = 0: state as is.
// Output (backward DCT-I to samples in z): NOUT = 5: u, v (continuity + omega_z definition), w,
// phi, D phi (the step: i kx phi and i ky phi are formed by the x and y passes); NOUT = 7:
// u, v, w, phi, i kx phi, i ky phi, D phi.
// COEF = 1: the NOUT lines are stored as Chebyshev coefficients (float64, bw typed double2) for
// the tensor-core backward transform instead of being transformed here.
template <typename T, int UPDATE, int NOUT, int COEF = 0>
__device__ __forceinline__ void zbwd_body(const GridDev& g, const double2* __restrict__ R,
                                          double2* __restrict__ st_om, double2* __restrict__ st_w,
                                          double2* __restrict__ st_phi,
                                          typename C2<T>::t* __restrict__ bw, long long fs,
                                          const FftPlan& pz, int line) {
  typedef typename C2<T>::t T2;
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const int tid = threadIdx.x;
  if (j == g.ny / 2) {
    for (int idx = tid; idx < NOUT * Nz; idx += blockDim.x) {
      const int f = idx / Nz, n = idx - f * Nz;
      bw[(long long)f * fs + off + n] = from_d2<T2>(make_double2(0.0, 0.0));
    }
    return;
  }
  const ZSmem z = carve(zsm, Nz, N);
  const bool is00 = (mx == 0 && j == 0);
  // shared lines: omega, w, phi, D w, D phi (the coefficient-space variant keeps only these
  // five, lines 0..4, and stores its outputs straight from registers; the DCT variant keeps them
  // in lines 10..14 and assembles the outputs in lines 0..NOUT-1 for its transforms)
  constexpr int LOM = COEF ? 0 : 10;
  double2* Lom = LN(z, LOM, Nz);
  double2* Lw = LN(z, LOM + 1, Nz);
  double2* Lph = LN(z, LOM + 2, Nz);
  double2* Ldw = LN(z, LOM + 3, Nz);
  double2* Ldp = LN(z, LOM + 4, Nz);
  for (int n = tid; n < Nz; n += blockDim.x) {
    double2 om = st_om[off + n], w = st_w[off + n], ph = st_phi[off + n];
    if (UPDATE) {
      om = R[off + n] - om;           // (q^{n+1} + q^n) - q^n
      w = R[fs + off + n] - w;
      ph = R[2 * fs + off + n];
      st_om[off + n] = om;
      st_w[off + n] = w;
      st_phi[off + n] = ph;
    }
    Lom[n] = om;
    Lw[n] = w;
    Lph[n] = ph;
  }
  __syncthreads();
  {
    double2* src[2] = {Lw, Lph};
    double2* dst[2] = {Ldw, Ldp};
    dz_tasks(src, dst, 2, N);
  }
  __syncthreads();
  const double k2 = ksq(kx, ky);
  const double rk2 = is00 ? 0.0 : 1.0 / k2;
  for (int n = tid; n < Nz; n += blockDim.x) {
    const double2 om = Lom[n];
    const double2 dw = Ldw[n];
    const double2 ph = Lph[n];
    double2 u, v;
    if (is00) {
      u = make_double2(om.x, 0.0);
      v = make_double2(om.y, 0.0);
    } else {
      // u = (i kx Dw + i ky om) / k^2,  v = (i ky Dw - i kx om) / k^2
      u = rk2 * mul_i(kx * dw + ky * om);
      v = rk2 * mul_i(ky * dw - kx * om);
    }
    if (COEF) {
      // NOUT = 5: u v w phi D phi
      bw[off + n] = from_d2<T2>(u);
      bw[fs + off + n] = from_d2<T2>(v);
      bw[2 * fs + off + n] = from_d2<T2>(Lw[n]);
      bw[3 * fs + off + n] = from_d2<T2>(ph);
      bw[4 * fs + off + n] = from_d2<T2>(Ldp[n]);
      continue;
    }
    LN(z, 0, Nz)[n] = u;
    LN(z, 1, Nz)[n] = v;
    LN(z, 2, Nz)[n] = Lw[n];
    LN(z, 3, Nz)[n] = ph;
    if (NOUT == 7) {
      LN(z, 4, Nz)[n] = kx * mul_i(ph);
      LN(z, 5, Nz)[n] = ky * mul_i(ph);
      LN(z, 6, Nz)[n] = Ldp[n];
    } else {
      LN(z, 4, Nz)[n] = Ldp[n];
    }
  }
  if (COEF) return;
  __syncthreads();
  // as few rounds of at most NBF lines as possible, balanced (5 fields: 3 + 2, not 4 + 1, so no
  // round runs a lone line through the barrier-separated FFT passes)
  constexpr int NR = (NOUT + NBF - 1) / NBF;
  int f0 = 0;
  for (int r = 0; r < NR; ++r) {
    const int cnt = (NOUT - f0 + (NR - r) - 1) / (NR - r);
    dct_backward_lines_store<T2>(z, f0, cnt, Nz, N, pz, g.zcs, bw, fs, off, f0, is00);
    f0 += cnt;
  }
}

template <typename T, int UPDATE, int NOUT, int COEF = 0>
__global__ void __launch_bounds__(COEF ? ZTC : ZT) zbwd_kernel(GridDev g, const double2* __restrict__ R,
                                                  double2* __restrict__ st_om,
                                                  double2* __restrict__ st_w,
                                                  double2* __restrict__ st_phi,
                                                  typename C2<T>::t* __restrict__ bw,
                                                  long long fs, FftPlan pz) {
  zbwd_body<T, UPDATE, NOUT, COEF>(g, R, st_om, st_w, st_phi, bw, fs, pz, blockIdx.x);
}

// set_fields projection: u, v, w, phi samples (after the x/y transforms) -> state
__global__ void __launch_bounds__(ZT) project_kernel(GridDev g, const double2* __restrict__ in,
                                                     long long fs, double2* st_om, double2* st_w,
                                                     double2* st_phi, double2* h_om,
                                                     double2* h_w, double2* h_phi, FftPlan pz) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const bool nyq = (j == g.ny / 2);
  const bool is00 = (mx == 0 && j == 0);
  const ZSmem z = carve(zsm, Nz, N);
  for (int idx = threadIdx.x; idx < 4 * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    LN(z, f, Nz)[n] = in[(long long)f * fs + off + n];
  }
  __syncthreads();
  dct_forward_lines(z, 0, 4, Nz, N, pz, g.zcs, is00);
  const double2 zero = make_double2(0.0, 0.0);
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 u = LN(z, 0, Nz)[n], v = LN(z, 1, Nz)[n];
    double2 om;
    if (is00) om = make_double2(u.x, v.x);           // ubar + i vbar
    else om = mul_i(kx * v - ky * u);                // i kx v - i ky u
    st_om[off + n] = nyq ? zero : om;
    st_w[off + n] = (nyq || is00) ? zero : LN(z, 2, Nz)[n];
    st_phi[off + n] = nyq ? zero : LN(z, 3, Nz)[n];
    h_om[off + n] = zero;
    h_w[off + n] = zero;
    h_phi[off + n] = zero;
  }
}

// DCT-I of nf fields per line (dir 0: samples -> coefficients; dir 1: coefficients -> samples)
template <typename T>
__global__ void __launch_bounds__(ZT) dct_lines_kernel(GridDev g, int dir,
                                                       const typename C2<T>::t* __restrict__ in,
                                                       double2* __restrict__ out, int nf,
                                                       long long fs, FftPlan pz) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const size_t off = (size_t)blockIdx.x * Nz;
  const ZSmem z = carve(zsm, Nz, N);
  for (int f0 = 0; f0 < nf; f0 += NBF) {
    const int cnt = (nf - f0 < NBF) ? nf - f0 : NBF;
    for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
      const int f = idx / Nz, n = idx - f * Nz;
      LN(z, f, Nz)[n] = to_d2(in[(long long)(f0 + f) * fs + off + n]);
    }
    __syncthreads();
    if (dir == 0) {
      dct_forward_lines(z, 0, cnt, Nz, N, pz, g.zcs, blockIdx.x == 0);
      for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
        const int f = idx / Nz, n = idx - f * Nz;
        out[(long long)(f0 + f) * fs + off + n] = LN(z, f, Nz)[n];
      }
      __syncthreads();
    } else {
      dct_backward_lines_store<double2>(z, 0, cnt, Nz, N, pz, g.zcs, out, fs, off, f0,
                                        blockIdx.x == 0);
    }
  }
}

// ---- diagnostics: per-block partial sums / maxima, then one finishing block
constexpr int DT = 256;

__global__ void __launch_bounds__(DT) diag_partial_kernel(GridDev g, const double* __restrict__ f7,
                                                          long long fs, const double* __restrict__ ccw,
                                                          const double* __restrict__ dzl,
                                                          double* __restrict__ part) {
  const long long npt = (long long)g.nz * g.ny * g.nx;
  const double dx = g.lx / g.nx, dy = g.ly / g.ny;
  double ke = 0, g2s = 0, fe = 0, cfl = 0, mphi = 0, nan = 0;
  for (long long i = blockIdx.x * (long long)DT + threadIdx.x; i < npt; i += (long long)gridDim.x * DT) {
    const int k = (int)(i / ((long long)g.ny * g.nx));
    const double wk = ccw[k] * dx * dy;
    const double u = f7[i], v = f7[fs + i], w = f7[2 * fs + i], ph = f7[3 * fs + i];
    const double fx = f7[4 * fs + i], fy = f7[5 * fs + i], fz = f7[6 * fs + i];
    const double gg = fx * fx + fy * fy + fz * fz;
    ke += 0.5 * wk * (u * u + v * v + w * w);
    g2s += wk * gg;
    const double q = ph * ph - 1.0;
    fe += wk * (0.25 * q * q + 0.5 * g.ch * g.ch * gg);
    const double c = g.dt * (fabs(u) / dx + fabs(v) / dy + fabs(w) / dzl[k]);
    cfl = fmax(cfl, c);
    mphi = fmax(mphi, fabs(ph));
    if (!isfinite(u) || !isfinite(v) || !isfinite(w) || !isfinite(ph)) nan = 1.0;
  }
  __shared__ double red[6][DT];
  red[0][threadIdx.x] = ke;
  red[1][threadIdx.x] = g2s;
  red[2][threadIdx.x] = fe;
  red[3][threadIdx.x] = cfl;
  red[4][threadIdx.x] = mphi;
  red[5][threadIdx.x] = nan;
  __syncthreads();
  for (int s = DT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      for (int q = 3; q < 6; ++q) red[q][threadIdx.x] = fmax(red[q][threadIdx.x], red[q][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void diag_final_kernel(GridDev g, int nblk, const double* __restrict__ part,
                                  const double2* __restrict__ st_phi, const double* __restrict__ qint,
                                  double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[3] = {0, 0, 0}, m[3] = {0, 0, 0};
  for (int b = 0; b < nblk; ++b) {
    for (int q = 0; q < 3; ++q) s[q] += part[b * 6 + q];
    for (int q = 0; q < 3; ++q) m[q] = fmax(m[q], part[b * 6 + 3 + q]);
  }
  double mass = 0.0;  // line (0,0) is the first line of the state
  for (int n = 0; n < g.nz; ++n) mass = fma(qint[n], st_phi[n].x, mass);
  out[0] = mass * g.lx * g.ly;
  out[1] = s[0];
  out[2] = s[1];
  out[3] = s[2];
  out[4] = m[0];
  out[5] = m[1];
  out[6] = m[2];
}

// ---- discrete adjoint of the step (float64) ----------------------------------------------
// Transposes are taken with respect to the real inner product <a, b> = sum Re(conj(a) b) over
// the stored components, so multiplication by a complex constant c transposes to conj(c).

// D^T in coefficient space: (D^T l)_p = 2 p sum_{n < p, n + p odd} l_n / c_n (c_0 = 2), so
// (D^T l)_0 = 0 and, for p = n + 1, a prefix sum over the parity class of n of w_n = l_n / c_n,
// times 2p.  Same warp layout as dz_line (four 8-lane segments, one per (component, parity of
// n), contiguous chunks, segmented shuffle scan); two float64 additions and one multiplication
// per entry.
__device__ void dzT_line(const double2* src, double2* dst, int N) {
  const int lane = threadIdx.x & 31;
  const int sl = lane & 7, comp = (lane >> 3) & 1, r = lane >> 4;
  const double* s = reinterpret_cast<const double*>(src) + comp;
  double* d = reinterpret_cast<double*>(dst) + comp;
  const int K = N / 2;                  // sources n = r + 2k, k = 0..K-1, output p = n + 1
  const int E = (K + 7) >> 3;
  const int k0 = sl * E;
  double acc = 0.0;
  for (int e = 0; e < E; ++e) {
    const int k = k0 + e;
    if (k < K) {
      const int n = r + 2 * k;
      acc += (n == 0) ? 0.5 * s[0] : s[2 * n];
      d[2 * n + 2] = acc;
    }
  }
  double v = acc;                       // inclusive prefix scan of the chunk sums in the segment
  for (int off = 1; off < 8; off <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, v, off, 8);
    if (sl >= off) v += o;
  }
  const double prv = __shfl_up_sync(0xffffffffu, v, 1, 8);
  const double excl = (sl > 0) ? prv : 0.0;
  for (int e = 0; e < E; ++e) {
    const int k = k0 + e;
    if (k < K) {
      const int p = r + 2 * k + 1;
      d[2 * p] = int_as_f64(2 * p) * (d[2 * p] + excl);
    }
  }
  if (r == 1 && sl == 0) d[0] = 0.0;
  __syncwarp();
}

__device__ void dzT_tasks(double2* const* src, double2* const* dst, int ntask, int N) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = warp; t < ntask; t += nw) dzT_line(src[t], dst[t], N);
}

// transpose of tau_sweep_c for parity p of one complex line, in place (x: solution adjoint in,
// right-hand-side adjoint out).  Reverses: a_i = P_i + Q_i a_0; a_0 = -rsq sum beta_i P_i;
// P_i = X_i + Y_i P_{i-1}; X_i = (g_i - U_i X_{i+1}) rd_i; g_i = t1 f_{n-2} - t2 f_n + t3 f_{n+2}.
// Returns rsq times the adjoint of a_0, which is the adjoint of the boundary-row value b when the
// row reads sum_n wb_n a_n = b (a_0 = (b - sum wb P) rsq; the forward sweep has b = 0).
__device__ double2 tau_sweep_ct(double2* x, int p, int N, double alpha, bool neumann,
                                const double* t1, const double* t2, const double* t3,
                                const double* __restrict__ Y, const double* __restrict__ RD,
                                const double* __restrict__ Q, int NK, double rsq) {
  const int I = (N - p) / 2;
  // a_0 collects the Q-weighted adjoints of a_1..a_I (table entries fetched KP at a time, as in
  // tau_sweep_c)
  double2 a0 = x[p];
  for (int i0 = 1; i0 <= I; i0 += KP) {
    double f[KP];
#pragma unroll
    for (int u = 0; u < KP; ++u)
      f[u] = (i0 + u <= I) ? __ldg(Q + (size_t)(p + 2 * (i0 + u)) * NK) : 0.0;
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int n = p + 2 * (i0 + u);
      if (i0 + u <= I) {
        a0.x = fma(f[u], x[n].x, a0.x);
        a0.y = fma(f[u], x[n].y, a0.y);
      }
    }
  }
  // P_i adjoint = a_i adjoint - rsq beta_i a_0 adjoint
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    const double wb = neumann ? int_as_f64(n * n) : 1.0;
    const double c = -rsq * wb;
    double2 v = x[n];
    v.x = fma(c, a0.x, v.x);
    v.y = fma(c, a0.y, v.y);
    x[n] = v;
  }
  // X adjoint: X_i = P_i + Y_{i+1} X_{i+1} (from the top)
  double2 xn = make_double2(0.0, 0.0);
  for (int i0 = I; i0 >= 1; i0 -= KP) {
    double f[KP];
    double2 xc[KP];
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 - u;
      f[u] = (i >= 1 && i < I) ? __ldg(Y + (size_t)(p + 2 * i + 2) * NK) : 0.0;
      xc[u] = (i >= 1) ? x[p + 2 * i] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 - u;
      if (i >= 1) {
        const int n = p + 2 * i;
        double2 v = xc[u];
        if (i < I) {
          v.x = fma(f[u], xn.x, v.x);
          v.y = fma(f[u], xn.y, v.y);
        }
        x[n] = v;
        xn = v;
      }
    }
  }
  // g adjoint: g_1 = X_1 rd_1, g_i = (X_i - U_{i-1} g_{i-1}) rd_i
  double2 gp = make_double2(0.0, 0.0);
  for (int i0 = 1; i0 <= I; i0 += KP) {
    double f[KP];
    double2 xc[KP];
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      f[u] = (i0 + u <= I) ? __ldg(RD + (size_t)(p + 2 * (i0 + u)) * NK) : 0.0;
      xc[u] = (i0 + u <= I) ? x[p + 2 * (i0 + u)] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < KP; ++u) {
      const int i = i0 + u;
      if (i <= I) {
        const int n = p + 2 * i;
        const double rd = f[u];
        double2 v = xc[u];
        if (i > 1) {
          const double U = -alpha * t3[n - 2];
          v.x = fma(-U, gp.x, v.x);
          v.y = fma(-U, gp.y, v.y);
        }
        v.x *= rd;
        v.y *= rd;
        x[n] = v;
        gp = v;
      }
    }
  }
  // f adjoint from the stencil: f_{n_k} = t1[n_{k+1}] g_{k+1} - t2[n_k] g_k + t3[n_{k-1}] g_{k-1}
  double2 gprev = make_double2(0.0, 0.0);  // g_{k-1}
  for (int k = 0; k <= I; ++k) {
    const int n = p + 2 * k;
    const double2 gk = (k >= 1) ? x[n] : make_double2(0.0, 0.0);
    const double2 gn = (k + 1 <= I) ? x[n + 2] : make_double2(0.0, 0.0);
    double2 f = make_double2(0.0, 0.0);
    if (k + 1 <= I) {
      f.x = t1[n + 2] * gn.x;
      f.y = t1[n + 2] * gn.y;
    }
    if (k >= 1) {
      f.x = fma(-t2[n], gk.x, f.x);
      f.y = fma(-t2[n], gk.y, f.y);
    }
    if (k >= 2) {
      f.x = fma(t3[n - 2], gprev.x, f.x);
      f.y = fma(t3[n - 2], gprev.y, f.y);
    }
    x[n] = f;
    gprev = gk;
  }
  return make_double2(rsq * a0.x, rsq * a0.y);
}

// adjoint of zsolve + state update: one thread per (line, parity); L = adjoint of the new
// state (3 fields), Rb = adjoint of the right-hand sides (3 fields, written).
// The adjoint differentiates the literal Crank-Nicolson map, whose solves impose the wall
// conditions on q^{n+1}.  The forward sweeps solve for S = q^{n+1} + q^n with homogeneous wall
// rows; on states that meet the wall conditions that is the same as imposing S's wall values =
// q^n's, and the adjoint of those values goes back to q^n: bb[(line, p)] = (omega wall value,
// w wall value, D w wall value) adjoints of parity p, added to the state adjoint by adj_zrhs.
__global__ void __launch_bounds__(ST) adj_zsolve_kernel(GridDev g, const double2* __restrict__ L,
                                                        double2* __restrict__ Rb, long long fs,
                                                        int nlines, double2* __restrict__ bb) {
  const int N = g.N, Nz = g.nz;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int line = t >> 1, p = t & 1;
  if (line >= nlines) return;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const int K = line_K(g, mx, j);
  const double k2 = ksq(kx, ky);
  const bool is00 = (mx == 0 && j == 0);
  const bool nyq = (j == g.ny / 2);
  const double *t1 = g.go1, *t2 = g.go2, *t3 = g.go3;
  const double2 zero = make_double2(0.0, 0.0);
  double2* bl = bb + (size_t)t * 3;
  for (int f = 0; f < 3; ++f) {
    const double2* in = L + f * fs + (size_t)line * Nz;
    double2* row = Rb + f * fs + (size_t)line * Nz;
    for (int n = p; n <= N; n += 2) row[n] = nyq ? zero : in[n];
  }
  if (nyq) {
    bl[0] = zero;
    bl[1] = zero;
    bl[2] = zero;
    return;
  }
  // omega (and the mean flow): S = Sol_beta(r; wall value of omega^n)
  double2* row = Rb + (size_t)line * Nz;
  bl[0] = tau_sweep_ct(row, p, N, k2 + g.beta, false, t1, t2, t3, fac_ptr(g, 0, 0, K),
                       fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK, fac_rsq(g, 0, p, K));
  // w: S_w = Omega_p + c Omega_h, Omega_p = Sol_0(Sol_beta r; wall value of w^n),
  //    c = (D w^n wall value - sum n^2 Omega_p) rsh
  row = Rb + fs + (size_t)line * Nz;
  if (is00) {
    for (int n = p; n <= N; n += 2) row[n] = zero;
    bl[1] = zero;
    bl[2] = zero;
  } else {
    const double* oh = fac_oh(g, K);
    const double rsh = fac_rsh(g, p, K);
    double2 sacc = zero;
    for (int n = p; n <= N; n += 2) {
      const double h = oh[(size_t)n * g.NK];
      sacc.x = fma(h, row[n].x, sacc.x);
      sacc.y = fma(h, row[n].y, sacc.y);
    }
    const double2 bD = make_double2(rsh * sacc.x, rsh * sacc.y);
    for (int n = p; n <= N; n += 2) {
      const double c = -(double)n * (double)n;
      double2 v = row[n];
      v.x = fma(c, bD.x, v.x);
      v.y = fma(c, bD.y, v.y);
      row[n] = v;
    }
    bl[2] = bD;
    bl[1] = tau_sweep_ct(row, p, N, k2, false, t1, t2, t3, fac_ptr(g, 1, 0, K),
                         fac_ptr(g, 1, 1, K), fac_ptr(g, 1, 2, K), g.NK, fac_rsq(g, 1, p, K));
    tau_sweep_ct(row, p, N, k2 + g.beta, false, t1, t2, t3, fac_ptr(g, 0, 0, K),
                 fac_ptr(g, 0, 1, K), fac_ptr(g, 0, 2, K), g.NK, fac_rsq(g, 0, p, K));
  }
  // phi: two Neumann solves with the same operator (implicit Euler: no wall-value term)
  row = Rb + 2 * fs + (size_t)line * Nz;
  for (int rep = 0; rep < 2; ++rep)
    tau_sweep_ct(row, p, N, k2 + g.lam, true, t1, t2, t3, fac_ptr(g, 2, 0, K), fac_ptr(g, 2, 1, K),
                 fac_ptr(g, 2, 2, K), g.NK, fac_rsq(g, 2, p, K));
}

// transpose of the forward DCT on lines [first, first+cnt): a = F x with F[n][j] =
// scale_n w_j cos(pi n j / N)  ->  x_bar = w (.) C (scale (.) a_bar), C the backward transform
__device__ void dct_forward_transpose_lines(const ZSmem& z, int first, int cnt, int Nz, int N,
                                            const FftPlan& pz, const double2* cs) {
  for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    const double sc = (n == 0 || n == N) ? 0.5 / N : 1.0 / N;
    LN(z, first + f, Nz)[n] = sc * LN(z, first + f, Nz)[n];
  }
  __syncthreads();
  dct1_lines(z, first, cnt, Nz, N, pz, cs, 1);
  for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
    const int f = idx / Nz, j = idx - f * Nz;
    if (j != 0 && j != N) LN(z, first + f, Nz)[j] = 2.0 * LN(z, first + f, Nz)[j];
  }
  __syncthreads();
}

// adjoint of zrhs (right-hand sides, AB2, assembly, forward DCT and combinations):
// inputs Rb (rhs adjoints), L (new-state adjoint), mu (adjoint of h_n), state s_n;
// outputs lam (adjoint of s_n, partial: update + rhs + phi in G), mu_prev (adjoint of h_{n-1}),
// nlb (9 non-linear sample adjoints, fp64)
__global__ void __launch_bounds__(ZT) adj_zrhs_kernel(GridDev g, const double2* __restrict__ Rb,
                                                      const double2* __restrict__ L,
                                                      const double2* __restrict__ mu,
                                                      double2* __restrict__ lam,
                                                      double2* __restrict__ mu_prev,
                                                      double2* __restrict__ nlb, long long fs,
                                                      int first, double nls,
                                                      const double2* __restrict__ bb, FftPlan pz) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const int tid = threadIdx.x;
  const double2 zero = make_double2(0.0, 0.0);
  if (j == g.ny / 2) {
    for (int n = tid; n < Nz; n += blockDim.x) {
      for (int f = 0; f < 3; ++f) {
        lam[f * fs + off + n] = zero;
        mu_prev[f * fs + off + n] = zero;
      }
      for (int f = 0; f < 9; ++f) nlb[f * fs + off + n] = zero;
    }
    return;
  }
  const ZSmem z = carve(zsm, Nz, N);
  const bool is00 = (mx == 0 && j == 0);
  const double k2 = ksq(kx, ky);
  const double a = first ? 1.0 : 1.5, b = first ? 0.0 : -0.5;
  const double twoRe = 2.0 * g.re, cphi = g.pe / (g.ch * g.ch), rdt = 1.0 / g.dt, rpe = 1.0 / g.pe;
  // lines: 10 hbar_om, 11 hbar_w, 12 hbar_phi, 13 -2 beta Rb_theta (for (D^2 - k^2)^T)
  for (int n = tid; n < Nz; n += blockDim.x) {
    const double2 ro = Rb[off + n], rt = Rb[fs + off + n], rp = Rb[2 * fs + off + n];
    const double2 Ho = (-twoRe) * ro, Hw = (-twoRe) * rt, Hp = cphi * rp;
    LN(z, 10, Nz)[n] = a * Ho + mu[off + n];
    LN(z, 11, Nz)[n] = a * Hw + mu[fs + off + n];
    LN(z, 12, Nz)[n] = a * Hp + mu[2 * fs + off + n];
    mu_prev[off + n] = b * Ho;
    mu_prev[fs + off + n] = b * Hw;
    mu_prev[2 * fs + off + n] = b * Hp;
    LN(z, 13, Nz)[n] = (-2.0 * g.beta) * rt;
    // state adjoint from the update, the right-hand sides (D^2 part of w added below) and the
    // wall values (bb, parity of n)
    const double2* bl = bb + ((size_t)line * 2 + (n & 1)) * 3;
    const double n2 = (double)n * (double)n;
    lam[off + n] = (-1.0) * L[off + n] + (-2.0 * g.beta) * ro + bl[0];
    lam[fs + off + n] = (-1.0) * L[fs + off + n] + (-k2) * LN(z, 13, Nz)[n] + bl[1] + n2 * bl[2];
    lam[2 * fs + off + n] = (cphi * rdt) * rp;
  }
  __syncthreads();
  // first derivatives transposed: D^T hbar_om -> 7 (Q), D^T hbar_w -> 8 (R), D^T hbar_phi -> 9
  // (w phi), D^T line13 -> 14, and on (0,0) D^T of the real parts of hbar_om
  if (is00) {
    for (int n = tid; n < Nz; n += blockDim.x) {
      const double2 h = LN(z, 10, Nz)[n];
      LN(z, 0, Nz)[n] = make_double2(h.x, 0.0);
      LN(z, 1, Nz)[n] = make_double2(h.y, 0.0);
    }
    __syncthreads();
  }
  {
    double2* src[6] = {LN(z, 10, Nz), LN(z, 11, Nz), LN(z, 12, Nz), LN(z, 13, Nz), LN(z, 0, Nz),
                       LN(z, 1, Nz)};
    double2* dst[6] = {LN(z, 7, Nz), LN(z, 8, Nz), LN(z, 9, Nz), LN(z, 14, Nz), LN(z, 2, Nz),
                       LN(z, 3, Nz)};
    dzT_tasks(src, dst, is00 ? 6 : 4, N);
  }
  __syncthreads();
  // second derivatives transposed: D^T(D^T hbar_w) -> 4, D^T(D^T hbar_phi) -> 5, D^T line14 -> 6
  {
    double2* src[3] = {LN(z, 8, Nz), LN(z, 9, Nz), LN(z, 14, Nz)};
    double2* dst[3] = {LN(z, 4, Nz), LN(z, 5, Nz), LN(z, 6, Nz)};
    dzT_tasks(src, dst, 3, N);
  }
  __syncthreads();
  // coefficient adjoints of the seven transformed lines c0..c6 into lines 0..6
  for (int n = tid; n < Nz; n += blockDim.x) {
    const double2 ho = LN(z, 10, Nz)[n], hw = LN(z, 11, Nz)[n], hp = LN(z, 12, Nz)[n];
    const double2 Gb = (-k2 * rpe) * hp + rpe * LN(z, 5, Nz)[n];      // G adjoint
    lam[fs + off + n] = lam[fs + off + n] + LN(z, 6, Nz)[n];           // (D^2)^T part of theta
    lam[2 * fs + off + n] = lam[2 * fs + off + n] - (1.0 + g.shat) * Gb;
    double2 c0, c1, c2, c3;
    if (is00) {
      c0 = LN(z, 2, Nz)[n];             // D^T of Re(hbar_om.x): Sxz
      c1 = LN(z, 3, Nz)[n];             // Syz
      c2 = zero;
      c3 = zero;
    } else {
      c0 = ho;                                          // P
      c1 = LN(z, 7, Nz)[n];                             // Q: D^T hbar_om
      c2 = (-k2) * hw - LN(z, 4, Nz)[n];                // C: -k^2 hbar_w - (D^2)^T hbar_w
      c3 = (-1.0) * LN(z, 8, Nz)[n];                    // R: -D^T hbar_w
    }
    const double2 c4 = hp;                              // F
    const double2 c5 = (-1.0) * LN(z, 9, Nz)[n];        // w phi: -D^T hbar_phi
    LN(z, 0, Nz)[n] = c0;
    LN(z, 1, Nz)[n] = c1;
    LN(z, 2, Nz)[n] = c2;
    LN(z, 3, Nz)[n] = c3;
    LN(z, 4, Nz)[n] = c4;
    LN(z, 5, Nz)[n] = c5;
    LN(z, 6, Nz)[n] = Gb;                               // phi^3 line
  }
  __syncthreads();
  for (int f0 = 0; f0 < 7; f0 += NBF)
    dct_forward_transpose_lines(z, f0, (7 - f0 < NBF) ? 7 - f0 : NBF, Nz, N, pz, g.zcs);
  // combinations transposed: samples of the nine non-linear fields
  for (int n = tid; n < Nz; n += blockDim.x) {
    const double2 c0 = LN(z, 0, Nz)[n], c1 = LN(z, 1, Nz)[n], c2 = LN(z, 2, Nz)[n];
    const double2 c3 = LN(z, 3, Nz)[n], c4 = LN(z, 4, Nz)[n], c5 = LN(z, 5, Nz)[n];
    const double2 c6 = LN(z, 6, Nz)[n];
    double2 s[9];
    for (int q = 0; q < 9; ++q) s[q] = zero;
    if (is00) {
      s[3] = c0;
      s[4] = c1;
    } else {
      // P = i kx B - i ky A, R = i kx A + i ky B  ->  A, B adjoints
      const double2 Ab = mul_i(ky * c0) + (-1.0) * mul_i(kx * c3);
      const double2 Bb = (-1.0) * mul_i(kx * c0) + (-1.0) * mul_i(ky * c3);
      s[0] = (-1.0) * mul_i(kx * Ab);                         // A = i kx s0 + i ky s2
      s[2] = (-1.0) * mul_i(ky * Ab) + (-1.0) * mul_i(kx * Bb);
      s[1] = (-1.0) * mul_i(ky * Bb);                         // B = i kx s2 + i ky s1
      s[4] = (-1.0) * mul_i(kx * c1) + (-1.0) * mul_i(ky * c2);   // Q = i kx s4 - i ky s3
      s[3] = mul_i(ky * c1) + (-1.0) * mul_i(kx * c2);            // C = i kx s3 + i ky s4
      s[6] = mul_i(kx * c4);                                      // F = -(i kx s6 + i ky s7)
      s[7] = mul_i(ky * c4);
    }
    s[8] = c5;
    s[5] = c6;
    // nls: the forward y pass's 1/(Px Py), moved here from the transposed (backward) y pass
    for (int q = 0; q < 9; ++q) nlb[q * fs + off + n] = nls * s[q];
  }
}

// adjoint of the backward fields of s_n (u, v, w, phi, D phi -> backward DCT): in = 5 sample
// adjoint fields; adds the state adjoint into lam
__global__ void __launch_bounds__(ZT) adj_zbwd_kernel(GridDev g, const double2* __restrict__ in5,
                                                      long long fs_in, double2* __restrict__ lam,
                                                      long long fs, FftPlan pz) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  if (j == g.ny / 2) return;
  const ZSmem z = carve(zsm, Nz, N);
  const bool is00 = (mx == 0 && j == 0);
  for (int idx = threadIdx.x; idx < 5 * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    LN(z, f, Nz)[n] = in5[(long long)f * fs_in + off + n];
  }
  __syncthreads();
  // the backward DCT matrix C[j][n] = cos(pi n j / N) is symmetric: its transpose is itself
  dct1_lines(z, 0, 4, Nz, N, pz, g.zcs, 1);
  dct1_lines(z, 4, 1, Nz, N, pz, g.zcs, 1);
  const double k2 = ksq(kx, ky);
  const double rk2 = is00 ? 0.0 : 1.0 / k2;
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 ub = LN(z, 0, Nz)[n], vb = LN(z, 1, Nz)[n];
    double2 omb, dwb;
    if (is00) {
      omb = make_double2(ub.x, vb.x);
      dwb = make_double2(0.0, 0.0);
    } else {
      // u = (i kx Dw + i ky om)/k^2, v = (i ky Dw - i kx om)/k^2
      omb = rk2 * ((-1.0) * mul_i(ky * ub) + mul_i(kx * vb));
      dwb = rk2 * ((-1.0) * mul_i(kx * ub) + (-1.0) * mul_i(ky * vb));
    }
    LN(z, 10, Nz)[n] = omb;
    LN(z, 11, Nz)[n] = dwb;
  }
  __syncthreads();
  {
    double2* src[2] = {LN(z, 11, Nz), LN(z, 4, Nz)};
    double2* dst[2] = {LN(z, 12, Nz), LN(z, 13, Nz)};
    dzT_tasks(src, dst, 2, N);
  }
  __syncthreads();
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    lam[off + n] = lam[off + n] + LN(z, 10, Nz)[n];
    lam[fs + off + n] = lam[fs + off + n] + LN(z, 2, Nz)[n] + LN(z, 12, Nz)[n];
    lam[2 * fs + off + n] = lam[2 * fs + off + n] + LN(z, 3, Nz)[n] + LN(z, 13, Nz)[n];
  }
}

// G a with G[n][m] = (q_{n+m} + q_{|n-m|}) / 2, q_k = 2/(1-k^2) (k even), 0 (k odd)
__device__ __forceinline__ double gram_q(int k) { return (k & 1) ? 0.0 : 2.0 / (1.0 - (double)k * k); }

// objective J = 1/2 int |u|^2 + int |grad phi|^2 (exact) per line: partial sums and gradient
__global__ void __launch_bounds__(ZT) objective_kernel(GridDev g, const double2* __restrict__ st_om,
                                                       const double2* __restrict__ st_w,
                                                       const double2* __restrict__ st_phi,
                                                       double2* __restrict__ lam, long long fs,
                                                       double* __restrict__ part) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const ZSmem z = carve(zsm, Nz, N);
  __shared__ double red[ZT];
  const bool nyq = (j == g.ny / 2);
  const bool is00 = (mx == 0 && j == 0);
  const double k2 = ksq(kx, ky);
  const double rk2 = is00 ? 0.0 : 1.0 / k2;
  const double wts = (mx == 0 ? 1.0 : 2.0) * g.lx * g.ly;
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    LN(z, 10, Nz)[n] = nyq ? make_double2(0.0, 0.0) : st_om[off + n];
    LN(z, 11, Nz)[n] = nyq ? make_double2(0.0, 0.0) : st_w[off + n];
    LN(z, 12, Nz)[n] = nyq ? make_double2(0.0, 0.0) : st_phi[off + n];
  }
  __syncthreads();
  {
    double2* src[2] = {LN(z, 11, Nz), LN(z, 12, Nz)};
    double2* dst[2] = {LN(z, 13, Nz), LN(z, 14, Nz)};
    dz_tasks(src, dst, 2, N);
  }
  __syncthreads();
  // lines 0 u, 1 v, 2 w, 3 D phi (coefficients)
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 om = LN(z, 10, Nz)[n], dw = LN(z, 13, Nz)[n];
    double2 u, v;
    if (is00) {
      u = make_double2(om.x, 0.0);
      v = make_double2(om.y, 0.0);
    } else {
      u = rk2 * mul_i(kx * dw + ky * om);
      v = rk2 * mul_i(ky * dw - kx * om);
    }
    LN(z, 0, Nz)[n] = u;
    LN(z, 1, Nz)[n] = v;
    LN(z, 2, Nz)[n] = LN(z, 11, Nz)[n];
    LN(z, 3, Nz)[n] = LN(z, 14, Nz)[n];
  }
  __syncthreads();
  // G times lines 0..3 and phi (line 12) into lines 4..8; partial J.  q_k (k = 0..2N) is
  // tabulated in line 15 (2 Nz >= 2N + 1 doubles)
  double jp = 0.0;
  double* qt = reinterpret_cast<double*>(LN(z, 15, Nz));
  for (int k = threadIdx.x; k <= 2 * N; k += blockDim.x) qt[k] = gram_q(k);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 5 * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    const double2* a = (f < 4) ? LN(z, f, Nz) : LN(z, 12, Nz);
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m <= N; ++m) {
      const double gnm = 0.5 * (qt[n + m] + qt[n > m ? n - m : m - n]);
      acc.x = fma(gnm, a[m].x, acc.x);
      acc.y = fma(gnm, a[m].y, acc.y);
    }
    LN(z, 4 + f, Nz)[n] = acc;
    const double2 an = a[n];
    const double wq = (f < 3) ? 0.5 : (f == 3 ? 1.0 : k2);  // u v w: 1/2; D phi: 1; phi: k^2
    jp += wq * (an.x * acc.x + an.y * acc.y);
  }
  red[threadIdx.x] = jp;
  __syncthreads();
  for (int s2 = ZT / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[line] = wts * red[0];
  // gradient: d/da Re(a^H G a) = 2 G a
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 ub = wts * LN(z, 4, Nz)[n], vb = wts * LN(z, 5, Nz)[n];
    double2 omb, dwb;
    if (is00) {
      omb = make_double2(ub.x, vb.x);
      dwb = make_double2(0.0, 0.0);
    } else {
      omb = rk2 * ((-1.0) * mul_i(ky * ub) + mul_i(kx * vb));
      dwb = rk2 * ((-1.0) * mul_i(kx * ub) + (-1.0) * mul_i(ky * vb));
    }
    LN(z, 0, Nz)[n] = omb;
    LN(z, 1, Nz)[n] = dwb;
    LN(z, 2, Nz)[n] = (2.0 * wts) * LN(z, 7, Nz)[n];   // D phi adjoint
  }
  __syncthreads();
  {
    double2* src[2] = {LN(z, 1, Nz), LN(z, 2, Nz)};
    double2* dst[2] = {LN(z, 9, Nz), LN(z, 13, Nz)};
    dzT_tasks(src, dst, 2, N);
  }
  __syncthreads();
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    if (nyq) {
      lam[off + n] = make_double2(0.0, 0.0);
      lam[fs + off + n] = make_double2(0.0, 0.0);
      lam[2 * fs + off + n] = make_double2(0.0, 0.0);
      continue;
    }
    lam[off + n] = LN(z, 0, Nz)[n];
    lam[fs + off + n] = is00 ? make_double2(0.0, 0.0)
                             : wts * LN(z, 6, Nz)[n] + LN(z, 9, Nz)[n];
    lam[2 * fs + off + n] = (2.0 * wts * k2) * LN(z, 8, Nz)[n] + LN(z, 13, Nz)[n];
  }
}

// adjoint of set_fields' projection and forward DCT: lam (3 state fields) -> four (Mx, Ny, Nz)
// sample-adjoint fields of u, v, w, phi, scaled for the transposed x/y transforms that follow:
// 1/(nx ny) (the forward normalisation) and 1/2 for kx >= 1 (a c2r then transposes the r2c)
__global__ void __launch_bounds__(ZT) adj_project_kernel(GridDev g, const double2* __restrict__ lam,
                                                         long long fs, double2* __restrict__ out4,
                                                         FftPlan pz) {
  extern __shared__ double2 zsm[];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const ZSmem z = carve(zsm, Nz, N);
  const bool nyq = (j == g.ny / 2);
  const bool is00 = (mx == 0 && j == 0);
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 ob = nyq ? make_double2(0.0, 0.0) : lam[off + n];
    const double2 wb = (nyq || is00) ? make_double2(0.0, 0.0) : lam[fs + off + n];
    const double2 pb = nyq ? make_double2(0.0, 0.0) : lam[2 * fs + off + n];
    double2 ub, vb;
    if (is00) {
      ub = make_double2(ob.x, 0.0);
      vb = make_double2(ob.y, 0.0);
    } else {
      ub = mul_i(ky * ob);              // om = i kx v - i ky u
      vb = (-1.0) * mul_i(kx * ob);
    }
    if (nyq) {
      ub = make_double2(0.0, 0.0);
      vb = make_double2(0.0, 0.0);
    }
    LN(z, 0, Nz)[n] = ub;
    LN(z, 1, Nz)[n] = vb;
    LN(z, 2, Nz)[n] = wb;
    LN(z, 3, Nz)[n] = pb;
  }
  __syncthreads();
  dct_forward_transpose_lines(z, 0, 4, Nz, N, pz, g.zcs);
  const double sc = (mx >= 1 ? 0.5 : 1.0) / ((double)g.nx * (double)g.ny);
  for (int idx = threadIdx.x; idx < 4 * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    out4[(long long)f * fs + off + n] = sc * LN(z, f, Nz)[n];
  }
}

// transpose of the backward y pass's field map: field 3 (phi) += -i ky field 4 (i ky phi), then
// field 4 <- field 5 (D phi), leaving u v w phi D phi adjoints in fields 0..4
__global__ void fold_dy_kernel(GridDev g, double2* __restrict__ f6, long long fs) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)g.Mx * g.ny * g.nz;
  if (i >= total) return;
  const int j = (int)((i / g.nz) % g.ny);
  const int my = (j < g.ny / 2) ? j : j - g.ny;
  const double ky = 6.283185307179586476925 * my / g.ly;
  const double2 d = f6[4 * fs + i];
  f6[3 * fs + i] = f6[3 * fs + i] + (-1.0) * mul_i(ky * d);
  f6[4 * fs + i] = f6[5 * fs + i];
}

// sum of n doubles in a fixed order (one CTA of 256 threads)
__global__ void __launch_bounds__(256) sum_kernel(const double* __restrict__ a, int n,
                                                  double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += a[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = 128; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// ---- grouped persistent launches (ensemble) ---------------------------------------------
__device__ __forceinline__ int member_of(const int* __restrict__ begin, int nmem, int item) {
  int m = 0;
  while (m + 1 < nmem && begin[m + 1] <= item) ++m;
  return m;
}

template <typename T>
__global__ void __launch_bounds__(ZT) grouped_zrhs_kernel(const Member* __restrict__ mem,
                                                          const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zrhs_body<T>(M.g, (const T2*)M.nl, M.fs, M.om, M.w, M.phi, M.hom, M.hw, M.hphi, M.R, M.first,
                 M.pz, item - begin[m]);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(ZT) grouped_zbwd_kernel(const Member* __restrict__ mem,
                                                          const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zbwd_body<T, 1, 5>(M.g, M.R, M.om, M.w, M.phi, (T2*)M.bw, M.fs, M.pz, item - begin[m]);
    __syncthreads();
  }
}

// tensor-core Chebyshev method: the products' coefficients are in M.cf (float64 whatever the
// working precision), and zbwd leaves the 5 backward fields' coefficients there
__global__ void __launch_bounds__(ZTC) grouped_zrhs_coef_kernel(const Member* __restrict__ mem,
                                                               const int* __restrict__ begin,
                                                               int nmem) {
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zrhs_body<double, 1, 0>(M.g, M.cf, M.fs, M.om, M.w, M.phi, M.hom, M.hw, M.hphi, M.R, M.first,
                         M.pz, item - begin[m]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(ZTC) grouped_zbwd_coef_kernel(const Member* __restrict__ mem,
                                                               const int* __restrict__ begin,
                                                               int nmem) {
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zbwd_body<double, 1, 5, 1>(M.g, M.R, M.om, M.w, M.phi, M.cf, M.fs, M.pz, item - begin[m]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TLT) grouped_zsolve_tile_kernel(const Member* __restrict__ mem,
                                                                     const int* __restrict__ begin,
                                                                     int nmem) {
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zsolve_tile_body(M.g, M.R, M.fs, M.g.Mx * M.g.ny, item - begin[m]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(ST) grouped_zsolve_kernel(const Member* __restrict__ mem,
                                                            const int* __restrict__ begin, int nmem) {
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of(begin, nmem, item);
    const Member& M = mem[m];
    zsolve_body(M.g, M.R, M.fs, M.g.Mx * M.g.ny, (item - begin[m]) * ST + threadIdx.x);
  }
}

}  // namespace

size_t zline_smem(const GridDev& g) {
  return (size_t)(NLINES * g.nz + 2 * NBF * g.N) * sizeof(double2);
}
// the coefficient-space kernels use the lines only (no DCT scratch): zrhs lines 0..12 (four
// CTAs per SM at nz = 257), zbwd five
static size_t zline_coef_smem(const GridDev& g) { return (size_t)13 * g.nz * sizeof(double2); }
static size_t zbwd_coef_smem(const GridDev& g) { return (size_t)5 * g.nz * sizeof(double2); }
size_t zline_coef_stage_smem(const GridDev& g, int stage) {
  // the grouped coefficient-space zrhs keeps omega and phi in shared memory (sixteen lines)
  return stage == 0 ? (size_t)NLINES * g.nz * sizeof(double2) : zbwd_coef_smem(g);
}

size_t fac_doubles(const GridDev& g) { return ((size_t)13 * g.nz + 20) * g.NK; }

cudaError_t build_factor_table(const GridDev& g, double* fac, cudaStream_t s) {
  const int n3 = g.NK;
  const int n1 = g.NK * 8, n2 = g.NK * 2;
  factor_kernel<<<(n1 + 127) / 128, 128, 0, s>>>(g, fac);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  homog_kernel<<<(n2 + 127) / 128, 128, 0, s>>>(g, fac);
  e = cudaGetLastError();
  if (e != cudaSuccess || g.bc < 2) return e;
  mixed_kernel<<<(n3 + 127) / 128, 128, 0, s>>>(g, fac);
  return cudaGetLastError();
}

cudaError_t launch_zrhs(int prec, const GridDev& g, const void* nl, long long fs,
                        const double2* st_om, const double2* st_w, const double2* st_phi,
                        double2* h_om, double2* h_w, double2* h_phi, double2* R, int first,
                        const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  cudaError_t e;
  if (prec == 0) {
    static SmemLimit cur;
    if ((e = ensure_smem(zrhs_kernel<double>, smem, &cur)) != cudaSuccess) return e;
    zrhs_kernel<double><<<g.Mx * g.ny, ZT, smem, s>>>(g, (const double2*)nl, fs, st_om, st_w, st_phi,
                                                      h_om, h_w, h_phi, R, first, pz);
  } else if (prec == 1) {
    static SmemLimit cur;
    if ((e = ensure_smem(zrhs_kernel<float>, smem, &cur)) != cudaSuccess) return e;
    zrhs_kernel<float><<<g.Mx * g.ny, ZT, smem, s>>>(g, (const float2*)nl, fs, st_om, st_w, st_phi,
                                                     h_om, h_w, h_phi, R, first, pz);
  } else {
    static SmemLimit cur;
    if ((e = ensure_smem(zrhs_kernel<df>, smem, &cur)) != cudaSuccess) return e;
    zrhs_kernel<df><<<g.Mx * g.ny, ZT, smem, s>>>(g, (const df2*)nl, fs, st_om, st_w, st_phi,
                                                  h_om, h_w, h_phi, R, first, pz);
  }
  return cudaGetLastError();
}

static SmemLimit cur_zrhs_coef, cur_zbwd_coef;

cudaError_t zline_coef_prepare(const GridDev& g) {
  const size_t smem = zline_coef_smem(g);
  cudaError_t e = ensure_smem(zrhs_kernel<double, 1>, smem, &cur_zrhs_coef);
  if (e == cudaSuccess)
    e = ensure_smem(zbwd_kernel<double, 1, 5, 1>, zbwd_coef_smem(g), &cur_zbwd_coef);
  return e;
}

cudaError_t launch_zrhs_coef(const GridDev& g, const double2* cf, long long fs,
                             const double2* st_om, const double2* st_w, const double2* st_phi,
                             double2* h_om, double2* h_w, double2* h_phi, double2* R, int first,
                             const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_coef_smem(g);
  cudaError_t e = ensure_smem(zrhs_kernel<double, 1>, smem, &cur_zrhs_coef);
  if (e != cudaSuccess) return e;
  zrhs_kernel<double, 1><<<g.Mx * g.ny, ZTC, smem, s>>>(g, cf, fs, st_om, st_w, st_phi, h_om, h_w,
                                                       h_phi, R, first, pz);
  return cudaGetLastError();
}

cudaError_t launch_zbwd_coef(const GridDev& g, const double2* R, double2* st_om, double2* st_w,
                             double2* st_phi, double2* cf, long long fs, const FftPlan& pz,
                             cudaStream_t s) {
  const size_t smem = zbwd_coef_smem(g);
  cudaError_t e = ensure_smem(zbwd_kernel<double, 1, 5, 1>, smem, &cur_zbwd_coef);
  if (e != cudaSuccess) return e;
  zbwd_kernel<double, 1, 5, 1><<<g.Mx * g.ny, ZTC, smem, s>>>(g, R, st_om, st_w, st_phi, cf, fs,
                                                             pz);
  return cudaGetLastError();
}

size_t zsolve_tile_smem(const GridDev& g) {
  return (size_t)TL * g.nz * sizeof(double2) + (size_t)3 * g.nz * sizeof(double);
}
int zsolve_tile_lines() { return TL; }
int zsolve_threads() { return ST; }

cudaError_t launch_grouped_z(int stage, int prec, const Member* mem, const int* begin, int nmem,
                             int grid, size_t smem, int zsolve_tile, int coef, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (coef && stage != 1) {
    if (stage == 0) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zrhs_coef_kernel, smem, &cur)) != cudaSuccess) return e;
      grouped_zrhs_coef_kernel<<<grid, ZTC, smem, s>>>(mem, begin, nmem);
    } else {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zbwd_coef_kernel, smem, &cur)) != cudaSuccess) return e;
      grouped_zbwd_coef_kernel<<<grid, ZTC, smem, s>>>(mem, begin, nmem);
    }
  } else if (stage == 0) {
    if (prec == 0) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zrhs_kernel<double>, smem, &cur)) != cudaSuccess) return e;
      grouped_zrhs_kernel<double><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    } else if (prec == 1) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zrhs_kernel<float>, smem, &cur)) != cudaSuccess) return e;
      grouped_zrhs_kernel<float><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    } else {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zrhs_kernel<df>, smem, &cur)) != cudaSuccess) return e;
      grouped_zrhs_kernel<df><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    }
  } else if (stage == 1) {
    if (zsolve_tile) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zsolve_tile_kernel, smem, &cur)) != cudaSuccess) return e;
      grouped_zsolve_tile_kernel<<<grid, TLT, smem, s>>>(mem, begin, nmem);
    } else {
      grouped_zsolve_kernel<<<grid, ST, 0, s>>>(mem, begin, nmem);
    }
  } else {
    if (prec == 0) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zbwd_kernel<double>, smem, &cur)) != cudaSuccess) return e;
      grouped_zbwd_kernel<double><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    } else if (prec == 1) {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zbwd_kernel<float>, smem, &cur)) != cudaSuccess) return e;
      grouped_zbwd_kernel<float><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    } else {
      static SmemLimit cur;
      if ((e = ensure_smem(grouped_zbwd_kernel<df>, smem, &cur)) != cudaSuccess) return e;
      grouped_zbwd_kernel<df><<<grid, ZT, smem, s>>>(mem, begin, nmem);
    }
  }
  return cudaGetLastError();
}

// grouped zrhs (stage 0) or zbwd (stage 2) kernel of a working precision
static const void* zkernel(int stage, int prec) {
  if (stage == 0)
    return prec == 0 ? (const void*)grouped_zrhs_kernel<double>
         : prec == 1 ? (const void*)grouped_zrhs_kernel<float>
                     : (const void*)grouped_zrhs_kernel<df>;
  return prec == 0 ? (const void*)grouped_zbwd_kernel<double>
       : prec == 1 ? (const void*)grouped_zbwd_kernel<float>
                   : (const void*)grouped_zbwd_kernel<df>;
}

int occupancy_z(int stage, int prec, size_t smem, int zsolve_tile, int coef) {
  int n = 0;
  // the opt-in above 48 KB must be in place before the query (init time, never during capture)
  if (smem > 48 * 1024) {
    const void* k = stage == 1 ? (const void*)grouped_zsolve_tile_kernel : zkernel(stage, prec);
    if (coef && stage != 1)
      k = stage == 0 ? (const void*)grouped_zrhs_coef_kernel : (const void*)grouped_zbwd_coef_kernel;
    if (stage != 1 || zsolve_tile)
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaGetLastError();
  }
  if (coef && stage != 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, stage == 0 ? (const void*)grouped_zrhs_coef_kernel : (const void*)grouped_zbwd_coef_kernel,
        ZTC, smem);
  else if (stage == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zkernel(0, prec), ZT, smem);
  else if (stage == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zsolve_tile ? (const void*)grouped_zsolve_tile_kernel
                                                                  : (const void*)grouped_zsolve_kernel,
                                                  zsolve_tile ? TLT : ST, zsolve_tile ? smem : 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zkernel(2, prec), ZT, smem);
  cudaGetLastError();
  return n;
}

cudaError_t launch_adj_zsolve(const GridDev& g, const double2* L, double2* Rb, long long fs,
                              double2* bb, cudaStream_t s) {
  const int nlines = g.Mx * g.ny;
  adj_zsolve_kernel<<<(2 * nlines + ST - 1) / ST, ST, 0, s>>>(g, L, Rb, fs, nlines, bb);
  return cudaGetLastError();
}

cudaError_t launch_adj_zrhs(const GridDev& g, const double2* Rb, const double2* L,
                            const double2* mu, double2* lam, double2* mu_prev, double2* nlb,
                            long long fs, int first, const double2* bb, const FftPlan& pz,
                            cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(adj_zrhs_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  adj_zrhs_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, Rb, L, mu, lam, mu_prev, nlb, fs, first,
                                                 1.0 / ((double)g.Px * (double)g.Py), bb, pz);
  return cudaGetLastError();
}

cudaError_t launch_adj_zbwd(const GridDev& g, const double2* in5, long long fs_in, double2* lam,
                            long long fs, const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(adj_zbwd_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  adj_zbwd_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, in5, fs_in, lam, fs, pz);
  return cudaGetLastError();
}

cudaError_t launch_objective(const GridDev& g, const double2* om, const double2* w,
                             const double2* phi, double2* lam, long long fs, double* part,
                             cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(objective_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  objective_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, om, w, phi, lam, fs, part);
  return cudaGetLastError();
}

cudaError_t launch_adj_project(const GridDev& g, const double2* lam, long long fs, double2* out4,
                               const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(adj_project_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  adj_project_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, lam, fs, out4, pz);
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* a, int n, double* out, cudaStream_t s) {
  sum_kernel<<<1, 256, 0, s>>>(a, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fold_dy(const GridDev& g, double2* f6, long long fs, cudaStream_t s) {
  const long long total = (long long)g.Mx * g.ny * g.nz;
  fold_dy_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, f6, fs);
  return cudaGetLastError();
}

cudaError_t launch_zsolve(const GridDev& g, double2* R, long long fs, cudaStream_t s) {
  const int nlines = g.Mx * g.ny;
  const size_t tile = (size_t)TL * g.nz * sizeof(double2) + (size_t)3 * g.nz * sizeof(double);
  if (tile <= 72 * 1024) {
    // short lines: a 32-line tile fits three CTAs per SM; staging in shared memory wins
    static SmemLimit cur;
    cudaError_t e = ensure_smem(zsolve_tile_kernel, tile, &cur);
    if (e != cudaSuccess) return e;
    zsolve_tile_kernel<<<(nlines + TL - 1) / TL, TLT, tile, s>>>(g, R, fs, nlines);
  } else {
    // long lines: sweep in global memory (L1/L2), occupancy set by registers
    const int nthreads = 2 * nlines;
    zsolve_kernel<<<(nthreads + ST - 1) / ST, ST, 0, s>>>(g, R, fs, nlines);
  }
  return cudaGetLastError();
}

template <typename T, int UPDATE, int NOUT>
static cudaError_t launch_zbwd_t(const GridDev& g, const double2* R, double2* st_om,
                                 double2* st_w, double2* st_phi, void* bw, long long fs,
                                 const FftPlan& pz, cudaStream_t s) {
  typedef typename C2<T>::t T2;
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(zbwd_kernel<T, UPDATE, NOUT>, smem, &cur);
  if (e != cudaSuccess) return e;
  zbwd_kernel<T, UPDATE, NOUT><<<g.Mx * g.ny, ZT, smem, s>>>(g, R, st_om, st_w, st_phi, (T2*)bw,
                                                             fs, pz);
  return cudaGetLastError();
}

cudaError_t launch_zbwd(int update, int prec, int nout, const GridDev& g, const double2* R,
                        double2* st_om, double2* st_w, double2* st_phi, void* bw, long long fs,
                        const FftPlan& pz, cudaStream_t s) {
  if (nout == 7)  // auxiliary paths: fp64, from the state
    return launch_zbwd_t<double, 0, 7>(g, R, st_om, st_w, st_phi, bw, fs, pz, s);
  if (prec == 0)
    return update ? launch_zbwd_t<double, 1, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s)
                  : launch_zbwd_t<double, 0, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s);
  if (prec == 2)
    return update ? launch_zbwd_t<df, 1, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s)
                  : launch_zbwd_t<df, 0, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s);
  return update ? launch_zbwd_t<float, 1, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s)
                : launch_zbwd_t<float, 0, 5>(g, R, st_om, st_w, st_phi, bw, fs, pz, s);
}

cudaError_t launch_project(const GridDev& g, const double2* uvwp, long long fs, double2* st_om,
                           double2* st_w, double2* st_phi, double2* h_om, double2* h_w,
                           double2* h_phi, const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(project_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  project_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, uvwp, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, pz);
  return cudaGetLastError();
}

cudaError_t launch_dct_lines(int dir, int prec, const GridDev& g, const void* in, double2* out,
                             int nf, long long fs, const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static SmemLimit cur64, cur32, curdf;
  cudaError_t e = ensure_smem(dct_lines_kernel<double>, smem, &cur64);
  if (e == cudaSuccess) e = ensure_smem(dct_lines_kernel<float>, smem, &cur32);
  if (e == cudaSuccess) e = ensure_smem(dct_lines_kernel<df>, smem, &curdf);
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    dct_lines_kernel<double><<<g.Mx * g.ny, ZT, smem, s>>>(g, dir, (const double2*)in, out, nf, fs, pz);
  } else if (prec == 1) {
    dct_lines_kernel<float><<<g.Mx * g.ny, ZT, smem, s>>>(g, dir, (const float2*)in, out, nf, fs, pz);
  } else {
    dct_lines_kernel<df><<<g.Mx * g.ny, ZT, smem, s>>>(g, dir, (const df2*)in, out, nf, fs, pz);
  }
  return cudaGetLastError();
}

cudaError_t launch_diag(const GridDev& g, const double* phys7, long long fs,
                        const double2* st_phi, const double* ccw, const double* dzl,
                        const double* qint, double* part, double* out, cudaStream_t s) {
  const int nblk = 304;
  diag_partial_kernel<<<nblk, DT, 0, s>>>(g, phys7, fs, ccw, dzl, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, s>>>(g, nblk, part, st_phi, qint, out);
  return cudaGetLastError();
}

}  // namespace chf
