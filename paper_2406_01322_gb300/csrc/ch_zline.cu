// Wall-normal (z-line) kernels: everything that happens along one (kx, ky) Chebyshev line.
//
// Per line (paper Sec. 2.2, steps ii)-v), and Sec. 3.2.1-3.2.2):
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
// Crank-Nicolson is applied in "sum form": for q in {omega_z, lap(w), ubar + i vbar},
//   (D^2 - k^2 - beta)(q^{n+1} + q^n) = -2 beta q^n - 2 Re AB2(h),   beta = 2 Re / dt,
// which is the CN equation (D^2-k^2-beta) q^{n+1} = -(D^2-k^2+beta) q^n - 2 Re AB2(h) with
// (D^2-k^2-beta) q^n added to both sides; q^{n+1} + q^n satisfies the same homogeneous
// wall conditions, so the same tau problem gives it and only D^2 (not D^4) of w^n is needed.
//
// All arithmetic in this file is float64.  One CTA of 128 threads owns one line.
#include "ch_internal.h"

namespace chf {

namespace {

constexpr int ZT = 128;   // threads per z-line CTA
constexpr int NBF = 2;    // DCT lines transformed per FFT call
constexpr int NLINES = 16;

// d/dz in Chebyshev coefficient space for one real component (comp 0 = re, 1 = im):
// c_n b_n = b_{n+2} + 2 (n+1) a_{n+1}, run downward from n = N.  src may alias dst.
__device__ void dz_component(const double2* src, double2* dst, int comp, int N) {
  const double* s = reinterpret_cast<const double*>(src) + comp;
  double* d = reinterpret_cast<double*>(dst) + comp;
  double bp1 = 0.0, bp2 = 0.0, ap1 = 0.0;
  for (int n = N; n >= 0; --n) {
    const double an = s[2 * n];
    const double bn = fma(2.0 * (n + 1), ap1, bp2);
    d[2 * n] = (n == 0) ? 0.5 * bn : bn;
    bp2 = bp1;
    bp1 = bn;
    ap1 = an;
  }
}

// run up to 8 derivative tasks (src -> dst) in parallel, one thread per (task, component)
__device__ void dz_tasks(double2* const* src, double2* const* dst, int ntask, int N) {
  const int t = threadIdx.x;
  if (t < 2 * ntask) dz_component(src[t >> 1], dst[t >> 1], t & 1, N);
}

// Gottlieb-Orszag factorisation of (D^2 - alpha) for one parity p (elimination from the top
// coefficient down; the boundary row closes the system at n = p).  Stores Y[n], RD[n] (=1/den)
// and Q[n] for n = p, p+2, ..., returns SQ = sum_i beta_i Q_i (beta = 1 Dirichlet, n^2 Neumann).
__device__ double tau_factor(double alpha, int p, int N, bool neumann, const double* t1,
                             const double* t2, const double* t3, double* Y, double* RD,
                             double* Q) {
  const int I = (N - p) / 2;
  double ynext = 0.0;
  for (int i = I; i >= 1; --i) {
    const int n = p + 2 * i;
    const double L = -alpha * t1[n];
    const double Dg = 1.0 + alpha * t2[n];
    const double U = -alpha * t3[n];
    const double rd = 1.0 / fma(U, ynext, Dg);
    const double y = -L * rd;
    Y[n] = y;
    RD[n] = rd;
    ynext = y;
  }
  double q = 1.0;
  Q[p] = 1.0;
  double sq = neumann ? (double)(p * p) : 1.0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    q *= Y[n];
    Q[n] = q;
    sq = fma(neumann ? (double)n * (double)n : 1.0, q, sq);
  }
  return sq;
}

// Solve (D^2 - alpha) a = f (tau rows in Gottlieb-Orszag form) for parity p of one component,
// in place: x[2n] holds f_n on entry and a_n on exit (n of parity p).  g0 = boundary value
// (sum of the parity-p coefficients, or of n^2 times them for Neumann).
__device__ void tau_sweep(double* x, int p, int N, double alpha, bool neumann, double g0,
                          const double* t1, const double* t2, const double* t3,
                          const double* Y, const double* RD, const double* Q, double sq) {
  const int I = (N - p) / 2;
  double xn = 0.0, fnp2 = 0.0;
  for (int i = I; i >= 1; --i) {
    const int n = p + 2 * i;
    const double fn = x[2 * n];
    const double fnm2 = x[2 * (n - 2)];
    const double gi = fma(t1[n], fnm2, fma(-t2[n], fn, t3[n] * fnp2));
    const double U = -alpha * t3[n];
    const double xi = fma(-U, xn, gi) * RD[n];
    x[2 * n] = xi;
    fnp2 = fn;
    xn = xi;
  }
  double P = 0.0, sp = 0.0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    P = fma(Y[n], P, x[2 * n]);
    x[2 * n] = P;
    sp = fma(neumann ? (double)n * (double)n : 1.0, P, sp);
  }
  const double a0 = (g0 - sp) / sq;
  x[2 * p] = a0;
  for (int i = 1; i <= I; ++i) {
    const int n = p + 2 * i;
    x[2 * n] = fma(Q[n], a0, x[2 * n]);
  }
}

struct ZSmem {
  double2* L;   // NLINES lines of Nz
  double2* FA;  // NBF * 2N
  double2* FB;
  double* Y;    // 3 * Nz
  double* RD;
  double* Q;
  double* t1;   // Nz each: Gottlieb-Orszag row tables
  double* t2;
  double* t3;
};

__device__ __forceinline__ ZSmem carve(double2* sm, int Nz, int N) {
  ZSmem z;
  z.L = sm;
  z.FA = sm + NLINES * Nz;
  z.FB = z.FA + NBF * 2 * N;
  double* d = reinterpret_cast<double*>(z.FB + NBF * 2 * N);
  z.Y = d;
  z.RD = d + 3 * Nz;
  z.Q = d + 6 * Nz;
  z.t1 = d + 9 * Nz;
  z.t2 = d + 10 * Nz;
  z.t3 = d + 11 * Nz;
  return z;
}

__device__ __forceinline__ double2* LN(const ZSmem& z, int i, int Nz) { return z.L + i * Nz; }

// forward DCT-I of cnt lines (in place): samples f_j -> a_n = G_n / (cbar_n N), where G is the
// 2N-point DFT of the even extension (Sec. 3.2.1).
__device__ void dct_forward_lines(const ZSmem& z, int first, int cnt, int Nz, int N,
                                  const FftPlan& pz) {
  const int NE = 2 * N;
  for (int idx = threadIdx.x; idx < cnt * NE; idx += blockDim.x) {
    const int f = idx / NE, m = idx - f * NE;
    const int jj = (m <= N) ? m : NE - m;
    z.FA[f * NE + m] = LN(z, first + f, Nz)[jj];
  }
  __syncthreads();
  const double2* R = block_fft<double, false>(z.FA, z.FB, cnt, NE, pz);
  const double sN = 1.0 / N;
  for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
    const int f = idx / Nz, n = idx - f * Nz;
    const double s = (n == 0 || n == N) ? 0.5 * sN : sN;
    LN(z, first + f, Nz)[n] = s * R[f * NE + n];
  }
  __syncthreads();
}

// backward DCT-I of cnt lines starting at line `first`: f_j = sum_n a_n cos(pi n j / N),
// evaluated as half the 2N-point DFT of the even extension of (2 a_0, a_1, .., a_{N-1}, 2 a_N).
// Results are written to out[(first+f) * fs + off + j].
template <typename T2>
__device__ void dct_backward_lines_store(const ZSmem& z, int first, int cnt, int Nz, int N,
                                         const FftPlan& pz, T2* out, long long fs, size_t off,
                                         int out_first) {
  const int NE = 2 * N;
  for (int idx = threadIdx.x; idx < cnt * NE; idx += blockDim.x) {
    const int f = idx / NE, m = idx - f * NE;
    const int jj = (m <= N) ? m : NE - m;
    double2 v = LN(z, first + f, Nz)[jj];
    if (jj == 0 || jj == N) v = 2.0 * v;
    z.FA[f * NE + m] = v;
  }
  __syncthreads();
  const double2* R = block_fft<double, false>(z.FA, z.FB, cnt, NE, pz);
  for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
    const int f = idx / Nz, j = idx - f * Nz;
    out[(long long)(out_first + f) * fs + off + j] = from_d2<T2>(0.5 * R[f * NE + j]);
  }
  __syncthreads();
}

__device__ __forceinline__ void line_wavenumbers(const GridDev& g, int line, int& mx, int& j,
                                                 double& kx, double& ky) {
  mx = line / g.ny;
  j = line - mx * g.ny;
  const int my = (j < g.ny / 2) ? j : j - g.ny;
  kx = 6.283185307179586476925 * mx / g.lx;
  ky = 6.283185307179586476925 * my / g.ly;
}

// the seven fields the non-linear terms need, from the state held in lines 10 (omega / mean),
// 11 (w), 12 (phi): u, v (continuity + omega_z definition), w, phi, i kx phi, i ky phi, D phi.
template <typename T2>
__device__ void backward_fields(const ZSmem& z, const GridDev& g, double kx, double ky,
                                bool is00, const FftPlan& pz, T2* bw, long long fs,
                                size_t off) {
  const int Nz = g.nz, N = g.N;
  {
    double2* src[2] = {LN(z, 11, Nz), LN(z, 12, Nz)};
    double2* dst[2] = {LN(z, 13, Nz), LN(z, 14, Nz)};
    dz_tasks(src, dst, 2, N);
  }
  __syncthreads();
  const double k2 = kx * kx + ky * ky;
  const double rk2 = is00 ? 0.0 : 1.0 / k2;
  for (int n = threadIdx.x; n < Nz; n += blockDim.x) {
    const double2 om = LN(z, 10, Nz)[n];
    const double2 dw = LN(z, 13, Nz)[n];
    const double2 ph = LN(z, 12, Nz)[n];
    double2 u, v;
    if (is00) {
      u = make_double2(om.x, 0.0);
      v = make_double2(om.y, 0.0);
    } else {
      // u = (i kx Dw + i ky om) / k^2,  v = (i ky Dw - i kx om) / k^2
      u = rk2 * mul_i(kx * dw + ky * om);
      v = rk2 * mul_i(ky * dw - kx * om);
    }
    LN(z, 0, Nz)[n] = u;
    LN(z, 1, Nz)[n] = v;
    LN(z, 2, Nz)[n] = LN(z, 11, Nz)[n];
    LN(z, 3, Nz)[n] = ph;
    LN(z, 4, Nz)[n] = kx * mul_i(ph);
    LN(z, 5, Nz)[n] = ky * mul_i(ph);
    LN(z, 6, Nz)[n] = LN(z, 14, Nz)[n];
  }
  __syncthreads();
  for (int f0 = 0; f0 < 7; f0 += NBF) {
    const int cnt = (7 - f0 < NBF) ? 7 - f0 : NBF;
    dct_backward_lines_store<T2>(z, f0, cnt, Nz, N, pz, bw, fs, off, f0);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(ZT) zline_kernel(GridDev g, const typename C2<T>::t* __restrict__ nl,
                                                   typename C2<T>::t* __restrict__ bw, long long fs,
                                                   double2* __restrict__ st_om,
                                                   double2* __restrict__ st_w,
                                                   double2* __restrict__ st_phi,
                                                   double2* __restrict__ h_om,
                                                   double2* __restrict__ h_w,
                                                   double2* __restrict__ h_phi, int first,
                                                   FftPlan pz) {
  typedef typename C2<T>::t T2;
  extern __shared__ double2 zsm[];
  __shared__ double sq[6];
  const int Nz = g.nz, N = g.N;
  const int line = blockIdx.x;
  int mx, j;
  double kx, ky;
  line_wavenumbers(g, line, mx, j, kx, ky);
  const size_t off = (size_t)line * Nz;
  const int tid = threadIdx.x;

  if (j == g.ny / 2) {  // y Nyquist row: identically zero
    for (int idx = tid; idx < 7 * Nz; idx += blockDim.x) {
      const int f = idx / Nz, n = idx - f * Nz;
      bw[(long long)f * fs + off + n] = from_d2<T2>(make_double2(0.0, 0.0));
    }
    return;
  }
  const ZSmem z = carve(zsm, Nz, N);
  const bool is00 = (mx == 0 && j == 0);
  const double k2 = kx * kx + ky * ky;

  for (int n = tid; n < Nz; n += blockDim.x) {
    LN(z, 10, Nz)[n] = st_om[off + n];
    LN(z, 11, Nz)[n] = st_w[off + n];
    LN(z, 12, Nz)[n] = st_phi[off + n];
    z.t1[n] = g.go1[n];
    z.t2[n] = g.go2[n];
    z.t3[n] = g.go3[n];
  }

  if (MODE == 0) {
    // ---- ten non-linear fields: samples -> Chebyshev coefficients
    for (int idx = tid; idx < 10 * Nz; idx += blockDim.x) {
      const int f = idx / Nz, n = idx - f * Nz;
      LN(z, f, Nz)[n] = to_d2(nl[(long long)f * fs + off + n]);
    }
    __syncthreads();
    for (int f0 = 0; f0 < 10; f0 += NBF) dct_forward_lines(z, f0, NBF, Nz, N, pz);
    // lines: 0 Sxx 1 Syy 2 Szz 3 Sxy 4 Sxz 5 Syz 6 phi^3 7 u phi 8 v phi 9 w phi
    {
      double2* src[3] = {LN(z, 4, Nz), LN(z, 5, Nz), LN(z, 2, Nz)};
      double2* dst[3] = {LN(z, 13, Nz), LN(z, 14, Nz), LN(z, 15, Nz)};
      dz_tasks(src, dst, 3, N);
    }
    __syncthreads();
    // S_i = i kx Sigma_ix + i ky Sigma_iy + D Sigma_iz
    for (int n = tid; n < Nz; n += blockDim.x) {
      const double2 sxx = LN(z, 0, Nz)[n], syy = LN(z, 1, Nz)[n];
      const double2 sxy = LN(z, 3, Nz)[n], sxz = LN(z, 4, Nz)[n], syz = LN(z, 5, Nz)[n];
      const double2 Sx = mul_i(kx * sxx + ky * sxy) + LN(z, 13, Nz)[n];
      const double2 Sy = mul_i(kx * sxy + ky * syy) + LN(z, 14, Nz)[n];
      const double2 Sz = mul_i(kx * sxz + ky * syz) + LN(z, 15, Nz)[n];
      double2 hom;
      if (is00) {  // mean flow: Sbar_x + i Sbar_y + (gx + i gy) delta_{n0}
        hom = make_double2(Sx.x + (n == 0 ? g.gx : 0.0), Sy.x + (n == 0 ? g.gy : 0.0));
      } else {
        hom = mul_i(kx * Sy - ky * Sx);  // i kx S_y - i ky S_x
      }
      LN(z, 2, Nz)[n] = Sz;
      LN(z, 3, Nz)[n] = hom;
      LN(z, 4, Nz)[n] = mul_i(kx * Sx + ky * Sy);  // i kx S_x + i ky S_y
      const double2 ph = LN(z, 12, Nz)[n];
      LN(z, 6, Nz)[n] = LN(z, 6, Nz)[n] - (1.0 + g.shat) * ph;  // G = phi^3 - (1+shat) phi
      LN(z, 7, Nz)[n] = -1.0 * mul_i(kx * LN(z, 7, Nz)[n] + ky * LN(z, 8, Nz)[n]);
    }
    __syncthreads();
    {
      double2* src[4] = {LN(z, 9, Nz), LN(z, 4, Nz), LN(z, 6, Nz), LN(z, 11, Nz)};
      double2* dst[4] = {LN(z, 13, Nz), LN(z, 14, Nz), LN(z, 15, Nz), LN(z, 5, Nz)};
      dz_tasks(src, dst, 4, N);
    }
    __syncthreads();
    {
      double2* src[2] = {LN(z, 15, Nz), LN(z, 5, Nz)};
      double2* dst[2] = {LN(z, 8, Nz), LN(z, 9, Nz)};
      dz_tasks(src, dst, 2, N);
    }
    __syncthreads();
    // h_w, S_phi, theta^n = (D^2 - k^2) w^n; AB2; right-hand sides
    const double twoRe = 2.0 * g.re;
    const double cphi = g.pe / (g.ch * g.ch);
    const double rdt = 1.0 / g.dt;
    const double rpe = 1.0 / g.pe;
    for (int n = tid; n < Nz; n += blockDim.x) {
      const double2 hw = is00 ? make_double2(0.0, 0.0)
                              : (-k2) * LN(z, 2, Nz)[n] - LN(z, 14, Nz)[n];
      const double2 sphi = LN(z, 7, Nz)[n] - LN(z, 13, Nz)[n] +
                           rpe * (LN(z, 8, Nz)[n] - k2 * LN(z, 6, Nz)[n]);
      const double2 hom = LN(z, 3, Nz)[n];
      const double2 th = LN(z, 9, Nz)[n] - k2 * LN(z, 11, Nz)[n];
      double2 Hom = hom, Hw = hw, Hphi = sphi;
      if (!first) {
        Hom = 1.5 * hom - 0.5 * h_om[off + n];
        Hw = 1.5 * hw - 0.5 * h_w[off + n];
        Hphi = 1.5 * sphi - 0.5 * h_phi[off + n];
      }
      h_om[off + n] = hom;
      h_w[off + n] = hw;
      h_phi[off + n] = sphi;
      LN(z, 0, Nz)[n] = (-2.0 * g.beta) * LN(z, 10, Nz)[n] - twoRe * Hom;
      LN(z, 1, Nz)[n] = (-2.0 * g.beta) * th - twoRe * Hw;
      LN(z, 4, Nz)[n] = cphi * (rdt * LN(z, 12, Nz)[n] + Hphi);
    }
    // ---- factor the three operators (both parities)
    if (tid < 6) {
      const int op = tid >> 1, p = tid & 1;
      const double alpha = (op == 0) ? k2 + g.beta : (op == 1) ? k2 : k2 + g.lam;
      sq[tid] = tau_factor(alpha, p, N, op == 2, z.t1, z.t2, z.t3, z.Y + op * Nz,
                           z.RD + op * Nz, z.Q + op * Nz);
    }
    __syncthreads();
    // ---- solves: warp 0 omega / mean flow, warp 1 w (influence matrix), warp 2 phi
    {
      const int warp = tid >> 5, lane = tid & 31;
      if (warp < 3 && lane < 4) {
        const int p = lane & 1, comp = lane >> 1;
        const int I = (N - p) / 2;
        if (warp == 0) {
          double* x = reinterpret_cast<double*>(LN(z, 0, Nz)) + comp;
          tau_sweep(x, p, N, k2 + g.beta, false, 0.0, z.t1, z.t2, z.t3, z.Y, z.RD, z.Q, sq[p]);
          double* o = reinterpret_cast<double*>(LN(z, 10, Nz)) + comp;
          for (int i = 0; i <= I; ++i) {
            const int n = p + 2 * i;
            o[2 * n] = x[2 * n] - o[2 * n];
          }
        } else if (warp == 1) {
          double* o = reinterpret_cast<double*>(LN(z, 11, Nz)) + comp;
          if (is00) {
            for (int i = 0; i <= I; ++i) o[2 * (p + 2 * i)] = 0.0;
          } else {
            double* x = reinterpret_cast<double*>(LN(z, 1, Nz)) + comp;
            double* hx = reinterpret_cast<double*>(LN(z, 2, Nz)) + comp;
            // particular pair: (D^2-k^2-beta) Psi = r, (D^2-k^2) Omega_p = Psi, Dirichlet 0
            tau_sweep(x, p, N, k2 + g.beta, false, 0.0, z.t1, z.t2, z.t3, z.Y, z.RD, z.Q, sq[p]);
            tau_sweep(x, p, N, k2, false, 0.0, z.t1, z.t2, z.t3, z.Y + Nz, z.RD + Nz, z.Q + Nz,
                      sq[2 + p]);
            // homogeneous pair of parity p: Psi_h = 1 at both walls (even) or +-1 (odd),
            // i.e. Psi_h = Q / SQ of the beta operator; then (D^2 - k^2) Omega_h = Psi_h
            for (int i = 0; i <= I; ++i) {
              const int n = p + 2 * i;
              hx[2 * n] = z.Q[n] / sq[p];
            }
            tau_sweep(hx, p, N, k2, false, 0.0, z.t1, z.t2, z.t3, z.Y + Nz, z.RD + Nz,
                      z.Q + Nz, sq[2 + p]);
            // choose c so that D Omega(+-1) = 0: sum n^2 (Omega_p + c Omega_h) = 0 per parity
            double sp = 0.0, sh = 0.0;
            for (int i = 0; i <= I; ++i) {
              const int n = p + 2 * i;
              const double n2 = (double)n * (double)n;
              sp = fma(n2, x[2 * n], sp);
              sh = fma(n2, hx[2 * n], sh);
            }
            const double c = -sp / sh;
            for (int i = 0; i <= I; ++i) {
              const int n = p + 2 * i;
              o[2 * n] = fma(c, hx[2 * n], x[2 * n]) - o[2 * n];
            }
          }
        } else {
          double* x = reinterpret_cast<double*>(LN(z, 4, Nz)) + comp;
          const double a = k2 + g.lam;
          tau_sweep(x, p, N, a, true, 0.0, z.t1, z.t2, z.t3, z.Y + 2 * Nz, z.RD + 2 * Nz,
                    z.Q + 2 * Nz, sq[4 + p]);
          tau_sweep(x, p, N, a, true, 0.0, z.t1, z.t2, z.t3, z.Y + 2 * Nz, z.RD + 2 * Nz,
                    z.Q + 2 * Nz, sq[4 + p]);
          double* o = reinterpret_cast<double*>(LN(z, 12, Nz)) + comp;
          for (int i = 0; i <= I; ++i) {
            const int n = p + 2 * i;
            o[2 * n] = x[2 * n];
          }
        }
      }
    }
    __syncthreads();
    for (int n = tid; n < Nz; n += blockDim.x) {
      st_om[off + n] = LN(z, 10, Nz)[n];
      st_w[off + n] = LN(z, 11, Nz)[n];
      st_phi[off + n] = LN(z, 12, Nz)[n];
    }
  } else {
    __syncthreads();
  }
  backward_fields<T2>(z, g, kx, ky, is00, pz, bw, fs, off);
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
  dct_forward_lines(z, 0, 2, Nz, N, pz);
  dct_forward_lines(z, 2, 2, Nz, N, pz);
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
      dct_forward_lines(z, 0, cnt, Nz, N, pz);
      for (int idx = threadIdx.x; idx < cnt * Nz; idx += blockDim.x) {
        const int f = idx / Nz, n = idx - f * Nz;
        out[(long long)(f0 + f) * fs + off + n] = LN(z, f, Nz)[n];
      }
      __syncthreads();
    } else {
      dct_backward_lines_store<double2>(z, 0, cnt, Nz, N, pz, out, fs, off, f0);
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

}  // namespace

size_t zline_smem(const GridDev& g) {
  return (size_t)(NLINES * g.nz + 2 * NBF * 2 * g.N) * sizeof(double2) +
         (size_t)12 * g.nz * sizeof(double);
}

template <typename T, int MODE>
static cudaError_t launch_zline_t(const GridDev& g, const void* nl, void* bw, long long fs,
                                  double2* st_om, double2* st_w, double2* st_phi, double2* h_om,
                                  double2* h_w, double2* h_phi, int first, const FftPlan& pz,
                                  cudaStream_t s) {
  typedef typename C2<T>::t T2;
  const size_t smem = zline_smem(g);
  static int cur = 0;
  cudaError_t e = ensure_smem(zline_kernel<T, MODE>, smem, &cur);
  if (e != cudaSuccess) return e;
  zline_kernel<T, MODE><<<g.Mx * g.ny, ZT, smem, s>>>(g, (const T2*)nl, (T2*)bw, fs, st_om, st_w,
                                                     st_phi, h_om, h_w, h_phi, first, pz);
  return cudaGetLastError();
}

cudaError_t launch_zline(int mode, int prec, const GridDev& g, const void* nl, void* bw,
                         long long fs, double2* st_om, double2* st_w, double2* st_phi,
                         double2* h_om, double2* h_w, double2* h_phi, int first,
                         const FftPlan& pz, cudaStream_t s) {
  if (prec == 0) {
    if (mode == 0)
      return launch_zline_t<double, 0>(g, nl, bw, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, first, pz, s);
    return launch_zline_t<double, 1>(g, nl, bw, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, first, pz, s);
  }
  if (mode == 0)
    return launch_zline_t<float, 0>(g, nl, bw, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, first, pz, s);
  return launch_zline_t<float, 1>(g, nl, bw, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, first, pz, s);
}

cudaError_t launch_project(const GridDev& g, const double2* uvwp, long long fs, double2* st_om,
                           double2* st_w, double2* st_phi, double2* h_om, double2* h_w,
                           double2* h_phi, const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static int cur = 0;
  cudaError_t e = ensure_smem(project_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  project_kernel<<<g.Mx * g.ny, ZT, smem, s>>>(g, uvwp, fs, st_om, st_w, st_phi, h_om, h_w, h_phi, pz);
  return cudaGetLastError();
}

cudaError_t launch_dct_lines(int dir, int prec, const GridDev& g, const void* in, double2* out,
                             int nf, long long fs, const FftPlan& pz, cudaStream_t s) {
  const size_t smem = zline_smem(g);
  static int cur64 = 0, cur32 = 0;
  cudaError_t e = ensure_smem(dct_lines_kernel<double>, smem, &cur64);
  if (e == cudaSuccess) e = ensure_smem(dct_lines_kernel<float>, smem, &cur32);
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    dct_lines_kernel<double><<<g.Mx * g.ny, ZT, smem, s>>>(g, dir, (const double2*)in, out, nf, fs, pz);
  } else {
    dct_lines_kernel<float><<<g.Mx * g.ny, ZT, smem, s>>>(g, dir, (const float2*)in, out, nf, fs, pz);
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
