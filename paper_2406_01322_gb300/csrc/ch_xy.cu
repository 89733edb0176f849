// Periodic-direction kernels: the y pass and the fused x-line kernel of the pseudo-spectral step.
//
// Paper Sec. 3.2.1: batched real-to-complex transforms along x and complex transforms along y
// (3/2-rule zero padding on the way to physical space, truncation on the way back), and
// Sec. 3.2.2: element-wise (Hadamard) products of collocated fields in physical space.  Here the
// x transforms and the products are one kernel, so the padded physical fields live only in
// shared memory and never reach HBM.
//
// Layout of every intermediate array: (mx, y or ky, z) with z fastest; a CTA owns a tile of
// lines and does the layout change through shared memory.
#include "ch_internal.h"

namespace chf {

namespace {

constexpr int YT = 256;   // threads of a y-pass CTA
constexpr int XT = 256;   // threads of an x-line CTA

// y pass: one CTA per (z tile, mx, field).
//   INV (backward): in (Mx, Ny, Nz) modes -> out (Mx, P, Nz) samples, modes |my| < Ny/2 placed,
//   the rest zero.  Forward: in (Mx, P, Nz) samples -> out (Mx, Ny, Nz) kept modes * scale.
template <typename T, bool INV>
__device__ __forceinline__ void ypass_body(const typename C2<T>::t* __restrict__ in,
                                           typename C2<T>::t* __restrict__ out, int Mx, int Ny,
                                           int P, int Nz, int TZ, long long fs_in,
                                           long long fs_out, T scale, const FftPlan& pl,
                                           const YMap& map, int bx, int by, int bz) {
  typedef typename C2<T>::t T2;
  extern __shared__ unsigned char ysm_raw[];
  const int LS = yline_stride(P);
  T2* A = reinterpret_cast<T2*>(ysm_raw);
  T2* B = A + TZ * LS;
  const int z0 = bx * TZ;
  const int mx = by;
  const int f = bz;                  // output field
  const int h = Ny / 2;
  const T2 zero = mk((T)0, (T)0);
  const int tzs = __ffs(TZ) - 1;     // TZ is a power of two: idx / TZ = idx >> tzs
  if (INV) {
    const T2* src = in + map.src[f] * fs_in + (size_t)mx * Ny * Nz;
    const bool dy = (map.dy_mask >> f) & 1;   // output d/dy of the input field (times i ky)
    for (int idx = threadIdx.x; idx < Ny * TZ; idx += blockDim.x) {
      const int jj = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      T2 v = zero;
      if (z < Nz && jj != h) v = src[(size_t)jj * Nz + z];
      if (dy) {
        const T ky = (T)map.kys * (T)((jj < h) ? jj : jj - Ny);
        v = mk(-ky * v.y, ky * v.x);
      }
      const int p = (jj < h) ? jj : P - Ny + jj;
      A[zz * LS + p] = v;
    }
    // positions h .. P-h-1 hold no mode; a pruned transform does not read them
    if (!pl.prune)
      for (int idx = threadIdx.x; idx < (P - Ny) * TZ; idx += blockDim.x) {
        const int q = idx >> tzs, zz = idx & (TZ - 1);
        A[zz * LS + h + q] = zero;
      }
  } else {
    const T2* src = in + map.src[f] * fs_in + (size_t)mx * P * Nz;
    for (int idx = threadIdx.x; idx < P * TZ; idx += blockDim.x) {
      const int y = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      A[zz * LS + y] = (z < Nz) ? src[(size_t)y * Nz + z] : zero;
    }
  }
  __syncthreads();
  const T2* R = block_fft<T, INV, true>(A, B, TZ, LS, pl, true);
  if (INV) {
    T2* dst = out + f * fs_out + (size_t)mx * P * Nz;
    for (int idx = threadIdx.x; idx < P * TZ; idx += blockDim.x) {
      const int y = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      if (z < Nz) dst[(size_t)y * Nz + z] = R[zz * LS + y];
    }
  } else {
    T2* dst = out + f * fs_out + (size_t)mx * Ny * Nz;
    for (int idx = threadIdx.x; idx < Ny * TZ; idx += blockDim.x) {
      const int jj = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      if (z >= Nz) continue;
      const int p = (jj < h) ? jj : P - Ny + jj;
      dst[(size_t)jj * Nz + z] = (jj == h) ? zero : scale * R[zz * LS + p];
    }
  }
}

template <typename T, bool INV>
__global__ void __launch_bounds__(YT) ypass_kernel(const typename C2<T>::t* __restrict__ in,
                                                   typename C2<T>::t* __restrict__ out, int Mx,
                                                   int Ny, int P, int Nz, int TZ, long long fs_in,
                                                   long long fs_out, T scale, FftPlan pl,
                                                   YMap map) {
  ypass_body<T, INV>(in, out, Mx, Ny, P, Nz, TZ, fs_in, fs_out, scale, pl, map, blockIdx.x,
                     blockIdx.y, blockIdx.z);
}

// Forward y pass with the assembly's combinations (launch_ycomb): work item -> (group, mx, z
// tile); the nine products are transformed in groups so that each CTA holds every input its
// outputs combine.  Groups and outputs as stated at launch_ycomb; the arithmetic of the
// combinations is that of the working precision T.
template <typename T>
__device__ __forceinline__ void ycomb_body(const typename C2<T>::t* __restrict__ in,
                                           typename C2<T>::t* __restrict__ out, int Mx, int Ny,
                                           int P, int Nz, int L, long long fs_in,
                                           long long fs_out, T scale, T kxs, T kys,
                                           const FftPlan& pl, int item) {
  typedef typename C2<T>::t T2;
  extern __shared__ unsigned char ysm_raw[];
  int grp = 0, rest = item;
  for (; grp < kYcGroups - 1; ++grp) {
    const int n = ycomb_group_items(grp, Mx, Nz, L);
    if (rest < n) break;
    rest -= n;
  }
  const int tzs = ycomb_tzs(grp, L);
  const int TZ = 1 << tzs;
  const int nzt = (Nz + TZ - 1) >> tzs;
  const int mx = rest / nzt;
  const int z0 = (rest - mx * nzt) * TZ;
  const int nin = ycomb_nin(grp);
  const int LS = yline_stride(P);
  T2* A = reinterpret_cast<T2*>(ysm_raw);
  T2* B = A + nin * TZ * LS;
  const T2 zero = mk((T)0, (T)0);
  // input products: 0 Sxx' 1 Syy' 2 Sxy 3 Sxz 4 Syz 5 phi^3 6 u phi 7 v phi 8 w phi
  const int f0 = grp == 0 ? 0 : grp == 1 ? 3 : grp == 2 ? 6 : grp == 3 ? 8 : 5;
  for (int f = 0; f < nin; ++f) {
    const T2* src = in + (f0 + f) * fs_in + (size_t)mx * P * Nz;
    T2* Af = A + f * TZ * LS;
    for (int idx = threadIdx.x; idx < P * TZ; idx += blockDim.x) {
      const int y = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      Af[zz * LS + y] = (z < Nz) ? src[(size_t)y * Nz + z] : zero;
    }
  }
  __syncthreads();
  const T2* R = block_fft<T, false, true>(A, B, nin * TZ, LS, pl, true);
  const int h = Ny / 2;
  const T kx = kxs * (T)mx;
  T2* dst = out + (size_t)mx * Ny * Nz;
  for (int idx = threadIdx.x; idx < Ny * TZ; idx += blockDim.x) {
    const int jj = idx >> tzs, zz = idx & (TZ - 1);
    const int z = z0 + zz;
    if (z >= Nz) continue;
    const size_t o = (size_t)jj * Nz + z;
    const int p = (jj < h) ? jj : P - Ny + jj;
    const bool nyq = (jj == h);   // the y Nyquist row is zero
    const bool mean = (mx == 0 && jj == 0);
    const T ky = kys * (T)((jj < h) ? jj : jj - Ny);
    T2 v[3];
#pragma unroll
    for (int f = 0; f < 3; ++f)
      v[f] = (nyq || f >= nin) ? zero : scale * R[(f * TZ + zz) * LS + p];
    if (grp == 0) {
      const T2 a = mul_i(kx * v[0] + ky * v[2]);
      const T2 b = mul_i(kx * v[2] + ky * v[1]);
      if (!mean) dst[o] = mul_i(kx * b - ky * a);
      dst[3 * fs_out + o] = mul_i(kx * a + ky * b);
    } else if (grp == 1) {
      if (mean) {
        dst[o] = v[0];
        dst[fs_out + o] = v[1];
      } else {
        dst[fs_out + o] = mul_i(kx * v[1] - ky * v[0]);
      }
      dst[2 * fs_out + o] = mul_i(kx * v[0] + ky * v[1]);
    } else if (grp == 2) {
      dst[4 * fs_out + o] = mul_mi(kx * v[0] + ky * v[1]);
    } else {
      dst[(grp == 3 ? 5 : 6) * fs_out + o] = v[0];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(YT) ycomb_kernel(const typename C2<T>::t* __restrict__ in,
                                                   typename C2<T>::t* __restrict__ out, int Mx,
                                                   int Ny, int P, int Nz, int L, long long fs_in,
                                                   long long fs_out, T scale, T kxs, T kys,
                                                   FftPlan pl) {
  ycomb_body<T>(in, out, Mx, Ny, P, Nz, L, fs_in, fs_out, scale, kxs, kys, pl, blockIdx.x);
}

// Fused x-line kernel.  One CTA per (pair of z rows, y).  The two rows z0, z0+1 of a field are
// packed as one complex signal a + i b, so one complex FFT of length Px transforms both.
//   1. six inputs u, v, w, phi, phi_y, phi_z (spectra kx < Mx); phi_x = i kx phi is formed from
//      phi's spectrum; seven c2r transforms (zero padded);
//   2. nine products at every padded point: Sigma_xx - Sigma_zz, Sigma_yy - Sigma_zz, Sigma_xy,
//      Sigma_xz, Sigma_yz (Sigma_ij = -u_i u_j + kappa (|grad phi|^2 delta_ij - phi_i phi_j);
//      the isotropic part Sigma_zz delta_ij is a gradient and drops out of h_omega and h_w),
//      phi^3, u phi, v phi, w phi;
//   3. r2c, keep kx < Mx, times `scale`.
// Shared memory: 7 + 5 + 5 lines of Px complex values.
template <typename T, bool LOOP = false>
__device__ __forceinline__ void xline_body(const typename C2<T>::t* __restrict__ in,
                                           typename C2<T>::t* __restrict__ out, int Mx, int Px,
                                           int Py, int Nz, long long fs, T kappa, T scale, T kxs,
                                           const FftPlan& pl, int bx, int by) {
  typedef typename C2<T>::t T2;
  extern __shared__ unsigned char xsm_raw[];
  T2* S = reinterpret_cast<T2*>(xsm_raw);
  const int LS = fft_line_stride(Px);   // line stride: room for the FFT's skewed intermediates
  const int z0 = 2 * bx;
  const int y = by;
  const bool two = (z0 + 1 < Nz);
  const T2 zero = mk((T)0, (T)0);
  const size_t base = (size_t)y * Nz + z0;
  const size_t mstride = (size_t)Py * Nz;
  // Start in S[0..6] for an even number of passes, in S[7..13] for an odd number, so that the
  // seven physical lines always end in S[0..6] and S[7..16] (ten lines) are free afterwards.
  T2* X = S;
  T2* Y = S + 7 * LS;
  T2* L0 = (pl.nst & 1) ? Y : X;
  // ---- 1. packed spectra: lines u v w phi phi_x phi_y phi_z
  const float inv_mx = 1.0f / (float)Mx;
  for (int idx = threadIdx.x; idx < 7 * Mx; idx += blockDim.x) {
    int m;
    const int f = fdivmod(idx, Mx, inv_mx, &m);
    const int src_f = (f < 4) ? f : f - 1;      // phi_x (line 4) comes from phi (input 3)
    const T2* src = in + src_f * fs + (size_t)m * mstride + base;
    T2 a = src[0];
    T2 b = two ? src[1] : zero;
    if (f == 4) {                                // i kx phi
      const T kx = kxs * (T)m;
      a = mk(-kx * a.y, kx * a.x);
      b = mk(-kx * b.y, kx * b.x);
    }
    T2* L = L0 + f * LS;
    if (m == 0) {
      L[0] = mk(a.x, b.x);  // the imaginary part of a DC coefficient is not used by c2r
    } else {
      L[m] = mk(a.x - b.y, a.y + b.x);         // a + i b
      L[Px - m] = mk(a.x + b.y, b.x - a.y);    // conj(a) + i conj(b)
    }
  }
  {
    // kx = Mx .. Px - Mx carry no mode; a pruned transform reads only the last of them
    const int w0 = pl.prune ? Px - 2 * Mx : 0;
    const int w = Px - 2 * Mx + 1 - w0;
    const float inv_w = 1.0f / (float)w;
    for (int idx = threadIdx.x; idx < 7 * w; idx += blockDim.x) {
      int q;
      const int f = fdivmod(idx, w, inv_w, &q);
      L0[f * LS + Mx + w0 + q] = zero;
    }
  }
  __syncthreads();
  const T2* in7 = block_fft<T, true, true, LOOP>(L0, (L0 == X) ? Y : X, 7, LS, pl, true);  // == X
  T2* prod = S + 7 * LS;   // five product lines
  T2* scr = S + 12 * LS;   // five scratch lines
  for (int g0 = 0; g0 < 9; g0 += 5) {
    const int cnt = (g0 == 0) ? 5 : 4;
    // ---- 2. products for outputs g0 .. g0+cnt-1 (rows z0 in .x, z0+1 in .y)
    for (int x = threadIdx.x; x < Px; x += blockDim.x) {
      const T2 u = in7[x], v = in7[LS + x], w = in7[2 * LS + x], ph = in7[3 * LS + x];
      const T2 fx = in7[4 * LS + x], fy = in7[5 * LS + x], fz = in7[6 * LS + x];
      if (g0 == 0) {
        const T2 wz = mk(w.x * w.x + kappa * fz.x * fz.x, w.y * w.y + kappa * fz.y * fz.y);
        prod[x] = mk(wz.x - u.x * u.x - kappa * fx.x * fx.x, wz.y - u.y * u.y - kappa * fx.y * fx.y);
        prod[LS + x] = mk(wz.x - v.x * v.x - kappa * fy.x * fy.x, wz.y - v.y * v.y - kappa * fy.y * fy.y);
        prod[2 * LS + x] = mk(-u.x * v.x - kappa * fx.x * fy.x, -u.y * v.y - kappa * fx.y * fy.y);
        prod[3 * LS + x] = mk(-u.x * w.x - kappa * fx.x * fz.x, -u.y * w.y - kappa * fx.y * fz.y);
        prod[4 * LS + x] = mk(-v.x * w.x - kappa * fy.x * fz.x, -v.y * w.y - kappa * fy.y * fz.y);
      } else {
        prod[x] = mk(ph.x * ph.x * ph.x, ph.y * ph.y * ph.y);
        prod[LS + x] = mk(u.x * ph.x, u.y * ph.y);
        prod[2 * LS + x] = mk(v.x * ph.x, v.y * ph.y);
        prod[3 * LS + x] = mk(w.x * ph.x, w.y * ph.y);
      }
    }
    __syncthreads();
    const T2* R = block_fft<T, false, true, LOOP>(prod, scr, cnt, LS, pl, true);
    // ---- 3. unpack: A_k = (Z_k + conj Z_{-k}) / 2, B_k = (Z_k - conj Z_{-k}) / (2 i)
    const T hs = (T)0.5 * scale;
    for (int idx = threadIdx.x; idx < cnt * Mx; idx += blockDim.x) {
      int m;
      const int q = fdivmod(idx, Mx, inv_mx, &m);
      const T2 Zk = R[q * LS + m];
      const T2 Zm = R[q * LS + (m == 0 ? 0 : Px - m)];
      T2* dst = out + (g0 + q) * fs + (size_t)m * mstride + base;
      dst[0] = mk(hs * (Zk.x + Zm.x), hs * (Zk.y - Zm.y));
      if (two) dst[1] = mk(hs * (Zk.y + Zm.y), hs * (Zm.x - Zk.x));
    }
    __syncthreads();
  }
}

template <typename T, bool LOOP, int NTH>
__global__ void __launch_bounds__(NTH) xline_kernel(const typename C2<T>::t* __restrict__ in,
                                                   typename C2<T>::t* __restrict__ out, int Mx,
                                                   int Px, int Py, int Nz, long long fs, T kappa,
                                                   T scale, T kxs, FftPlan pl) {
  xline_body<T, LOOP>(in, out, Mx, Px, Py, Nz, fs, kappa, scale, kxs, pl, blockIdx.x, blockIdx.y);
}

// plain r2c along x of physical rows (Nz, Ny, Nx) -> (Mx, Ny, Nz); two z rows per CTA
__global__ void __launch_bounds__(128) x_r2c_kernel(const double* __restrict__ phys,
                                                    double2* __restrict__ out, int Nx, int Ny,
                                                    int Nz, long long fs_phys, long long fs_spec,
                                                    FftPlan pl) {
  extern __shared__ double2 xs[];
  double2* A = xs;
  double2* B = xs + Nx;
  const int z0 = 2 * blockIdx.x, y = blockIdx.y, f = blockIdx.z;
  const bool two = (z0 + 1 < Nz);
  const int Mx = Nx / 2;
  const double* r0 = phys + f * fs_phys + ((size_t)z0 * Ny + y) * Nx;
  const double* r1 = r0 + (size_t)Ny * Nx;
  for (int x = threadIdx.x; x < Nx; x += blockDim.x) A[x] = make_double2(r0[x], two ? r1[x] : 0.0);
  __syncthreads();
  const double2* R = block_fft<double, false>(A, B, 1, Nx, pl);
  double2* dst = out + f * fs_spec + (size_t)y * Nz + z0;
  for (int m = threadIdx.x; m < Mx; m += blockDim.x) {
    const double2 Zk = R[m], Zm = R[m == 0 ? 0 : Nx - m];
    dst[(size_t)m * Ny * Nz] = make_double2(0.5 * (Zk.x + Zm.x), 0.5 * (Zk.y - Zm.y));
    if (two) dst[(size_t)m * Ny * Nz + 1] = make_double2(0.5 * (Zk.y + Zm.y), 0.5 * (Zm.x - Zk.x));
  }
}

// plain c2r along x: (Mx, Ny, Nz) -> physical rows (Nz, Ny, Nx)
__global__ void __launch_bounds__(128) x_c2r_kernel(const double2* __restrict__ in,
                                                    double* __restrict__ phys, int Nx, int Ny,
                                                    int Nz, long long fs_spec, long long fs_phys,
                                                    FftPlan pl) {
  extern __shared__ double2 xs[];
  double2* A = xs;
  double2* B = xs + Nx;
  const int z0 = 2 * blockIdx.x, y = blockIdx.y, f = blockIdx.z;
  const bool two = (z0 + 1 < Nz);
  const int Mx = Nx / 2;
  const double2* src = in + f * fs_spec + (size_t)y * Nz + z0;
  for (int m = threadIdx.x; m < Mx; m += blockDim.x) {
    const double2 a = src[(size_t)m * Ny * Nz];
    const double2 b = two ? src[(size_t)m * Ny * Nz + 1] : make_double2(0.0, 0.0);
    if (m == 0) {
      A[0] = make_double2(a.x, b.x);
      A[Mx] = make_double2(0.0, 0.0);  // x Nyquist
    } else {
      A[m] = make_double2(a.x - b.y, a.y + b.x);
      A[Nx - m] = make_double2(a.x + b.y, b.x - a.y);
    }
  }
  __syncthreads();
  const double2* R = block_fft<double, true>(A, B, 1, Nx, pl);
  double* r0 = phys + f * fs_phys + ((size_t)z0 * Ny + y) * Nx;
  double* r1 = r0 + (size_t)Ny * Nx;
  for (int x = threadIdx.x; x < Nx; x += blockDim.x) {
    r0[x] = R[x].x;
    if (two) r1[x] = R[x].y;
  }
}

// Transposed x-line kernel (float64, discrete adjoint of xline_kernel with scale 1).
// Per (pair of z rows, y): the seven forward inputs are re-synthesised from `in` (as in the
// forward kernel); the nine product adjoints `pb` (kept modes kx < Mx) go to physical space by
// the transpose of the truncated r2c, i.e. a c2r of the half spectrum with modes kx >= 1 halved;
// the pointwise Jacobian of the nine products is applied transposed, accumulating the adjoints
// of u, v, w, phi, phi_x, phi_y, phi_z; those go back by the transpose of the zero-padded c2r,
// an r2c with modes kx >= 1 doubled; phi_x = i kx phi folds into phi with -i kx.
// Outputs (spectra kx < Mx, layout of `in`): u, v, w, phi, phi_y, phi_z adjoints.
// Shared memory: 24 lines of Px complex values (7 forward, 7 accumulators, 5 + 5 product/scratch).
__global__ void __launch_bounds__(XT) adj_xline_kernel(const double2* __restrict__ in,
                                                       const double2* __restrict__ pb,
                                                       double2* __restrict__ out, int Mx, int Px,
                                                       int Py, int Nz, long long fs, double kappa,
                                                       double kxs, FftPlan pl) {
  extern __shared__ double2 axs[];
  double2* S = axs;
  const int z0 = 2 * blockIdx.x;
  const int y = blockIdx.y;
  const bool two = (z0 + 1 < Nz);
  const double2 zero = make_double2(0.0, 0.0);
  const size_t base = (size_t)y * Nz + z0;
  const size_t mstride = (size_t)Py * Nz;
  const bool odd = (pl.nst & 1);
  // ---- forward inputs: start so that the result lands in S[0..6]
  double2* F0 = odd ? S + 7 * Px : S;
  for (int idx = threadIdx.x; idx < 7 * Mx; idx += blockDim.x) {
    const int f = idx / Mx, m = idx - f * Mx;
    const int src_f = (f < 4) ? f : f - 1;
    const double2* src = in + src_f * fs + (size_t)m * mstride + base;
    double2 a = src[0];
    double2 b = two ? src[1] : zero;
    if (f == 4) {
      const double kx = kxs * m;
      a = make_double2(-kx * a.y, kx * a.x);
      b = make_double2(-kx * b.y, kx * b.x);
    }
    double2* L = F0 + f * Px;
    if (m == 0) {
      L[0] = make_double2(a.x, b.x);
    } else {
      L[m] = make_double2(a.x - b.y, a.y + b.x);
      L[Px - m] = make_double2(a.x + b.y, b.x - a.y);
    }
  }
  {
    const int w = Px - 2 * Mx + 1;
    for (int idx = threadIdx.x; idx < 7 * w; idx += blockDim.x) {
      const int f = idx / w, q = idx - f * w;
      F0[f * Px + Mx + q] = zero;
    }
  }
  __syncthreads();
  const double2* in7 = block_fft<double, true>(F0, odd ? S : S + 7 * Px, 7, Px, pl);  // == S
  double2* acc = S + 7 * Px;       // seven accumulator lines
  double2* P0 = S + 14 * Px;       // five product-adjoint lines (result position)
  double2* P1 = S + 19 * Px;       // five scratch lines
  for (int g0 = 0; g0 < 9; g0 += 5) {
    const int cnt = (g0 == 0) ? 5 : 4;
    double2* L0 = odd ? P1 : P0;
    for (int idx = threadIdx.x; idx < cnt * Mx; idx += blockDim.x) {
      const int q = idx / Mx, m = idx - q * Mx;
      const double2* src = pb + (g0 + q) * fs + (size_t)m * mstride + base;
      double2 a = src[0];
      double2 b = two ? src[1] : zero;
      double2* L = L0 + q * Px;
      if (m == 0) {
        L[0] = make_double2(a.x, b.x);
      } else {
        a = 0.5 * a;
        b = 0.5 * b;
        L[m] = make_double2(a.x - b.y, a.y + b.x);
        L[Px - m] = make_double2(a.x + b.y, b.x - a.y);
      }
    }
    {
      const int w = Px - 2 * Mx + 1;
      for (int idx = threadIdx.x; idx < cnt * w; idx += blockDim.x) {
        const int q = idx / w, r = idx - q * w;
        L0[q * Px + Mx + r] = zero;
      }
    }
    __syncthreads();
    const double2* pr = block_fft<double, true>(L0, odd ? P0 : P1, cnt, Px, pl);  // == P0
    for (int x = threadIdx.x; x < Px; x += blockDim.x) {
      const double2 u = in7[x], v = in7[Px + x], w = in7[2 * Px + x], ph = in7[3 * Px + x];
      const double2 fx = in7[4 * Px + x], fy = in7[5 * Px + x], fz = in7[6 * Px + x];
      if (g0 == 0) {
        const double2 b0 = pr[x], b1 = pr[Px + x], b2 = pr[2 * Px + x], b3 = pr[3 * Px + x],
                      b4 = pr[4 * Px + x];
        double2 r;
#define ADJ0(C)                                                                             \
        r.C = -2.0 * u.C * b0.C - v.C * b2.C - w.C * b3.C;                                  \
        acc[x].C = r.C;                                                                     \
        r.C = -2.0 * v.C * b1.C - u.C * b2.C - w.C * b4.C;                                  \
        acc[Px + x].C = r.C;                                                                \
        r.C = 2.0 * w.C * (b0.C + b1.C) - u.C * b3.C - v.C * b4.C;                          \
        acc[2 * Px + x].C = r.C;                                                            \
        acc[3 * Px + x].C = 0.0;                                                            \
        r.C = kappa * (-2.0 * fx.C * b0.C - fy.C * b2.C - fz.C * b3.C);                     \
        acc[4 * Px + x].C = r.C;                                                            \
        r.C = kappa * (-2.0 * fy.C * b1.C - fx.C * b2.C - fz.C * b4.C);                     \
        acc[5 * Px + x].C = r.C;                                                            \
        r.C = kappa * (2.0 * fz.C * (b0.C + b1.C) - fx.C * b3.C - fy.C * b4.C);             \
        acc[6 * Px + x].C = r.C;
        ADJ0(x)
        ADJ0(y)
#undef ADJ0
      } else {
        const double2 b5 = pr[x], b6 = pr[Px + x], b7 = pr[2 * Px + x], b8 = pr[3 * Px + x];
#define ADJ1(C)                                                                             \
        acc[x].C += ph.C * b6.C;                                                            \
        acc[Px + x].C += ph.C * b7.C;                                                       \
        acc[2 * Px + x].C += ph.C * b8.C;                                                   \
        acc[3 * Px + x].C = 3.0 * ph.C * ph.C * b5.C + u.C * b6.C + v.C * b7.C + w.C * b8.C;
        ADJ1(x)
        ADJ1(y)
#undef ADJ1
      }
    }
    __syncthreads();
  }
  // ---- r2c of the seven accumulators (kx >= 1 doubled), fold phi_x into phi
  const double2* R = block_fft<double, false>(acc, P0, 7, Px, pl);
  for (int idx = threadIdx.x; idx < 6 * Mx; idx += blockDim.x) {
    const int q = idx / Mx, m = idx - q * Mx;
    const int line = (q < 4) ? q : q + 1;           // skip phi_x (line 4)
    const double hs = (m == 0) ? 0.5 : 1.0;
    const int mm = (m == 0) ? 0 : Px - m;
    double2 Zk = R[line * Px + m], Zm = R[line * Px + mm];
    double2 A = make_double2(hs * (Zk.x + Zm.x), hs * (Zk.y - Zm.y));
    double2 B = make_double2(hs * (Zk.y + Zm.y), hs * (Zm.x - Zk.x));
    if (q == 3) {  // + (-i kx) phi_x adjoint
      const double2 Xk = R[4 * Px + m], Xm = R[4 * Px + mm];
      const double2 Ax = make_double2(hs * (Xk.x + Xm.x), hs * (Xk.y - Xm.y));
      const double2 Bx = make_double2(hs * (Xk.y + Xm.y), hs * (Xm.x - Xk.x));
      const double kx = kxs * m;
      A = make_double2(A.x + kx * Ax.y, A.y - kx * Ax.x);
      B = make_double2(B.x + kx * Bx.y, B.y - kx * Bx.x);
    }
    double2* dst = out + q * fs + (size_t)m * mstride + base;
    dst[0] = A;
    if (two) dst[1] = B;
  }
}

int ytile_local(int P, size_t elem) {
  // z tile: 8 columns (128 B of fp64 complex), fewer when the lines are long
  int tz = 8;
  while (tz > 1 && ysmem_bytes(P, tz, elem) > 160 * 1024) tz /= 2;
  return tz;
}

// ---- grouped persistent launches (ensemble) ---------------------------------------------
__device__ __forceinline__ int member_of_xy(const int* __restrict__ begin, int nmem, int item) {
  int m = 0;
  while (m + 1 < nmem && begin[m + 1] <= item) ++m;
  return m;
}

template <typename T, bool INV>
__global__ void __launch_bounds__(YT) grouped_ypass_kernel(const Member* __restrict__ mem,
                                                           const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of_xy(begin, nmem, item);
    const Member& M = mem[m];
    const int TZ = INV ? M.tzb : M.tzf;
    const int nzt = (M.g.nz + TZ - 1) / TZ;
    const int local = item - begin[m];
    const int bx = local % nzt, rest = local / nzt;
    const int by = rest % M.g.Mx, bz = rest / M.g.Mx;
    if (INV)
      ypass_body<T, true>((const T2*)M.bw, (T2*)M.ya, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, TZ, M.fs,
                          M.fsy, (T)1, M.py, M.ym, bx, by, bz);
    else
      ypass_body<T, false>((const T2*)M.yb, (T2*)M.nl, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, TZ, M.fsy,
                           M.fs, (T)M.yscale, M.py, M.yf, bx, by, bz);
    __syncthreads();
  }
}

// grouped forward y pass with the combinations: items (group, mx, z tile) member by member
template <typename T>
__global__ void __launch_bounds__(YT) grouped_ycomb_kernel(const Member* __restrict__ mem,
                                                           const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of_xy(begin, nmem, item);
    const Member& M = mem[m];
    ycomb_body<T>((const T2*)M.yb, (T2*)M.nl, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, M.tzf, M.fsy, M.fs,
                  (T)M.yscale, (T)M.kxs, (T)M.ym.kys, M.py, item - begin[m]);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(XT) grouped_xline_kernel(const Member* __restrict__ mem,
                                                           const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of_xy(begin, nmem, item);
    const Member& M = mem[m];
    const int nzp = (M.g.nz + 1) / 2;
    const int local = item - begin[m];
    xline_body<T>((const T2*)M.ya, (T2*)M.yb, M.g.Mx, M.g.Px, M.g.Py, M.g.nz, M.fsy,
                  (T)M.g.kappa, (T)1, (T)M.kxs, M.px, local % nzp, local / nzp);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_ypass(int dir, int prec, const GridDev& g, int P, const void* in, void* out,
                         int nf, long long fs_in, long long fs_out, double scale,
                         const FftPlan& py, cudaStream_t s, const YMap* mapp) {
  YMap map;
  if (mapp) {
    map = *mapp;
  } else {
    for (int f = 0; f < YMap::kMax; ++f) map.src[f] = f;
    map.dy_mask = 0;
  }
  map.kys = 6.283185307179586476925 / g.ly;
  const size_t elem = prec == 1 ? sizeof(float2) : sizeof(double2);
  const int TZ = ytile_local(P, elem);
  const size_t smem = ysmem_bytes(P, TZ, elem);
  dim3 grid((g.nz + TZ - 1) / TZ, g.Mx, nf);
  static SmemLimit cur[6];
  cudaError_t e = cudaSuccess;
  if (prec == 0) e = dir == 1 ? ensure_smem(ypass_kernel<double, true>, smem, &cur[0])
                              : ensure_smem(ypass_kernel<double, false>, smem, &cur[1]);
  else if (prec == 1) e = dir == 1 ? ensure_smem(ypass_kernel<float, true>, smem, &cur[2])
                                   : ensure_smem(ypass_kernel<float, false>, smem, &cur[3]);
  else e = dir == 1 ? ensure_smem(ypass_kernel<df, true>, smem, &cur[4])
                    : ensure_smem(ypass_kernel<df, false>, smem, &cur[5]);
  if (e != cudaSuccess) return e;
#define YL(T, INV)                                                                            \
  ypass_kernel<T, INV><<<grid, YT, smem, s>>>((const C2<T>::t*)in, (C2<T>::t*)out, g.Mx, g.ny, \
                                              P, g.nz, TZ, fs_in, fs_out, T(scale), py, map);
  if (prec == 0) {
    if (dir == 1) { YL(double, true) } else { YL(double, false) }
  } else if (prec == 1) {
    if (dir == 1) { YL(float, true) } else { YL(float, false) }
  } else {
    if (dir == 1) { YL(df, true) } else { YL(df, false) }
  }
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_ycomb(int prec, const GridDev& g, const void* in, void* out, long long fs_in,
                         long long fs_out, double scale, const FftPlan& py, cudaStream_t s) {
  const size_t elem = prec == 1 ? sizeof(float2) : sizeof(double2);
  const int L = ytile_local(g.Py, elem);
  const size_t smem = ycomb_smem(g.Py, L, elem);
  const int items = ycomb_items(g.Mx, g.nz, L);
  static SmemLimit cur[3];
  cudaError_t e = prec == 0   ? ensure_smem(ycomb_kernel<double>, smem, &cur[0])
                  : prec == 1 ? ensure_smem(ycomb_kernel<float>, smem, &cur[1])
                              : ensure_smem(ycomb_kernel<df>, smem, &cur[2]);
  if (e != cudaSuccess) return e;
  const double kxs = 6.283185307179586476925 / g.lx, kys = 6.283185307179586476925 / g.ly;
  if (prec == 0)
    ycomb_kernel<double><<<items, YT, smem, s>>>((const double2*)in, (double2*)out, g.Mx, g.ny,
                                                 g.Py, g.nz, L, fs_in, fs_out, scale, kxs, kys,
                                                 py);
  else if (prec == 1)
    ycomb_kernel<float><<<items, YT, smem, s>>>((const float2*)in, (float2*)out, g.Mx, g.ny,
                                                g.Py, g.nz, L, fs_in, fs_out, (float)scale,
                                                (float)kxs, (float)kys, py);
  else
    ycomb_kernel<df><<<items, YT, smem, s>>>((const df2*)in, (df2*)out, g.Mx, g.ny, g.Py, g.nz,
                                             L, fs_in, fs_out, df(scale), df(kxs), df(kys), py);
  return cudaGetLastError();
}

template <bool LOOP, int NTH>
cudaError_t launch_xline_t(int prec, const GridDev& g, const void* in7, void* out10,
                           long long fs, double scale, const FftPlan& px, size_t smem,
                           cudaStream_t s) {
  dim3 grid((g.nz + 1) / 2, g.Py);
  static SmemLimit cur64, cur32, curdf;
  cudaError_t e = prec == 0 ? ensure_smem(xline_kernel<double, LOOP, NTH>, smem, &cur64)
                  : prec == 1 ? ensure_smem(xline_kernel<float, LOOP, NTH>, smem, &cur32)
                              : ensure_smem(xline_kernel<df, LOOP, NTH>, smem, &curdf);
  if (e != cudaSuccess) return e;
  const double kxs = 6.283185307179586476925 / g.lx;
  if (prec == 0) {
    xline_kernel<double, LOOP, NTH><<<grid, NTH, smem, s>>>(
        (const double2*)in7, (double2*)out10, g.Mx, g.Px, g.Py, g.nz, fs, g.kappa, scale, kxs,
        px);
  } else if (prec == 1) {
    xline_kernel<float, LOOP, NTH><<<grid, NTH, smem, s>>>(
        (const float2*)in7, (float2*)out10, g.Mx, g.Px, g.Py, g.nz, fs, (float)g.kappa,
        (float)scale, (float)kxs, px);
  } else {
    xline_kernel<df, LOOP, NTH><<<grid, NTH, smem, s>>>(
        (const df2*)in7, (df2*)out10, g.Mx, g.Px, g.Py, g.nz, fs, df(g.kappa), df(scale),
        df(kxs), px);
  }
  return cudaGetLastError();
}

cudaError_t launch_xline(int prec, const GridDev& g, const void* in7, void* out10, long long fs,
                         double scale, const FftPlan& px, cudaStream_t s) {
  const size_t elem = prec == 1 ? sizeof(float2) : sizeof(double2);
  const size_t smem = xline_smem(g.Px, elem);
  // Long x lines, where shared memory limits the CTAs per SM to two (float32) or one (16-byte
  // elements): float32 takes the line-loop passes (more registers, less index work per
  // butterfly: 6.31 -> 5.48 ms at Px = 768), float64 and double-float twice the threads per
  // CTA with the per-butterfly passes (more warps to cover the float64 pipe's latency: 45.9 ->
  // 44.5 ms).  Shorter lines: the per-butterfly passes, 256 threads.
  if (3 * smem > (size_t)kMaxSmemPerSm) {
    if (prec == 1) return launch_xline_t<true, XT>(prec, g, in7, out10, fs, scale, px, smem, s);
    return launch_xline_t<false, 512>(prec, g, in7, out10, fs, scale, px, smem, s);
  }
  return launch_xline_t<false, XT>(prec, g, in7, out10, fs, scale, px, smem, s);
}

size_t adj_xline_smem(int Px) { return (size_t)24 * Px * sizeof(double2); }

cudaError_t launch_adj_xline(const GridDev& g, const double2* in6, const double2* pb9,
                             double2* out6, long long fs, const FftPlan& px, cudaStream_t s) {
  const size_t smem = adj_xline_smem(g.Px);
  dim3 grid((g.nz + 1) / 2, g.Py);
  static SmemLimit cur;
  cudaError_t e = ensure_smem(adj_xline_kernel, smem, &cur);
  if (e != cudaSuccess) return e;
  adj_xline_kernel<<<grid, XT, smem, s>>>(in6, pb9, out6, g.Mx, g.Px, g.Py, g.nz, fs, g.kappa,
                                          6.283185307179586476925 / g.lx, px);
  return cudaGetLastError();
}

cudaError_t launch_x_r2c(const GridDev& g, const double* phys, double2* out, int nf,
                         long long fs_phys, long long fs_spec, const FftPlan& px,
                         cudaStream_t s) {
  dim3 grid((g.nz + 1) / 2, g.ny, nf);
  x_r2c_kernel<<<grid, 128, 2 * g.nx * sizeof(double2), s>>>(phys, out, g.nx, g.ny, g.nz, fs_phys,
                                                             fs_spec, px);
  return cudaGetLastError();
}

cudaError_t launch_x_c2r(const GridDev& g, const double2* in, double* phys, int nf,
                         long long fs_spec, long long fs_phys, const FftPlan& px,
                         cudaStream_t s) {
  dim3 grid((g.nz + 1) / 2, g.ny, nf);
  x_c2r_kernel<<<grid, 128, 2 * g.nx * sizeof(double2), s>>>(in, phys, g.nx, g.ny, g.nz, fs_spec,
                                                             fs_phys, px);
  return cudaGetLastError();
}

}  // namespace chf

namespace chf {

int ytile_for(int P, size_t elem) { return ytile_local(P, elem); }
size_t xline_smem(int Px, size_t elem) { return (size_t)17 * fft_line_stride(Px) * elem; }

cudaError_t launch_grouped_xy(int stage, int prec, const Member* mem, const int* begin, int nmem,
                              int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  static SmemLimit cur[9];
#define GL(K, idx, T_)                                                   \
  if ((e = ensure_smem(K, smem, &cur[idx])) != cudaSuccess) return e;    \
  K<<<grid, (stage == 4 ? XT : YT), smem, s>>>(mem, begin, nmem);
  if (stage == 3) {
    if (prec == 0) { GL((grouped_ypass_kernel<double, true>), 0, double) }
    else if (prec == 1) { GL((grouped_ypass_kernel<float, true>), 1, float) }
    else { GL((grouped_ypass_kernel<df, true>), 6, df) }
  } else if (stage == 4) {
    if (prec == 0) { GL(grouped_xline_kernel<double>, 2, double) }
    else if (prec == 1) { GL(grouped_xline_kernel<float>, 3, float) }
    else { GL(grouped_xline_kernel<df>, 7, df) }
  } else {
    if (prec == 0) { GL(grouped_ycomb_kernel<double>, 4, double) }
    else if (prec == 1) { GL(grouped_ycomb_kernel<float>, 5, float) }
    else { GL(grouped_ycomb_kernel<df>, 8, df) }
  }
#undef GL
  return cudaGetLastError();
}

int occupancy_xy(int stage, int prec, size_t smem) {
  int n = 0;
  const void* k;
  if (stage == 3)
    k = prec == 0 ? (const void*)grouped_ypass_kernel<double, true>
      : prec == 1 ? (const void*)grouped_ypass_kernel<float, true>
                  : (const void*)grouped_ypass_kernel<df, true>;
  else if (stage == 4)
    k = prec == 0 ? (const void*)grouped_xline_kernel<double>
      : prec == 1 ? (const void*)grouped_xline_kernel<float>
                  : (const void*)grouped_xline_kernel<df>;
  else
    k = prec == 0 ? (const void*)grouped_ycomb_kernel<double>
      : prec == 1 ? (const void*)grouped_ycomb_kernel<float>
                  : (const void*)grouped_ycomb_kernel<df>;
  if (smem > 48 * 1024) {  // opt-in first (init time, never during capture)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaGetLastError();
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, stage == 4 ? XT : YT, smem);
  cudaGetLastError();
  return n;
}

}  // namespace chf
