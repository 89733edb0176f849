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
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "ch_internal.h"

namespace chf {

namespace {

constexpr int YT = 256;   // threads of a y-pass CTA
constexpr int XT = 256;   // threads of an x-line CTA

// ---- warp-level FFTs (float32, length P = 32 R, R = 3 Q) -------------------------------------
// One warp transforms one complex line of length P = 32 R with the line in registers: lane l
// holds element l + 32 m in register m (natural layout).  The transform is factored as
// P = R x 32 (Sec. 3.2.1's batched Fourier transforms, written as a two-level Cooley-Tukey
// split): an R-point DFT over the registers of each lane, the twiddles W_P^(l k), and a
// 32-point DFT across the lanes of each register by a radix-2 network of warp shuffles.
//   backward (exp(+i)), natural input:  R-point DFT, twiddles, decimation-in-frequency network
//     -> lane l, register k holds output k + R rev5(l) (rev5: 5-bit reversal);
//   forward (exp(-i)) from that layout:  decimation-in-time network (bit-reversed input,
//     natural output), twiddles, R-point DFT -> lane l, register m holds output l + 32 m.
// So the physical samples stay in the backward transform's permuted order: the products are
// pointwise and the forward transform reads them in that order.  The R-point DFT is split
// R = 3 x Q: radix-3 DFTs over (m, m + Q, m + 2Q), twiddles W_R^(m k), then Q-point DFTs.
// A backward transform of the 3/2-rule padding has zero input in registers Q .. 2Q - 1 (modes
// Mx .. 2 Mx - 1), which its radix-3 DFTs skip.

// R-point DFT of v (R = 3 Q) in registers, natural order in and out, exp(-i) or (INV) exp(+i);
// tw: the length-32R table W_P^t, so W_R^j = tw[32 j]; PRUNE: v[Q .. 2Q - 1] are zero.
template <int Q, bool INV, bool PRUNE>
__device__ __forceinline__ void dft3q(float2 (&v)[3 * Q], const float2* __restrict__ tw) {
  float2 t[3][Q];
  const float s3 = 0.86602540378443864676f;   // sin(2 pi / 3)
  const float sp = INV ? -s3 : s3;
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    const float2 a0 = v[m], a2 = v[m + 2 * Q];
    float2 y0, y1, y2;
    if (PRUNE) {
      // a1 = 0: y0 = a0 + a2, y1,2 = a0 - a2 / 2 -+ i s (-a2)
      const float2 mm = make_float2(fmaf(-0.5f, a2.x, a0.x), fmaf(-0.5f, a2.y, a0.y));
      y0 = a0 + a2;
      y1 = make_float2(fmaf(-sp, a2.y, mm.x), fmaf(sp, a2.x, mm.y));
      y2 = make_float2(fmaf(sp, a2.y, mm.x), fmaf(-sp, a2.x, mm.y));
    } else {
      const float2 a1 = v[m + Q];
      const float2 s = a1 + a2, d = a1 - a2;
      const float2 mm = make_float2(fmaf(-0.5f, s.x, a0.x), fmaf(-0.5f, s.y, a0.y));
      y0 = a0 + s;
      y1 = make_float2(fmaf(sp, d.y, mm.x), fmaf(-sp, d.x, mm.y));
      y2 = make_float2(fmaf(-sp, d.y, mm.x), fmaf(sp, d.x, mm.y));
    }
    t[0][m] = y0;
    if (m == 0) {
      t[1][m] = y1;
      t[2][m] = y2;
    } else {
      const float2 w1 = tw[32 * m], w2 = tw[64 * m];
      t[1][m] = INV ? cmulc(y1, w1) : cmul(y1, w1);
      t[2][m] = INV ? cmulc(y2, w2) : cmul(y2, w2);
    }
  }
#pragma unroll
  for (int k3 = 0; k3 < 3; ++k3) {
    if constexpr (Q > 1) Dft<float, Q, INV>::run(t[k3]);
#pragma unroll
    for (int kq = 0; kq < Q; ++kq) v[k3 + 3 * kq] = t[k3][kq];
  }
}

// 32-point DFT across the lanes of every register.  DIF (natural in, bit-reversed out) for the
// backward transform, DIT (bit-reversed in, natural out) for the forward one; ws[s] is this
// lane's twiddle of the stage with span 16 >> s (DIF) or 1 << s (DIT): W_{2h}^(lane mod h)
// for the lanes whose bit h is set, 1 otherwise (conjugated by the caller for INV).
template <int R>
__device__ __forceinline__ void lanes_dif(float2 (&v)[R], const float2 (&ws)[5], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int h = 16 >> s;
    const bool up = (lane & h) != 0;
    const float sg = up ? -1.0f : 1.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const float px = __shfl_xor_sync(0xffffffffu, v[k].x, h);
      const float py = __shfl_xor_sync(0xffffffffu, v[k].y, h);
      const float2 d = make_float2(fmaf(sg, v[k].x, px), fmaf(sg, v[k].y, py));
      v[k] = (s < 4) ? cmul(d, ws[s]) : d;
    }
  }
}
template <int R>
__device__ __forceinline__ void lanes_dit(float2 (&v)[R], const float2 (&ws)[5], int lane) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int h = 1 << s;
    const bool up = (lane & h) != 0;
    const float sg = up ? -1.0f : 1.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const float2 x = (s > 0) ? cmul(v[k], ws[s]) : v[k];
      const float px = __shfl_xor_sync(0xffffffffu, x.x, h);
      const float py = __shfl_xor_sync(0xffffffffu, x.y, h);
      v[k] = make_float2(fmaf(sg, x.x, px), fmaf(sg, x.y, py));
    }
  }
}

// In-place float32 FFT of one line of P = 32 R points in shared memory by one warp (natural
// order in and out): the R-point DFTs, twiddles W_P^(-+ l k) and the DIF lane network, the result
// written back through the register-order index k 32 + l and read by warp_line_at.  PRUNE: the
// line's middle third (positions 32 Q .. 64 Q - 1) is zero and not read.
template <int Q, bool INV, bool PRUNE>
__device__ __forceinline__ void warp_fft_line(float2* __restrict__ line,
                                              const float2* __restrict__ tw, int lane) {
  constexpr int R = 3 * Q;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m)
    v[m] = (PRUNE && m >= Q && m < 2 * Q) ? make_float2(0.0f, 0.0f) : line[lane + 32 * m];
  __syncwarp();
  dft3q<Q, INV, PRUNE>(v, tw);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = INV ? cmulc(v[k], tw[k * lane]) : cmul(v[k], tw[k * lane]);
  float2 ws[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int h = 16 >> s;
    ws[s] = (lane & h) ? tw[(lane & (h - 1)) * (16 * R / h)] : make_float2(1.0f, 0.0f);
    if (INV) ws[s].y = -ws[s].y;
  }
  lanes_dif<R>(v, ws, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) line[k * 32 + lane] = v[k];
  __syncwarp();
}
// shared-memory index of output position p of warp_fft_line (p = k + R rev5(l) sits at k 32 + l)
template <int Q>
__device__ __forceinline__ int warp_line_at(int p) {
  constexpr int R = 3 * Q;
  const int j = p / R;
  return (p - j * R) * 32 + (int)(__brev((unsigned)j) >> 27);
}

// Every line of a shared-memory tile (nlines lines of stride ls) through warp_fft_line, the warps
// of the CTA taking lines in turn; q = P / 96 (QM: the only q when EXACT, else the largest q
// the switch covers).  mid_zero: the lines' middle thirds are zero (a backward transform of the
// 3/2-rule padding) and are not read.
template <bool INV, int QM, bool EXACT>
__device__ __forceinline__ void warp_lines(float2* A, int nlines, int ls, int q,
                                           const float2* __restrict__ tw, bool mid_zero) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int ln = warp; ln < nlines; ln += nw) {
    float2* L = A + ln * ls;
    if constexpr (EXACT) {
      mid_zero ? warp_fft_line<QM, INV, true>(L, tw, lane)
               : warp_fft_line<QM, INV, false>(L, tw, lane);
    } else {
      if (q == 1) {
        mid_zero ? warp_fft_line<1, INV, true>(L, tw, lane) : warp_fft_line<1, INV, false>(L, tw, lane);
      } else if (q == 2) {
        mid_zero ? warp_fft_line<2, INV, true>(L, tw, lane) : warp_fft_line<2, INV, false>(L, tw, lane);
      } else if constexpr (QM >= 4) {
        if (q == 4) {
          mid_zero ? warp_fft_line<4, INV, true>(L, tw, lane) : warp_fft_line<4, INV, false>(L, tw, lane);
        } else if constexpr (QM >= 8) {
          mid_zero ? warp_fft_line<8, INV, true>(L, tw, lane) : warp_fft_line<8, INV, false>(L, tw, lane);
        }
      }
    }
  }
  __syncthreads();
}
// y transform of nl lines of a tile, in place (warp path, float32) or through the block passes
// into A or B; returns the result buffer, *wq = the warp path's q (0: block passes).  WQ > 0:
// the warp path with q = WQ only; WQ < 0: the warp path for q <= -WQ, else the block passes;
// WQ = 0: the block passes.
template <typename T, bool INV, int WQ>
__device__ __forceinline__ const typename C2<T>::t* y_transform(typename C2<T>::t* A,
                                                                typename C2<T>::t* B, int nl,
                                                                int LS, int P, bool mid_zero,
                                                                const FftPlan& pl, int* wq) {
  if constexpr (std::is_same<T, float>::value && WQ != 0) {
    const int q = WQ > 0 ? WQ : warp_fft_q(P);
    if (WQ > 0 || (q != 0 && q <= -WQ)) {
      warp_lines<INV, (WQ > 0 ? WQ : -WQ), (WQ > 0)>(A, nl, LS, q,
                                                     reinterpret_cast<const float2*>(pl.tw),
                                                     mid_zero);
      *wq = q;
      return A;
    }
  }
  *wq = 0;
  if constexpr (WQ > 0) {
    return A;   // not reached: the exact warp path always applies
  } else {
    return block_fft<T, INV, true>(A, B, nl, LS, pl, true);
  }
}
// shared-memory index of position p of a line transformed by warp_fft_line (R = 3 q; inv_r =
// 1 / R as a float)
__device__ __forceinline__ int warp_pos(int p, int R, float inv_r) {
  int k;
  const int j = fdivmod(p, R, inv_r, &k);
  return k * 32 + (int)(__brev((unsigned)j) >> 27);
}

// y pass: one CTA per (z tile, mx, field).
//   INV (backward): in (Mx, Ny, Nz) modes -> out (Mx, P, Nz) samples, modes |my| < Ny/2 placed,
//   the rest zero.  Forward: in (Mx, P, Nz) samples -> out (Mx, Ny, Nz) kept modes * scale.
template <typename T, bool INV, int WQ>
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
  // float32 lines of 96 q points: one warp per line in registers (warp_fft_line), the result
  // in the register order that warp_pos maps; otherwise the block-cooperative passes
  int wq;
  const T2* R = y_transform<T, INV, WQ>(A, B, TZ, LS, P, INV && 2 * P == 3 * Ny, pl, &wq);
  const int wr = 3 * wq;
  const float inv_wr = wq ? 1.0f / (float)wr : 0.0f;
  if (INV) {
    T2* dst = out + f * fs_out + (size_t)mx * P * Nz;
    for (int idx = threadIdx.x; idx < P * TZ; idx += blockDim.x) {
      const int y = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      if (z < Nz) dst[(size_t)y * Nz + z] = R[zz * LS + (wq ? warp_pos(y, wr, inv_wr) : y)];
    }
  } else {
    T2* dst = out + f * fs_out + (size_t)mx * Ny * Nz;
    for (int idx = threadIdx.x; idx < Ny * TZ; idx += blockDim.x) {
      const int jj = idx >> tzs, zz = idx & (TZ - 1);
      const int z = z0 + zz;
      if (z >= Nz) continue;
      const int p = (jj < h) ? jj : P - Ny + jj;
      dst[(size_t)jj * Nz + z] =
          (jj == h) ? zero : scale * R[zz * LS + (wq ? warp_pos(p, wr, inv_wr) : p)];
    }
  }
}

template <typename T, bool INV, int WQ>
__global__ void __launch_bounds__(YT, (WQ >= 1 && WQ <= 4) ? 4 : 1) ypass_kernel(const typename C2<T>::t* __restrict__ in,
                                                   typename C2<T>::t* __restrict__ out, int Mx,
                                                   int Ny, int P, int Nz, int TZ, long long fs_in,
                                                   long long fs_out, T scale, FftPlan pl,
                                                   YMap map) {
  ypass_body<T, INV, WQ>(in, out, Mx, Ny, P, Nz, TZ, fs_in, fs_out, scale, pl, map, blockIdx.x,
                         blockIdx.y, blockIdx.z);
}

// Forward y pass with the assembly's combinations (launch_ycomb): work item -> (group, mx, z
// tile); the nine products are transformed in groups so that each CTA holds every input its
// outputs combine.  Groups and outputs as stated at launch_ycomb; the arithmetic of the
// combinations is that of the working precision T.
template <typename T, int WQ>
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
  int wq;
  const T2* R = y_transform<T, false, WQ>(A, B, nin * TZ, LS, P, false, pl, &wq);
  const int wr = 3 * wq;
  const float inv_wr = wq ? 1.0f / (float)wr : 0.0f;
  const int h = Ny / 2;
  const T kx = kxs * (T)mx;
  T2* dst = out + (size_t)mx * Ny * Nz;
  for (int idx = threadIdx.x; idx < Ny * TZ; idx += blockDim.x) {
    const int jj = idx >> tzs, zz = idx & (TZ - 1);
    const int z = z0 + zz;
    if (z >= Nz) continue;
    const size_t o = (size_t)jj * Nz + z;
    const int p0 = (jj < h) ? jj : P - Ny + jj;
    const int p = wq ? warp_pos(p0, wr, inv_wr) : p0;
    const bool nyq = (jj == h);   // the y Nyquist row is zero
    const bool mean = (mx == 0 && jj == 0);
    const T ky = kys * (T)((jj < h) ? jj : jj - Ny);
    T2 v[3];
#pragma unroll
    for (int f = 0; f < 3; ++f)
      v[f] = (nyq || f >= nin) ? zero : scale * R[(f * TZ + zz) * LS + p];
    // ca x + cb y with explicit fused multiply-adds (the single-grid and grouped kernels round
    // alike)
    auto lin = [](T ca, T2 x, T cb, T2 y) {
      return mk(fmx(ca, x.x, cb * y.x), fmx(ca, x.y, cb * y.y));
    };
    if (grp == 0) {
      const T2 a = mul_i(lin(kx, v[0], ky, v[2]));
      const T2 b = mul_i(lin(kx, v[2], ky, v[1]));
      if (!mean) dst[o] = mul_i(lin(kx, b, -ky, a));
      dst[3 * fs_out + o] = mul_i(lin(kx, a, ky, b));
    } else if (grp == 1) {
      if (mean) {
        dst[o] = v[0];
        dst[fs_out + o] = v[1];
      } else {
        dst[fs_out + o] = mul_i(lin(kx, v[1], -ky, v[0]));
      }
      dst[2 * fs_out + o] = mul_i(lin(kx, v[0], ky, v[1]));
    } else if (grp == 2) {
      dst[4 * fs_out + o] = mul_mi(lin(kx, v[0], ky, v[1]));
    } else {
      dst[(grp == 3 ? 5 : 6) * fs_out + o] = v[0];
    }
  }
}

template <typename T, int WQ>
__global__ void __launch_bounds__(YT, (WQ >= 1 && WQ <= 4) ? 4 : 1) ycomb_kernel(const typename C2<T>::t* __restrict__ in,
                                                   typename C2<T>::t* __restrict__ out, int Mx,
                                                   int Ny, int P, int Nz, int L, long long fs_in,
                                                   long long fs_out, T scale, T kxs, T kys,
                                                   FftPlan pl) {
  ycomb_body<T, WQ>(in, out, Mx, Ny, P, Nz, L, fs_in, fs_out, scale, kxs, kys, pl, blockIdx.x);
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

// Fused x line on warp FFTs, one item = (pair of z rows, y) as in xline_body.  A backward line
// takes input line f (u v w phi phi_x phi_y phi_z) of an item to physical space in the backward
// transform's order (shared memory, P float2, index k * 32 + lane); a forward line forms product
// g (of nine) in registers from the seven samples, transforms it forward and stores its kept
// modes.  One warp does each line.  The twiddles W_P^(l k) sit in shared memory as [k][l]
// (R x 32 float2).
constexpr int XWT = 256;
template <int Q>
__device__ __forceinline__ void xw_backward(const float2* __restrict__ in, float2* __restrict__ phys,
                                            int f, int Mx, size_t base, size_t mstride, bool two,
                                            long long fs, float kxs,
                                            const float2* __restrict__ tw,
                                            const float2* __restrict__ twl, int lane) {
  constexpr int R = 3 * Q, P = 32 * R;
  // the lane-stage twiddles W_{2h}^j = W_P^(j 16 R / h), conjugated (backward: exp(+i))
  float2 wdif[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int hf = 16 >> s;
    wdif[s] = (lane & hf) ? tw[(lane & (hf - 1)) * (16 * R / hf)] : make_float2(1.0f, 0.0f);
    wdif[s].y = -wdif[s].y;
  }
  const int src_f = (f < 4) ? f : f - 1;      // phi_x (line 4) comes from phi (input 3)
  const float2* src = in + src_f * fs + base;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    v[m] = make_float2(0.0f, 0.0f);
    if (m >= Q && m < 2 * Q) continue;         // modes Mx .. 2 Mx - 1: zero padding
    const int n = lane + 32 * m;
    const int q = (m < Q) ? n : P - n;         // mode index (the upper third: negative modes)
    if (q >= Mx) continue;                     // mode Mx (x Nyquist) is not kept
    const float2* pq = src + (size_t)q * mstride;
    float2 a, b;
    if (two && (reinterpret_cast<uintptr_t>(pq) & 15) == 0) {   // the pair in one 16-byte load
      const float4 ab = *reinterpret_cast<const float4*>(pq);
      a = make_float2(ab.x, ab.y);
      b = make_float2(ab.z, ab.w);
    } else {
      a = pq[0];
      b = two ? pq[1] : make_float2(0.0f, 0.0f);
    }
    if (f == 4) {                              // i kx phi
      const float kx = kxs * (float)q;
      a = make_float2(-kx * a.y, kx * a.x);
      b = make_float2(-kx * b.y, kx * b.x);
    }
    if (n == 0) v[m] = make_float2(a.x, b.x);  // the imaginary part of a DC coefficient is not used
    else if (m < Q) v[m] = make_float2(a.x - b.y, a.y + b.x);   // a + i b
    else v[m] = make_float2(a.x + b.y, b.x - a.y);              // conj(a) + i conj(b)
  }
  dft3q<Q, true, true>(v, tw);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], twl[k * 32 + lane]);
  lanes_dif<R>(v, wdif, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) phys[(f * R + k) * 32 + lane] = v[k];
}

// product g (rows z0 in .x, z0+1 in .y) of the seven samples in `phys`, forward transform, kept
// modes to `out`
template <int Q>
__device__ __forceinline__ void xw_forward(const float2* __restrict__ phys, float2* __restrict__ out,
                                           int g, int Mx, size_t base, size_t mstride, bool two,
                                           long long fs, float kappa, float scale,
                                           const float2* __restrict__ tw,
                                           const float2* __restrict__ twl, int lane) {
  constexpr int R = 3 * Q;
  float2 wdit[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int ht = 1 << s;
    wdit[s] = (lane & ht) ? tw[(lane & (ht - 1)) * (16 * R / ht)] : make_float2(1.0f, 0.0f);
  }
  const float hs = 0.5f * scale;
  float2 v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = k * 32 + lane;
    const float2 u = phys[i], vv = phys[R * 32 + i], w = phys[2 * R * 32 + i];
    const float2 ph = phys[3 * R * 32 + i], fx = phys[4 * R * 32 + i];
    const float2 fy = phys[5 * R * 32 + i], fz = phys[6 * R * 32 + i];
    // explicit fused multiply-adds: the single-grid and grouped kernels round alike
    float2 r;
    switch (g) {
      case 0:
        r.x = fmaf(kappa * fz.x, fz.x, w.x * w.x) - fmaf(kappa * fx.x, fx.x, u.x * u.x);
        r.y = fmaf(kappa * fz.y, fz.y, w.y * w.y) - fmaf(kappa * fx.y, fx.y, u.y * u.y);
        break;
      case 1:
        r.x = fmaf(kappa * fz.x, fz.x, w.x * w.x) - fmaf(kappa * fy.x, fy.x, vv.x * vv.x);
        r.y = fmaf(kappa * fz.y, fz.y, w.y * w.y) - fmaf(kappa * fy.y, fy.y, vv.y * vv.y);
        break;
      case 2:
        r = make_float2(-fmaf(kappa * fx.x, fy.x, u.x * vv.x), -fmaf(kappa * fx.y, fy.y, u.y * vv.y));
        break;
      case 3:
        r = make_float2(-fmaf(kappa * fx.x, fz.x, u.x * w.x), -fmaf(kappa * fx.y, fz.y, u.y * w.y));
        break;
      case 4:
        r = make_float2(-fmaf(kappa * fy.x, fz.x, vv.x * w.x), -fmaf(kappa * fy.y, fz.y, vv.y * w.y));
        break;
      case 5: r = make_float2(ph.x * ph.x * ph.x, ph.y * ph.y * ph.y); break;
      case 6: r = make_float2(u.x * ph.x, u.y * ph.y); break;
      case 7: r = make_float2(vv.x * ph.x, vv.y * ph.y); break;
      default: r = make_float2(w.x * ph.x, w.y * ph.y); break;
    }
    v[k] = r;
  }
  lanes_dit<R>(v, wdit, lane);
#pragma unroll
  for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twl[k * 32 + lane]);
  dft3q<Q, false, false>(v, tw);
  // unpack the two real rows: A_k = (Z_k + conj Z_{P-k}) / 2, B_k = (Z_k - conj Z_{P-k}) / (2 i)
  // for the kept modes k = lane + 32 m < Mx (m < Q); Z_{P-k} sits in lane -k mod 32, register
  // R - 1 - m (lane 0: its own register R - m)
  float2* dst = out + g * fs + base;
#pragma unroll
  for (int m = 0; m < Q; ++m) {
    const float2 o = v[R - 1 - m];
    const int pl = (32 - lane) & 31;
    float2 Zm = make_float2(__shfl_sync(0xffffffffu, o.x, pl), __shfl_sync(0xffffffffu, o.y, pl));
    if (lane == 0) Zm = (m == 0) ? v[0] : v[(R - m) % R];
    const float2 Zk = v[m];
    const int k = lane + 32 * m;
    if (k < Mx) {
      float2* d = dst + (size_t)k * mstride;
      const float2 A = make_float2(hs * (Zk.x + Zm.x), hs * (Zk.y - Zm.y));
      const float2 B = make_float2(hs * (Zk.y + Zm.y), hs * (Zm.x - Zk.x));
      if (two && (reinterpret_cast<uintptr_t>(d) & 15) == 0) {
        *reinterpret_cast<float4*>(d) = make_float4(A.x, A.y, B.x, B.y);
      } else {
        d[0] = A;
        if (two) d[1] = B;
      }
    }
  }
}

// Item j of row y: the z rows it packs.  Rows pair so that the pair's offset y Nz + z0 is even
// (16-byte aligned pairs when the field's base is): where y Nz is odd, row 0 stands alone and
// the pairs are (1, 2), (3, 4), ...; otherwise (0, 1), (2, 3), ...  Either way (Nz + 1) / 2
// items per y.
__device__ __forceinline__ void xw_item(int j, int y, int Nz, int* z0, bool* two) {
  if (((long long)y * Nz & 1) == 0) {
    *z0 = 2 * j;
    *two = 2 * j + 1 < Nz;
  } else {
    *z0 = j == 0 ? 0 : 2 * j - 1;
    *two = j > 0 && 2 * j < Nz;
  }
}

// One item (z rows of item bx at y = by) with 8 warps: warps 0..6 the backward lines, then
// each warp a product line (9 over the 8 warps).  Shared memory: seven lines of P float2 and the
// twiddle table.
template <int Q>
__device__ __forceinline__ void xline_warp_body(const float2* __restrict__ in,
                                                float2* __restrict__ out, int Mx, int Py, int Nz,
                                                long long fs, float kappa, float scale, float kxs,
                                                const float2* __restrict__ tw, int bx, int by) {
  constexpr int R = 3 * Q, P = 32 * R;
  extern __shared__ float2 xw_sm[];
  float2* phys = xw_sm;
  float2* twl = xw_sm + 7 * P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int z0;
  bool two;
  xw_item(bx, by, Nz, &z0, &two);
  const size_t base = (size_t)by * Nz + z0;
  const size_t mstride = (size_t)Py * Nz;
  for (int i = threadIdx.x; i < R * 32; i += blockDim.x) {
    const int k = i >> 5, l = i & 31;
    twl[i] = tw[k * l];                 // k l < P
  }
  __syncthreads();
  if (warp < 7) xw_backward<Q>(in, phys, warp, Mx, base, mstride, two, fs, kxs, tw, twl, lane);
  __syncthreads();
  for (int g = warp; g < 9; g += 8)
    xw_forward<Q>(phys, out, g, Mx, base, mstride, two, fs, kappa, scale, tw, twl, lane);
}

// v through an opaque move that is also a compiler memory barrier: nothing derived from the
// result is computed, and no memory access is moved, across it
__device__ __forceinline__ int opaque_int(int v) {
  int r;
  asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v) : "memory");
  return r;
}

// Persistent x line: each CTA walks the items t = blockIdx.x, + gridDim.x, ... (z pair fastest)
// with two buffers of seven lines.  A round holds 16 line tasks, two per warp: the nine forward
// lines of item t (warp w line w, warp 7 also line 8) and the seven backward lines of the next
// item (warps 0..6) into the other buffer, so no warp idles and the next item's loads overlap
// the products' transforms; one barrier per round.  Round-robin keeps the items in flight on
// all CTAs neighbours in memory (contiguous runs per CTA spread them over the whole field and
// ran at half the speed), at the price of some sectors whose two halves, read by neighbouring
// items on CTAs that have drifted apart, come from DRAM twice.  Per line the same arithmetic
// as xline_warp_body.
template <int Q>
__global__ void __launch_bounds__(XWT, Q >= 8 ? 2 : 3)
    xline_warp_kernel(const float2* __restrict__ in, float2* __restrict__ out, int Mx, int Py,
                      int Nz, long long fs, float kappa, float scale, float kxs,
                      const float2* __restrict__ tw0) {
  constexpr int R = 3 * Q, P = 32 * R;
  extern __shared__ float2 xp_sm[];
  float2* twl = xp_sm + 14 * P;
  const int lane0 = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nzp = (Nz + 1) / 2, nitems = nzp * Py;
  const size_t mstride = (size_t)Py * Nz;
  for (int i = threadIdx.x; i < R * 32; i += blockDim.x) {
    const int k = i >> 5, l = i & 31;
    twl[i] = tw0[k * l];
  }
  __syncthreads();
  int t = blockIdx.x;
  if (t >= nitems) return;
  if (warp < 7) {
    int z0;
    bool two;
    xw_item(t % nzp, t / nzp, Nz, &z0, &two);
    xw_backward<Q>(in, xp_sm, warp, Mx, (size_t)(t / nzp) * Nz + z0, mstride, two, fs, kxs,
                   tw0, twl, lane0);
  }
  __syncthreads();
  int b = 0;
#pragma unroll 1
  for (; t < nitems; t += gridDim.x) {
    // the lane index passes through an opaque move before each line, so the compiler neither
    // holds a line's mode offsets and twiddles across the loop nor starts the next line's loads
    // inside the previous one (either would double the registers of a line)
    const int lane = opaque_int(lane0);
    const float2* cur = xp_sm + b * 7 * P;
    float2* nxt = xp_sm + (b ^ 1) * 7 * P;
    int z0;
    bool two;
    xw_item(t % nzp, t / nzp, Nz, &z0, &two);
    const size_t base = (size_t)(t / nzp) * Nz + z0;
    xw_forward<Q>(cur, out, warp, Mx, base, mstride, two, fs, kappa, scale, tw0, twl, lane);
    const int tn = t + gridDim.x;
    __syncwarp();   // ptxas moves no memory access across it: the next line's loads start here
    const int lane2 = opaque_int(lane0);
    if (warp == 7) {
      xw_forward<Q>(cur, out, 8, Mx, base, mstride, two, fs, kappa, scale, tw0, twl, lane2);
    } else if (tn < nitems) {
      int zn;
      bool twon;
      xw_item(tn % nzp, tn / nzp, Nz, &zn, &twon);
      xw_backward<Q>(in, nxt, warp, Mx, (size_t)(tn / nzp) * Nz + zn, mstride, twon, fs, kxs,
                     tw0, twl, lane2);
    }
    __syncthreads();
    b ^= 1;
  }
}
// shared memory of the persistent warp-FFT x line: two buffers of seven lines and the twiddles
__host__ __device__ __forceinline__ size_t xline_warp_smem(int Px) {
  return (size_t)15 * Px * sizeof(float2);
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

// GQ: the largest warp-FFT q among the members (0, 2 or 8; float32), the same path per member as
// the single-grid launch takes
template <typename T, bool INV, int GQ>
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
      ypass_body<T, true, -GQ>((const T2*)M.bw, (T2*)M.ya, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, TZ,
                               M.fs, M.fsy, (T)1, M.py, M.ym, bx, by, bz);
    else
      ypass_body<T, false, -GQ>((const T2*)M.yb, (T2*)M.nl, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, TZ,
                                M.fsy, M.fs, (T)M.yscale, M.py, M.yf, bx, by, bz);
    __syncthreads();
  }
}

// grouped forward y pass with the combinations: items (group, mx, z tile) member by member
template <typename T, int GQ>
__global__ void __launch_bounds__(YT) grouped_ycomb_kernel(const Member* __restrict__ mem,
                                                           const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of_xy(begin, nmem, item);
    const Member& M = mem[m];
    ycomb_body<T, -GQ>((const T2*)M.yb, (T2*)M.nl, M.g.Mx, M.g.ny, M.g.Py, M.g.nz, M.tzf,
                       M.fsy, M.fs, (T)M.yscale, (T)M.kxs, (T)M.ym.kys, M.py, item - begin[m]);
    __syncthreads();
  }
}

// GQ: as in grouped_ypass_kernel, for the members' padded x lengths (float32 lines of 96 q
// points take the warp-FFT body, as the single-grid launch does)
template <typename T, int GQ>
__global__ void __launch_bounds__(XT, GQ >= 8 ? 2 : 3) grouped_xline_kernel(const Member* __restrict__ mem,
                                                           const int* __restrict__ begin, int nmem) {
  typedef typename C2<T>::t T2;
  const int total = begin[nmem];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int m = member_of_xy(begin, nmem, item);
    const Member& M = mem[m];
    const int nzp = (M.g.nz + 1) / 2;
    const int local = item - begin[m];
    const int bx = local % nzp, by = local / nzp;
    bool done = false;
    if constexpr (std::is_same<T, float>::value && GQ > 0) {
      const int q = (M.px.n == M.g.Px) ? warp_fft_q(M.g.Px) : 0;
      const float2* tw = (const float2*)M.px.tw;
      if (q == 1) {
        xline_warp_body<1>((const float2*)M.ya, (float2*)M.yb, M.g.Mx, M.g.Py, M.g.nz, M.fsy,
                           (float)M.g.kappa, 1.0f, (float)M.kxs, tw, bx, by);
        done = true;
      } else if (q == 2) {
        xline_warp_body<2>((const float2*)M.ya, (float2*)M.yb, M.g.Mx, M.g.Py, M.g.nz, M.fsy,
                           (float)M.g.kappa, 1.0f, (float)M.kxs, tw, bx, by);
        done = true;
      } else if constexpr (GQ >= 8) {
        if (q == 4) {
          xline_warp_body<4>((const float2*)M.ya, (float2*)M.yb, M.g.Mx, M.g.Py, M.g.nz, M.fsy,
                             (float)M.g.kappa, 1.0f, (float)M.kxs, tw, bx, by);
          done = true;
        } else if (q == 8) {
          xline_warp_body<8>((const float2*)M.ya, (float2*)M.yb, M.g.Mx, M.g.Py, M.g.nz, M.fsy,
                             (float)M.g.kappa, 1.0f, (float)M.kxs, tw, bx, by);
          done = true;
        }
      }
    }
    if (!done)
      xline_body<T>((const T2*)M.ya, (T2*)M.yb, M.g.Mx, M.g.Px, M.g.Py, M.g.nz, M.fsy,
                    (T)M.g.kappa, (T)1, (T)M.kxs, M.px, bx, by);
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
  // float32 lines of 96 q points take the warp-FFT kernels (one instantiation per q)
  const int wq = prec == 1 ? warp_fft_q(P) : 0;
  static SmemLimit cur[6][5];
  const int ci = wq == 0 ? 0 : wq == 1 ? 1 : wq == 2 ? 2 : wq == 4 ? 3 : 4;
  cudaError_t e = cudaSuccess;
#define YL(T, INV, Q, K)                                                                       \
  {                                                                                            \
    if ((e = ensure_smem(ypass_kernel<T, INV, Q>, smem, &cur[K][ci])) != cudaSuccess) return e;  \
    ypass_kernel<T, INV, Q><<<grid, YT, smem, s>>>((const C2<T>::t*)in, (C2<T>::t*)out, g.Mx,   \
                                                   g.ny, P, g.nz, TZ, fs_in, fs_out, T(scale),  \
                                                   py, map);                                    \
  }
#define YLF(INV, K)                                       \
  switch (wq) {                                           \
    case 1: YL(float, INV, 1, K) break;                   \
    case 2: YL(float, INV, 2, K) break;                   \
    case 4: YL(float, INV, 4, K) break;                   \
    case 8: YL(float, INV, 8, K) break;                   \
    default: YL(float, INV, 0, K) break;                  \
  }
  if (prec == 0) {
    if (dir == 1) YL(double, true, 0, 0) else YL(double, false, 0, 1)
  } else if (prec == 1) {
    if (dir == 1) { YLF(true, 2) } else { YLF(false, 3) }
  } else {
    if (dir == 1) YL(df, true, 0, 4) else YL(df, false, 0, 5)
  }
#undef YLF
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_ycomb(int prec, const GridDev& g, const void* in, void* out, long long fs_in,
                         long long fs_out, double scale, const FftPlan& py, cudaStream_t s) {
  const size_t elem = prec == 1 ? sizeof(float2) : sizeof(double2);
  const int L = ytile_local(g.Py, elem);
  const size_t smem = ycomb_smem(g.Py, L, elem);
  const int items = ycomb_items(g.Mx, g.nz, L);
  const int wq = prec == 1 ? warp_fft_q(g.Py) : 0;
  static SmemLimit cur[7];
  cudaError_t e = cudaSuccess;
  const double kxs = 6.283185307179586476925 / g.lx, kys = 6.283185307179586476925 / g.ly;
#define YC(T, Q, K, ...)                                                                      \
  {                                                                                           \
    if ((e = ensure_smem(ycomb_kernel<T, Q>, smem, &cur[K])) != cudaSuccess) return e;         \
    ycomb_kernel<T, Q><<<items, YT, smem, s>>>((const C2<T>::t*)in, (C2<T>::t*)out, g.Mx, g.ny, \
                                               g.Py, g.nz, L, fs_in, fs_out, __VA_ARGS__, py);  \
  }
  if (prec == 0) {
    YC(double, 0, 0, scale, kxs, kys)
  } else if (prec == 1) {
    const float a = (float)scale, b = (float)kxs, c = (float)kys;
    switch (wq) {
      case 1: YC(float, 1, 1, a, b, c) break;
      case 2: YC(float, 2, 2, a, b, c) break;
      case 4: YC(float, 4, 3, a, b, c) break;
      case 8: YC(float, 8, 4, a, b, c) break;
      default: YC(float, 0, 5, a, b, c) break;
    }
  } else {
    YC(df, 0, 6, df(scale), df(kxs), df(kys))
  }
#undef YC
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

template <int Q>
cudaError_t launch_xline_warp(const GridDev& g, const void* in7, void* out10, long long fs,
                              double scale, const FftPlan& px, cudaStream_t s) {
  const size_t smem = xline_warp_smem(g.Px);
  static SmemLimit cur;
  static SmemLimit ctas;   // persistent grid per device: SMs x resident CTAs
  cudaError_t e = ensure_smem(xline_warp_kernel<Q>, smem, &cur);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nct = (dev >= 0 && dev < kMaxSmemDevices) ? ctas.v[dev].load(std::memory_order_acquire) : 0;
  if (nct <= 0) {
    int nsm = 0, per = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, xline_warp_kernel<Q>, XWT, smem);
    if (e != cudaSuccess) return e;
    nct = std::max(1, nsm * per);
    if (dev >= 0 && dev < kMaxSmemDevices) ctas.v[dev].store(nct, std::memory_order_release);
  }
  const long long items = (long long)((g.nz + 1) / 2) * g.Py;
  if (items == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(items, nct);
  xline_warp_kernel<Q><<<grid, XWT, smem, s>>>((const float2*)in7, (float2*)out10, g.Mx, g.Py,
                                               g.nz, fs, (float)g.kappa, (float)scale,
                                               (float)(6.283185307179586476925 / g.lx),
                                               (const float2*)px.tw);
  return cudaGetLastError();
}

cudaError_t launch_xline(int prec, const GridDev& g, const void* in7, void* out10, long long fs,
                         double scale, const FftPlan& px, cudaStream_t s) {
  // float32 lines of 96, 192, 384 or 768 points: the warp-FFT kernel
  if (prec == 1 && g.Px % 96 == 0 && px.n == g.Px) {
    switch (g.Px / 96) {
      case 1: return launch_xline_warp<1>(g, in7, out10, fs, scale, px, s);
      case 2: return launch_xline_warp<2>(g, in7, out10, fs, scale, px, s);
      case 4: return launch_xline_warp<4>(g, in7, out10, fs, scale, px, s);
      case 8: return launch_xline_warp<8>(g, in7, out10, fs, scale, px, s);
      default: break;
    }
  }
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

// the grouped y-pass kernel of a stage (3 backward, 5 forward), precision and member warp-FFT
// level ywq (0, 2 or 8)
static const void* grouped_y_kernel(int stage, int prec, int ywq) {
  if (stage == 3) {
    if (prec == 0) return (const void*)grouped_ypass_kernel<double, true, 0>;
    if (prec == 2) return (const void*)grouped_ypass_kernel<df, true, 0>;
    return ywq == 0 ? (const void*)grouped_ypass_kernel<float, true, 0>
         : ywq == 2 ? (const void*)grouped_ypass_kernel<float, true, 2>
                    : (const void*)grouped_ypass_kernel<float, true, 8>;
  }
  if (prec == 0) return (const void*)grouped_ycomb_kernel<double, 0>;
  if (prec == 2) return (const void*)grouped_ycomb_kernel<df, 0>;
  return ywq == 0 ? (const void*)grouped_ycomb_kernel<float, 0>
       : ywq == 2 ? (const void*)grouped_ycomb_kernel<float, 2>
                  : (const void*)grouped_ycomb_kernel<float, 8>;
}

cudaError_t launch_grouped_xy(int stage, int prec, const Member* mem, const int* begin, int nmem,
                              int grid, size_t smem, int ywq, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  static SmemLimit cur[5];
  static SmemLimit cury[2][3][3];
  if (stage == 4) {
#define GL(K, idx)                                                     \
  if ((e = ensure_smem(K, smem, &cur[idx])) != cudaSuccess) return e;  \
  K<<<grid, XT, smem, s>>>(mem, begin, nmem);
    if (prec == 0) { GL((grouped_xline_kernel<double, 0>), 0) }
    else if (prec == 1) {
      if (ywq == 0) { GL((grouped_xline_kernel<float, 0>), 1) }
      else if (ywq == 2) { GL((grouped_xline_kernel<float, 2>), 3) }
      else { GL((grouped_xline_kernel<float, 8>), 4) }
    } else { GL((grouped_xline_kernel<df, 0>), 2) }
#undef GL
    return cudaGetLastError();
  }
  const void* k = grouped_y_kernel(stage, prec, ywq);
  const int wi = ywq == 0 ? 0 : ywq == 2 ? 1 : 2;
  if ((e = ensure_smem(k, smem, &cury[stage == 3 ? 0 : 1][prec][wi])) != cudaSuccess) return e;
  void* args[] = {(void*)&mem, (void*)&begin, (void*)&nmem};
  e = cudaLaunchKernel(k, dim3(grid), dim3(YT), args, smem, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  return cudaSuccess;
}

int occupancy_xy(int stage, int prec, size_t smem, int ywq) {
  int n = 0;
  const void* k;
  if (stage == 4)
    k = prec == 0 ? (const void*)grouped_xline_kernel<double, 0>
      : prec == 2 ? (const void*)grouped_xline_kernel<df, 0>
      : ywq == 0  ? (const void*)grouped_xline_kernel<float, 0>
      : ywq == 2  ? (const void*)grouped_xline_kernel<float, 2>
                  : (const void*)grouped_xline_kernel<float, 8>;
  else
    k = grouped_y_kernel(stage, prec, ywq);
  if (smem > 48 * 1024) {  // opt-in first (init time, never during capture)
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaGetLastError();
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, stage == 4 ? XT : YT, smem);
  cudaGetLastError();
  return n;
}

}  // namespace chf
