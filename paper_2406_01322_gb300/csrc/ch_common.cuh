// Device-side building blocks shared by the solver kernels: complex helpers, radix-2/3/4/8
// butterflies and a block-cooperative Stockham FFT over lines held in shared memory.
//
// The transforms are those of Sec. 3.2.1 of the paper (batched Fourier transforms in x and y,
// the Chebyshev transform as a DCT-I computed through a 2N-point FFT of the even extension),
// written here as hand-rolled mixed-radix Stockham passes instead of library calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace chf {

// ---------------------------------------------------------------------------------------------
// complex helpers (double2 / float2)
template <typename T> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// i * a and -i * a
template <typename T2> __device__ __forceinline__ T2 mul_i(T2 a) { return mk(-a.y, a.x); }
template <typename T2> __device__ __forceinline__ T2 mul_mi(T2 a) { return mk(a.y, -a.x); }

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2((double)a.x, (double)a.y); }
template <typename T2> __device__ __forceinline__ T2 from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// ---------------------------------------------------------------------------------------------
// double-float: the unevaluated sum h + l of two floats with |l| <= ulp(h) / 2 (about 48
// significant bits), so that FP64-accurate transforms run on the FP32 pipe.  Built from the
// error-free transformations of Knuth (TwoSum: s + e = a + b exactly) and of Dekker with a fused
// multiply-add (TwoProduct: p + e = a * b exactly); the sum adds the low parts after TwoSum of
// the high parts and renormalises (the "sloppy" double-float addition: relative error about
// 2^-47 of max(|a|, |b|), enough for the norm-wise error bounds of FFTs and products); the
// product drops the l * l term.  Range is that of float.
struct df {
  float h, l;
  df() = default;
  __host__ __device__ __forceinline__ df(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ __forceinline__ df(double v) {
    h = (float)v;
    l = (float)(v - (double)h);
  }
};
struct __align__(16) df2 {
  df x, y;
};
template <> struct C2<df> { typedef df2 t; };

__device__ __forceinline__ df df_quick(float s, float e) {   // |s| >= |e|
  const float h = s + e;
  return df(h, e - (h - s));
}
__device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return df_quick(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_quick(p, e);
}
__device__ __forceinline__ df2 mk(df x, df y) {
  df2 r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ df2 operator+(df2 a, df2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ df2 operator-(df2 a, df2 b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ df2 operator*(df s, df2 a) { return mk(s * a.x, s * a.y); }
__device__ __forceinline__ df2 cmul(df2 a, df2 b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ df2 cmulc(df2 a, df2 b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 to_d2(df2 a) {
  return make_double2((double)a.x.h + (double)a.x.l, (double)a.y.h + (double)a.y.l);
}
template <> __device__ __forceinline__ df2 from_d2<df2>(double2 a) {
  return mk(df(a.x), df(a.y));
}

// ---------------------------------------------------------------------------------------------
// FFT plan: length n = product of radices (each 2, 3, 4 or 8), twiddle table
// tw[t] = exp(-2 pi i t / n), t = 0..n-1, in the working precision (double2, float2 or df2).
#define CHF_MAX_STAGES 16
struct FftPlan {
  int n;
  int nst;
  int rad[CHF_MAX_STAGES];
  const void* tw;
  // 1: the schedule starts with radix 3 and the transforms of the 3/2-rule padding may prune it
  // (block_fft's `prune`): zero middle third of a backward transform's input, unused middle
  // third of a forward transform's output
  int prune;
};

// radix-R DFT of v[0..R-1] in registers; INV selects exp(+2 pi i / R).
// a * b + c in one rounding where the type has a fused multiply-add (double-float: the product
// and the sum of its operators)
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df fmx(df a, df b, df c) { return a * b + c; }

template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 2, INV> {
  typedef typename C2<T>::t T2;
  __device__ __forceinline__ static void run(T2* v) {
    T2 a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, bool INV> struct Dft<T, 3, INV> {
  typedef typename C2<T>::t T2;
  __device__ __forceinline__ static void run(T2* v) {
    const T s3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
    T2 t = v[1] + v[2];
    T2 d = v[1] - v[2];
    T2 m = mk(v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y);
    v[0] = v[0] + t;
    // forward: y1 = m - i s3 d, y2 = m + i s3 d; inverse swaps the sign (s3 fused into the adds)
    const T sp = INV ? -s3 : s3;
    v[1] = mk(fmx(sp, d.y, m.x), fmx(-sp, d.x, m.y));
    v[2] = mk(fmx(-sp, d.y, m.x), fmx(sp, d.x, m.y));
  }
};

template <typename T, bool INV> struct Dft<T, 4, INV> {
  typedef typename C2<T>::t T2;
  __device__ __forceinline__ static void run(T2* v) {
    T2 t0 = v[0] + v[2], t1 = v[0] - v[2];
    T2 t2 = v[1] + v[3], t3 = v[1] - v[3];
    t3 = INV ? mul_i(t3) : mul_mi(t3);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

template <typename T, bool INV> struct Dft<T, 8, INV> {
  typedef typename C2<T>::t T2;
  __device__ __forceinline__ static void run(T2* v) {
    const T h = (T)0.70710678118654752440;  // sqrt(2)/2
    // radix-2 layer on (r, r+4)
    T2 a0 = v[0] + v[4], a4 = v[0] - v[4];
    T2 a1 = v[1] + v[5], a5 = v[1] - v[5];
    T2 a2 = v[2] + v[6], a6 = v[2] - v[6];
    T2 a3 = v[3] + v[7], a7 = v[3] - v[7];
    // even outputs: radix-4 DFT of a0..a3
    T2 e[4] = {a0, a1, a2, a3};
    Dft<T, 4, INV>::run(e);
    v[0] = e[0]; v[2] = e[1]; v[4] = e[2]; v[6] = e[3];
    // odd outputs: radix-4 DFT of (a4, w a5, w^2 a6, w^3 a7), w = exp(-+ i pi / 4).  w a5 = h p
    // and w^3 a7 = h r, so the radix-4's sums of those two lines are h (p + r) and h (p - r),
    // and the factor h is fused into the output additions.
    const T2 p = INV ? mk(a5.x - a5.y, a5.x + a5.y) : mk(a5.x + a5.y, a5.y - a5.x);
    const T2 r = INV ? mk(-(a7.x + a7.y), a7.x - a7.y) : mk(a7.y - a7.x, -(a7.x + a7.y));
    const T2 o2 = INV ? mul_i(a6) : mul_mi(a6);
    const T2 t0 = a4 + o2, t1 = a4 - o2;
    const T2 sm = p + r, df_ = p - r;
    v[1] = mk(fmx(h, sm.x, t0.x), fmx(h, sm.y, t0.y));
    v[5] = mk(fmx(-h, sm.x, t0.x), fmx(-h, sm.y, t0.y));
    // (t1 +- rot(h (p - r))), rot = -i (forward) or i (inverse)
    const T hs = INV ? -h : h;
    v[3] = mk(fmx(hs, df_.y, t1.x), fmx(-hs, df_.x, t1.y));
    v[7] = mk(fmx(-hs, df_.y, t1.x), fmx(hs, df_.x, t1.y));
  }
};

// q = t / d and t - q d for 0 <= t < 2^22, 0 < d, through a float estimate corrected once (the
// estimate is within one of the quotient there); inv = 1 / d as a float
__device__ __forceinline__ int fdivmod(int t, int d, float inv, int* rem) {
  int q = __float2int_rz((float)t * inv);
  int r = t - q * d;
  if (r < 0) {
    --q;
    r += d;
  } else if (r >= d) {
    ++q;
    r -= d;
  }
  *rem = r;
  return q;
}

// Position of element e of a line in the skewed layout of the FFT's intermediate buffers: one
// pad element after every 16.  A Stockham pass with small Ns writes its R outputs at a stride of
// R elements; skewed, 16 consecutive threads of the first pass hit 16 different 8-byte bank
// pairs (float32 complex: no conflict; 16-byte elements: two-way), where the plain layout puts
// them on two.  Lines of the skewed buffers need n + ceil(n / 16) elements (fft_line_stride).
__host__ __device__ __forceinline__ int fft_line_stride(int n) { return n + ((n + 15) >> 4); }

// Line stride of the y pass's shared tiles: the tile is filled and drained with z (the line
// index) fastest, so consecutive threads touch the same position of consecutive lines; a stride
// of 4 modulo 16 elements spreads the 8-byte (float32 complex) and 16-byte (float64 and
// double-float complex) elements of a warp over all banks with the fewest wavefronts.  The
// smallest such stride that holds a skewed line.
__host__ __device__ __forceinline__ int yline_stride(int P) {
  const int m = fft_line_stride(P);
  return m + ((20 - (m & 15)) & 15);
}

// one Stockham pass of radix R over `nlines` lines of length n (line stride ls) in shared memory;
// ski / sko: the input / output lines are in the skewed layout.  Two thread mappings:
// LOOP = false: one butterfly (line, j) per iteration (the fewest registers);
// LOOP = true: a thread owns one butterfly position j of a group of lines (line g, g + G, ...;
// G = blockDim / (n / R) groups when a line has fewer butterflies than the block has threads):
// its index arithmetic is formed once per pass, not once per butterfly, and for float32 its
// R - 1 twiddles too.  The loop costs registers, so it pays where shared memory, not registers,
// limits the CTAs per SM (the long x lines).
template <typename T, int R, bool INV, bool LOOP>
__device__ __forceinline__ void stockham_pass(const typename C2<T>::t* __restrict__ A,
                                              typename C2<T>::t* __restrict__ B, int nlines,
                                              int ls, int n, int Ns,
                                              const typename C2<T>::t* __restrict__ tw, bool ski,
                                              bool sko) {
  typedef typename C2<T>::t T2;
  const int nb = n / R;
  const int tws = n / (Ns * R);
  const float inv_nb = 1.0f / (float)nb, inv_ns = 1.0f / (float)Ns;
  const int mi = ski ? -1 : 0, mo = sko ? -1 : 0;
  if (!LOOP) {
    for (int t = threadIdx.x; t < nlines * nb; t += blockDim.x) {
      int j;
      const int line = fdivmod(t, nb, inv_nb, &j);
      int k;
      fdivmod(j, Ns, inv_ns, &k);
      const T2* in = A + line * ls;
      T2* out = B + line * ls;
      T2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = j + r * nb;
        v[r] = in[e + ((e >> 4) & mi)];
      }
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const T2 wv = tw[r * k * tws];
          v[r] = INV ? cmulc(v[r], wv) : cmul(v[r], wv);
        }
      }
      Dft<T, R, INV>::run(v);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = base + r * Ns;
        out[e + ((e >> 4) & mo)] = v[r];
      }
    }
    return;
  }
  const int G = nb >= (int)blockDim.x ? 1 : (int)blockDim.x / nb;
  for (int w = threadIdx.x; w < nb * G; w += blockDim.x) {
    int j;
    const int g = fdivmod(w, nb, inv_nb, &j);
    int k;
    fdivmod(j, Ns, inv_ns, &k);
    constexpr bool HOIST = sizeof(T2) == 8;
    const int ti = k * tws;
    T2 wr[HOIST ? R : 1];
    if (HOIST && k != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) wr[HOIST ? r : 0] = tw[r * ti];
    }
    const int base = (j - k) * R + k;
    for (int line = g; line < nlines; line += G) {
      const T2* in = A + line * ls;
      T2* out = B + line * ls;
      T2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = j + r * nb;
        v[r] = in[e + ((e >> 4) & mi)];
      }
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const T2 wv = HOIST ? wr[HOIST ? r : 0] : tw[r * ti];
          v[r] = INV ? cmulc(v[r], wv) : cmul(v[r], wv);
        }
      }
      Dft<T, R, INV>::run(v);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = base + r * Ns;
        out[e + ((e >> 4) & mo)] = v[r];
      }
    }
  }
}

// Pruned radix-3 passes of the 3/2-rule padded transforms (n = 3 m; a backward transform's input
// is zero at positions m .. 2m - 1, a forward transform's outputs there are not used).
// First pass of a backward transform (Ns = 1): butterfly j reads j, j + m, j + 2m, and the
// middle input is zero: y0 = v0 + v2, y1,2 = v0 - v2 / 2 -+ i s (-v2), s = +-sin(2 pi / 3).
template <typename T, bool INV>
__device__ __forceinline__ void pruned_first_pass3(const typename C2<T>::t* __restrict__ A,
                                                   typename C2<T>::t* __restrict__ B, int nlines,
                                                   int ls, int n, bool sko) {
  typedef typename C2<T>::t T2;
  const int m = n / 3;
  const float inv_m = 1.0f / (float)m;
  const int mo = sko ? -1 : 0;
  const T s3 = (T)0.86602540378443864676;
  const T sp = INV ? -s3 : s3;
  for (int t = threadIdx.x; t < nlines * m; t += blockDim.x) {
    int j;
    const int line = fdivmod(t, m, inv_m, &j);
    const T2* in = A + line * ls;
    T2* out = B + line * ls;
    const T2 v0 = in[j], v2 = in[j + 2 * m];
    const T2 mm = mk(fmx((T)-0.5, v2.x, v0.x), fmx((T)-0.5, v2.y, v0.y));
    T2 y[3];
    y[0] = v0 + v2;
    // d = v1 - v2 = -v2: y1 = m + (s d.y, -s d.x), y2 = m - (s d.y, -s d.x)
    y[1] = mk(fmx(-sp, v2.y, mm.x), fmx(sp, v2.x, mm.y));
    y[2] = mk(fmx(sp, v2.y, mm.x), fmx(-sp, v2.x, mm.y));
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int e = 3 * j + r;
      out[e + ((e >> 4) & mo)] = y[r];
    }
  }
}
// Last pass of a forward transform (Ns = m): butterfly j writes j, j + m, j + 2m; the middle
// output is not computed.
template <typename T>
__device__ __forceinline__ void pruned_last_pass3(const typename C2<T>::t* __restrict__ A,
                                                  typename C2<T>::t* __restrict__ B, int nlines,
                                                  int ls, int n,
                                                  const typename C2<T>::t* __restrict__ tw,
                                                  bool ski) {
  typedef typename C2<T>::t T2;
  const int m = n / 3;
  const float inv_m = 1.0f / (float)m;
  const int mi = ski ? -1 : 0;
  const T s3 = (T)0.86602540378443864676;
  for (int t = threadIdx.x; t < nlines * m; t += blockDim.x) {
    int j;
    const int line = fdivmod(t, m, inv_m, &j);
    const T2* in = A + line * ls;
    T2* out = B + line * ls;
    T2 v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int e = j + r * m;
      v[r] = in[e + ((e >> 4) & mi)];
    }
    if (j != 0) {
      v[1] = cmul(v[1], tw[j]);
      v[2] = cmul(v[2], tw[2 * j]);
    }
    const T2 tt = v[1] + v[2], d = v[1] - v[2];
    const T2 mm = mk(v[0].x - (T)0.5 * tt.x, v[0].y - (T)0.5 * tt.y);
    out[j] = v[0] + tt;
    out[j + 2 * m] = mk(fmx(-s3, d.y, mm.x), fmx(s3, d.x, mm.y));
  }
}

// Block-cooperative FFT of nlines lines (stride ls) held in A; B is a scratch buffer of the same
// shape.  Returns the buffer holding the result (A or B).  Unnormalised; INV = exp(+).
// Every thread of the block must call it (it contains __syncthreads()).  SKEW: the buffers
// between passes use the skewed layout (ls >= fft_line_stride(n)); input and result are plain.
// prune (with a pruning plan, pl.prune): the transform of a 3/2-rule padding.  Backward: the
// input's middle third is zero and is not read (the radix-3 pass runs first).  Forward: the
// radix-3 pass runs last and the middle third of the output is not written.
template <typename T, bool INV, bool SKEW = false, bool LOOP = false>
__device__ typename C2<T>::t* block_fft(typename C2<T>::t* A, typename C2<T>::t* B, int nlines,
                                        int ls, const FftPlan& pl, bool prune = false) {
  typedef typename C2<T>::t T2;
  const T2* tw = reinterpret_cast<const T2*>(pl.tw);
  prune = prune && pl.prune && pl.nst >= 2 && pl.rad[0] == 3;
  int Ns = 1;
  for (int q = 0; q < pl.nst; ++q) {
    // pass order: the schedule's, except that a pruned forward transform takes its first
    // (radix-3) stage last
    const int s = (prune && !INV) ? (q + 1 < pl.nst ? q + 1 : 0) : q;
    const int R = pl.rad[s];
    const bool ski = SKEW && q > 0, sko = SKEW && q + 1 < pl.nst;
    if (prune && INV && q == 0) pruned_first_pass3<T, INV>(A, B, nlines, ls, pl.n, sko);
    else if (prune && !INV && q + 1 == pl.nst) pruned_last_pass3<T>(A, B, nlines, ls, pl.n, tw, ski);
    else if (R == 4) stockham_pass<T, 4, INV, LOOP>(A, B, nlines, ls, pl.n, Ns, tw, ski, sko);
    else if (R == 8) stockham_pass<T, 8, INV, LOOP>(A, B, nlines, ls, pl.n, Ns, tw, ski, sko);
    else if (R == 2) stockham_pass<T, 2, INV, LOOP>(A, B, nlines, ls, pl.n, Ns, tw, ski, sko);
    else stockham_pass<T, 3, INV, LOOP>(A, B, nlines, ls, pl.n, Ns, tw, ski, sko);
    __syncthreads();
    T2* tmp = A;
    A = B;
    B = tmp;
    Ns *= R;
  }
  return A;
}

// ---------------------------------------------------------------------------------------------
// per-grid constants handed to the kernels by value
struct GridDev {
  int nx, ny, nz, N, Mx, Px, Py;
  double lx, ly, re, we, ch, pe, dt, gx, gy;
  double beta;   // 2 Re / dt
  double lam;    // sqrt(Pe / (Ch^2 dt))
  double shat;   // 2 lam Ch^2
  double kappa;  // 3/sqrt(8) Ch / We
  // Gottlieb-Orszag row coefficients (device arrays of length nz):
  // t1[n] = c_{n-2}/(4n(n-1)), t2[n] = [n<=N-2]/(2(n^2-1)), t3[n] = [n+2<=N-2]/(4n(n+1))
  const double* go1;
  const double* go2;
  const double* go3;
  // time-independent tau-operator tables, one column per distinct k^2 (index
  // K = mx (ny/2 + 1) + |my|, NK columns), layout described in ch_zline.cu
  const double* fac;
  int NK;
  // cos(pi j / N), sin(pi j / N), j = 0..N-1 (Chebyshev transform through an N-point FFT)
  const double2* zcs;
  // wall conditions: 0 no-slip (u = v = w = dw/dz = 0), 1 free-slip (du/dz = dv/dz = 0, w = 0,
  // d2w/dz2 = 0) at both walls
  int bc;
};

}  // namespace chf
