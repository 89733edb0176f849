// Chebyshev transforms along z (Sec. 3.2.1) as float64-accurate matrix products on the tensor
// cores: tcgen05 MMAs with bf16 operands staged in shared memory and fp32 accumulators in tensor
// memory.
//
// The transform of one line is a product with a fixed Nz x Nz matrix B (rows = outputs):
//   forward (samples at z_k = cos(pi k / N) -> coefficients)
//     a_n = sum_k W_nk f_k,  W_nk = e_k cos(pi n k / N) / (cbar_n N),
//     e_k = 1 at k = 0, N and 2 otherwise, cbar_n = 2 at n = 0, N and 1 otherwise;
//   backward (coefficients -> samples)  f_j = sum_n cos(pi n j / N) a_n.
// Real and imaginary parts are separate rows of the left operand.
//
// Exact split (Ozaki scheme).  A row x with max |x_k| < 2^E becomes the integer vector
// X_k = round(x_k 2^(54-E)), |X_k| < 2^54 (53 significant bits for the largest element, as in
// float64), written with signed base-128 digits
//   X_k = sum_{i=0..7} a_ik 128^(7-i),  a_ik in [-64, 63]
// (X + bias, bias = 64 sum_t 128^t, stays inside eight 7-bit groups for |X| < 2^54)
// (bf16 holds these exactly); each output row n of B likewise with its own scale 2^F_n and
// digits b_jnk.  A digit product C_ij = sum_k a_ik b_jnk is an integer with |C_ij| <= 64*64*K,
// and the eight products with the same i + j = d share one fp32 accumulator G_d:
// |G_d| <= 8*64*64*K < 2^24 for K < 512, so every accumulation is exact.  Keeping d <= 7 (36
// products) drops terms of order 2^-54 of the row-max x column-max scale; with the 2^-55
// quantisation of both operands and the final rounding the error stays at a few units of 2^-53
// of max|x| x max_n sum_k |B_nk|, the accuracy of a float64 transform.  The result
//   sum_k x_k B_nk = 2^(E + F_n - 108) sum_{d<=7} 128^(14-d) G_d
// is recombined in 64-bit integers and rounded once to float64 (or float32) with integer
// operations only (the float64 pipe is the scarce resource on this part).
//
// One CTA (512 threads, 1 per SM) computes a 128-row x NT-column tile: the 128 rows are the re
// and im parts of 64 lines of one field, the NT columns one slice of the outputs.  Per K-chunk of
// at most 144: the eight B digit planes of the slice arrive by one bulk async copy; the threads
// turn their row elements into the biased integers X + bias (registers) and write one A digit
// plane at a time into a double-buffered shared-memory tile in the tensor cores' canonical
// no-swizzle K-major layout, while one thread issues the MMAs of the previous plane.  The eight
// accumulators G_0..G_7 (8 NT fp32 columns) live in tensor memory until the epilogue.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ch_internal.h"

namespace chf {

namespace {

constexpr int TCT = 512;          // producer threads per CTA (plus one issuer warp)
constexpr int TCM = 128;          // rows per tile = tensor-memory lanes
constexpr int TCKC = 144;         // K per chunk
constexpr int TCG = TCKC / 8;     // 8-element core-matrix groups per chunk
constexpr unsigned long long kBias = 0x0081020408102040ull;   // 64 * sum_{t<8} 128^t
constexpr uint64_t kWaitNs = 1000000000ull;                   // bound of every device wait

// ---- PTX wrappers -----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor, no swizzle: lbo = byte stride between core matrices along K,
// sbo = byte stride between 8-row core-matrix groups along M (or N); version 1 at bit 46
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase with the given parity; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = gtime();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtime() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// eight 4-column loads of this warp's 32 lanes, then one wait that the values depend on
__device__ __forceinline__ void tmem_ld8x4(uint32_t addr, int stride, uint32_t (&v)[8][4]) {
#pragma unroll
  for (int d = 0; d < 8; ++d)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3])
                 : "r"(addr + (uint32_t)(d * stride)));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[0][2]), "+r"(v[0][3]), "+r"(v[1][0]),
                 "+r"(v[1][1]), "+r"(v[1][2]), "+r"(v[1][3]), "+r"(v[2][0]), "+r"(v[2][1]),
                 "+r"(v[2][2]), "+r"(v[2][3]), "+r"(v[3][0]), "+r"(v[3][1]), "+r"(v[3][2]),
                 "+r"(v[3][3]), "+r"(v[4][0]), "+r"(v[4][1]), "+r"(v[4][2]), "+r"(v[4][3]),
                 "+r"(v[5][0]), "+r"(v[5][1]), "+r"(v[5][2]), "+r"(v[5][3]), "+r"(v[6][0]),
                 "+r"(v[6][1]), "+r"(v[6][2]), "+r"(v[6][3]), "+r"(v[7][0]), "+r"(v[7][1]),
                 "+r"(v[7][2]), "+r"(v[7][3])
               :
               : "memory");
}

// ---- float bits -> biased fixed point, digits, and back ---------------------------------------
template <typename T> struct FBits;
template <> struct FBits<double> {
  typedef unsigned long long U;
  static constexpr int MB = 52, EMAX = 0x7FF, SH0 = 1, EOFF = 1022;
  __device__ static U bits(double x) { return (U)__double_as_longlong(x); }
};
template <> struct FBits<float> {
  typedef unsigned int U;
  static constexpr int MB = 23, EMAX = 0xFF, SH0 = 30, EOFF = 126;
  __device__ static U bits(float x) { return __float_as_uint(x); }
};

// X + bias for an element with bit pattern b in a row whose largest exponent field is maxe
// (X = round(x 2^(54-E)), E = maxe - EOFF; |X| < 2^54 so X + bias has eight 7-bit groups,
// group i holding digit a_i + 64)
template <typename T>
__device__ __forceinline__ unsigned long long to_biased(typename FBits<T>::U b, int maxe) {
  typedef FBits<T> F;
  if (maxe >= F::EMAX) return kBias;
  const int ef = (int)((b >> F::MB) & (typename F::U)F::EMAX);
  unsigned long long mant = (unsigned long long)(b & ((((typename F::U)1) << F::MB) - 1));
  if (ef) mant |= 1ull << F::MB;
  const int s = (ef ? ef : 1) - maxe + F::SH0;
  unsigned long long X;
  if (s >= 0) {
    X = mant << s;
  } else {
    const int sh = -s;
    X = sh >= 64 ? 0ull : (mant + (1ull << (sh - 1))) >> sh;
  }
  const bool neg = (b >> (8 * sizeof(typename F::U) - 1)) & 1;
  return neg ? kBias - X : kBias + X;
}

// digits at bit offset sh of two elements, as two bf16 packed in one word (first in the low half)
__device__ __forceinline__ uint32_t digit_pair(unsigned long long y0, unsigned long long y1,
                                               int sh) {
  const uint32_t u0 = (uint32_t)(y0 >> sh) & 127u, u1 = (uint32_t)(y1 >> sh) & 127u;
  const float f0 = __uint_as_float(0x4B000000u | u0) - 8388672.0f;   // u - 64, exact
  const float f1 = __uint_as_float(0x4B000000u | u1) - 8388672.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// integer value of an fp32 accumulator (integer-valued, |v| < 2^24)
__device__ __forceinline__ int acc_int(uint32_t b) {
  int e = (int)((b >> 23) & 0xFF);
  if (e < 127) return 0;
  if (e > 150) e = 150;
  const int v = (int)((b & 0x7FFFFFu) | 0x800000u) >> (150 - e);
  return (b >> 31) ? -v : v;
}

// T 2^e rounded to nearest even, by integer operations (ldexp fallback outside the normal range)
template <typename TO> __device__ TO scaled(long long T, int e);
template <> __device__ __forceinline__ double scaled<double>(long long T, int e) {
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  unsigned long long a = neg ? 0ull - (unsigned long long)T : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mant = a >> 11;
  const unsigned long long rem = a & 0x7FFull;
  int ex = 63 - lz + e;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++ex;
    }
  }
  const int be = ex + 1023;
  if (be <= 0 || be >= 2047) return ldexp((double)T, e);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                          ((unsigned long long)be << 52) |
                                          (mant & 0xFFFFFFFFFFFFFull)));
}
template <> __device__ __forceinline__ float scaled<float>(long long T, int e) {
  if (T == 0) return 0.0f;
  const bool neg = T < 0;
  unsigned long long a = neg ? 0ull - (unsigned long long)T : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mant = a >> 40;
  const unsigned long long rem = a & 0xFFFFFFFFFFull, half = 1ull << 39;
  int ex = 63 - lz + e;
  if (rem > half || (rem == half && (mant & 1ull))) {
    ++mant;
    if (mant >> 24) {
      mant >>= 1;
      ++ex;
    }
  }
  const int be = ex + 127;
  if (be <= 0 || be >= 255) return ldexpf((float)T, e);
  return __uint_as_float(((unsigned)neg << 31) | ((unsigned)be << 23) |
                         (unsigned)(mant & 0x7FFFFFull));
}
template <typename TO> __device__ __forceinline__ TO qnan();
template <> __device__ __forceinline__ double qnan<double>() {
  return __longlong_as_double(0x7FF8000000000000ll);
}
template <> __device__ __forceinline__ float qnan<float>() { return __uint_as_float(0x7FC00000u); }

__host__ __device__ constexpr size_t tc_smem_bytes(int NT) {
  return (size_t)8 * NT * TCKC * 2 + (size_t)2 * TCM * TCKC * 2 + TCM * sizeof(int) + 64;
}

// ---- the transform kernel ---------------------------------------------------------------------
// in / out: nf fields of complex lines (re, im interleaved), field stride fsi / fso complex
// elements, line stride Nz; bdig: nNt output slices of 8 NT Kp bf16 digits (per slice: per chunk
// of K, the eight digit planes, each NT x KC in the canonical core-matrix layout); fexp: F_n.
//
// Warps 0..15 produce (row exponents, digit planes) and run the epilogue; warp 16 allocates the
// tensor memory and one of its lanes issues the bulk copies and the MMAs.  Plane t goes to
// shared buffer t % 2: the producers wait for `empty` of that buffer (the MMAs of plane t - 2
// completed, signalled by tcgen05.commit), write the plane and arrive on `full` (one arrival
// per warp); the issuer waits for `full`, issues the plane's MMAs and commits to `empty`.
template <typename TI, typename TO, int NT>
__global__ void __launch_bounds__(TCT + 32, 1)
    cheb_tc_kernel(const TI* __restrict__ in, long long fsi, TO* __restrict__ out, long long fso,
                   int nlines, int Nz, int Kp, int tpf, int nNt,
                   const uint16_t* __restrict__ bdig, const int* __restrict__ fexp,
                   int* __restrict__ err) {
  typedef FBits<TI> F;
  typedef typename F::U U;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sB = tsm;
  unsigned char* sA = sB + (size_t)8 * NT * TCKC * 2;
  int* sE = reinterpret_cast<int*>(sA + (size_t)2 * TCM * TCKC * 2);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sE + TCM);
  uint32_t* sT = reinterpret_cast<uint32_t*>(bars + 5);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.x % nNt, tile = blockIdx.x / nNt;
  const int fld = tile / tpf;
  const int line0 = (tile - fld * tpf) * (TCM / 2);
  const int nchunk = (Kp + TCKC - 1) / TCKC;
  // barriers: B loaded; full[b] (16 producer warps arrived); empty[b] (MMAs of the plane done)
  const uint32_t barB = su32(&bars[0]), barFull = su32(&bars[1]), barEmpty = su32(&bars[3]);
  const size_t bslice = (size_t)8 * NT * Kp;
  const bool issuer = (warp == TCT / 32);
  if (issuer && lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barB));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 16;" ::"r"(barFull));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 16;" ::"r"(barFull + 8));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barEmpty));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barEmpty + 8));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bulk_load(su32(sB), bdig + (size_t)nt * bslice, (uint32_t)(8 * NT * min(TCKC, Kp) * 2), barB);
  }
  if (issuer) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(sT)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sT;
  bool ok = true;

  if (issuer) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                             ((uint32_t)(TCM >> 4) << 24);   // bf16 x bf16 -> fp32, K-major
      const uint32_t sA0 = su32(sA), sB0 = su32(sB);
      for (int ch = 0; ch < nchunk; ++ch) {
        const int KCc = min(TCKC, Kp - ch * TCKC);
        if (ch > 0) {
          // the previous chunk's last plane (t = 8 ch - 1, buffer 1) must be consumed first
          ok = mbar_wait(barEmpty + 8, ((8 * ch - 1) >> 1) & 1) && ok;
          bulk_load(sB0, bdig + (size_t)nt * bslice + (size_t)ch * 8 * NT * TCKC,
                    (uint32_t)(8 * NT * KCc * 2), barB);
        }
        ok = mbar_wait(barB, ch & 1) && ok;
        for (int i = 0; i < 8; ++i) {
          const int t = ch * 8 + i, bf = t & 1;
          ok = mbar_wait(barFull + 8 * bf, (t >> 1) & 1) && ok;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // descriptors of k-step 0; a k-step adds 2 core-matrix groups to the start address
          const uint64_t ad = sdesc(sA0 + (uint32_t)(bf * TCM * TCKC * 2), 2048, 128);
          for (int j = 0; i + j < 8; ++j) {
            const uint64_t bd =
                sdesc(sB0 + (uint32_t)(j * NT * KCc * 2), (NT / 8) * 128, 128);
            const uint32_t dt = tmem + (uint32_t)((i + j) * NT);
            for (int s = 0; s < KCc / 16; ++s)
              mma_bf16(dt, ad + (uint64_t)(s * 256), bd + (uint64_t)(s * 16 * (NT / 8)), idesc,
                       (uint32_t)((ch | i | s) != 0));
          }
          mma_commit(barEmpty + 8 * bf);
        }
      }
    }
    __syncwarp();
  } else {
    // producers: warp = 8-row core-matrix group, lane = (row in the group, pair of k)
    const int r = lane >> 2, q = lane & 3;
    const int m = warp * 8 + r;
    const int line = line0 + (m >> 1);
    const bool rowok = line < nlines;
    const TI* src = in + ((size_t)fld * fsi + (size_t)(rowok ? line : 0) * Nz) * 2 + (m & 1);
    // chunk 0 in registers; the largest exponent field of the row over all of K
    unsigned long long y[2 * TCG];
    int maxe = 1;
    {
      const int ngr = min(TCKC, Kp) / 8;
#pragma unroll
      for (int gl = 0; gl < TCG; ++gl)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = 8 * gl + 2 * q + e;
          U b = 0;
          if (gl < ngr && rowok && k < Nz) b = F::bits(src[2 * (size_t)k]);
          y[2 * gl + e] = (unsigned long long)b;
          maxe = max(maxe, (int)((b >> F::MB) & (U)F::EMAX));
        }
    }
    for (int ch = 1; ch < nchunk; ++ch) {
      const int ngr = min(TCKC, Kp - ch * TCKC) / 8;
#pragma unroll
      for (int gl = 0; gl < TCG; ++gl)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = ch * TCKC + 8 * gl + 2 * q + e;
          if (gl < ngr && rowok && k < Nz)
            maxe = max(maxe, (int)((F::bits(src[2 * (size_t)k]) >> F::MB) & (U)F::EMAX));
        }
    }
    maxe = max(maxe, __shfl_xor_sync(0xffffffffu, maxe, 1));
    maxe = max(maxe, __shfl_xor_sync(0xffffffffu, maxe, 2));
    if (q == 0) sE[m] = maxe;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int ngr = min(TCKC, Kp - ch * TCKC) / 8;
      if (ch == 0) {
#pragma unroll
        for (int i = 0; i < 2 * TCG; ++i) y[i] = to_biased<TI>((U)y[i], maxe);
      } else {
#pragma unroll
        for (int gl = 0; gl < TCG; ++gl)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = ch * TCKC + 8 * gl + 2 * q + e;
            U b = 0;
            if (gl < ngr && rowok && k < Nz) b = F::bits(src[2 * (size_t)k]);
            y[2 * gl + e] = to_biased<TI>(b, maxe);
          }
      }
      for (int i = 0; i < 8; ++i) {
        const int t = ch * 8 + i, bf = t & 1;
        if (t >= 2) ok = mbar_wait(barEmpty + 8 * bf, ((t - 2) >> 1) & 1) && ok;
        uint32_t* dst = reinterpret_cast<uint32_t*>(sA + (size_t)bf * TCM * TCKC * 2);
        const int sh = 7 * (7 - i);
#pragma unroll
        for (int gl = 0; gl < TCG; ++gl)
          if (gl < ngr)
            dst[(gl * 16 + warp) * 32 + lane] = digit_pair(y[2 * gl], y[2 * gl + 1], sh);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(barFull + 8 * bf)
                       : "memory");
      }
    }
    const int tl = 8 * nchunk - 1;
    ok = mbar_wait(barEmpty + 8 * (tl & 1), (tl >> 1) & 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // sE of the other warps' rows: written before their first plane, read after all MMAs,
    // which needed every warp's planes; the named barrier below orders it for the compiler
    asm volatile("bar.sync 1, %0;" ::"r"(TCT) : "memory");

    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its rows), columns
    // (w / 4) NT/4 .. + NT/4 - 1 of each of the eight accumulators
    constexpr int CW = NT / 4;
    const int qd = warp & 3, cg = warp >> 2;
    const int mm = qd * 32 + lane;
    const int oline = line0 + (mm >> 1);
    const int me = sE[mm];
    const bool orow = ok && oline < nlines;
    TO* dstp =
        out + ((size_t)fld * fso + (size_t)(oline < nlines ? oline : 0) * Nz) * 2 + (mm & 1);
    const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(cg * CW);
    for (int c0 = 0; c0 < CW; c0 += 4) {
      uint32_t v[8][4];
      tmem_ld8x4(tb + (uint32_t)c0, NT, v);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n = nt * NT + cg * CW + c0 + e;
        if (orow && n < Nz) {
          long long H = 0, L = 0;
#pragma unroll
          for (int d = 0; d < 4; ++d) H = H * 128 + acc_int(v[d][e]);
#pragma unroll
          for (int d = 4; d < 8; ++d) L = L * 128 + acc_int(v[d][e]);
          const long long T = H * 262144ll + (L >> 10);   // (H 2^28 + L) / 2^10
          // sum = 2^(E + F - 108) 2^49 (H 2^28 + L) = T 2^(E + F - 49)
          dstp[2 * (size_t)n] =
              me >= F::EMAX ? qnan<TO>() : scaled<TO>(T, me - F::EOFF + fexp[n] - 49);
        }
      }
    }
  }
  if (!ok) atomicOr(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (issuer)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <typename TI, typename TO, int NT>
cudaError_t launch_t(const void* in, long long fsi, void* out, long long fso, int nf, int nlines,
                     int Nz, const ChebTc& t, int* err, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(NT);
  const int tpf = (nlines + TCM / 2 - 1) / (TCM / 2);
  const long long nblk = (long long)nf * tpf * t.nNt;
  if (nblk <= 0) return cudaSuccess;
  cheb_tc_kernel<TI, TO, NT><<<(unsigned)nblk, TCT + 32, smem, s>>>(
      (const TI*)in, fsi, (TO*)out, fso, nlines, Nz, t.Kp, tpf, t.nNt, t.dig, t.fexp, err);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_nt(const void* in, long long fsi, void* out, long long fso, int nf,
                      int nlines, int Nz, const ChebTc& t, int* err, cudaStream_t s) {
  return t.NT == 48 ? launch_t<TI, TO, 48>(in, fsi, out, fso, nf, nlines, Nz, t, err, s)
                    : launch_t<TI, TO, 64>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
}

uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  return (uint16_t)(u >> 16);   // exact: the digits have at most 7 significant bits
}

}  // namespace

int cheb_tc_tables(int N, int dir, std::vector<uint16_t>& dig, std::vector<int>& fexp, int& NT,
                   int& nNt, int& Kp) {
  const int Nz = N + 1;
  Kp = (Nz + 15) / 16 * 16;
  if (N < 2 || Kp >= 512) return -1;
  // output slice width: 48 (more MMAs, each smem-bound) or 64 (fewer padded columns)
  const int c48 = (Nz + 47) / 48 * 48, c64 = (Nz + 63) / 64 * 64;
  NT = (5 * c48 <= 4 * c64) ? 48 : 64;
  nNt = (Nz + NT - 1) / NT;
  dig.assign((size_t)nNt * 8 * NT * Kp, 0);
  fexp.assign((size_t)nNt * NT, 0);
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> row(Nz);
  std::vector<long long> Y(Nz);
  for (int n = 0; n < Nz; ++n) {
    long double mx = 0.0L;
    for (int k = 0; k < Nz; ++k) {
      int a = (int)(((long long)n * k) % (2 * N));
      if (a > N) a = 2 * N - a;   // cos(pi a / N) = cos(pi (2N - a) / N)
      long double c;
      if (2 * a == N) c = 0.0L;
      else if (2 * a < N) c = cosl(pi * (long double)a / (long double)N);
      else c = -cosl(pi * (long double)(N - a) / (long double)N);
      long double v = c;
      if (dir == 0) {
        const long double ek = (k == 0 || k == N) ? 1.0L : 2.0L;
        const long double cb = (n == 0 || n == N) ? 2.0L : 1.0L;
        v = ek * c / (cb * (long double)N);
      }
      row[k] = v;
      if (fabsl(v) > mx) mx = fabsl(v);
    }
    int F = 0;
    if (mx > 0.0L) {
      F = ilogbl(mx) + 1;
      for (;;) {
        bool fit = true;
        for (int k = 0; k < Nz; ++k) {
          Y[k] = llroundl(ldexpl(row[k], 54 - F));
          if (Y[k] >= (1ll << 54) || Y[k] <= -(1ll << 54)) fit = false;
        }
        if (fit) break;
        ++F;
      }
    } else {
      for (int k = 0; k < Nz; ++k) Y[k] = 0;
    }
    fexp[n] = F;
    const int nt = n / NT, nl = n % NT;
    for (int k = 0; k < Nz; ++k) {
      const unsigned long long yb = (unsigned long long)Y[k] + kBias;
      const int ch = k / TCKC, kl = k % TCKC;
      const int KCc = std::min(TCKC, Kp - ch * TCKC);
      const size_t base = (size_t)nt * 8 * NT * Kp + (size_t)ch * 8 * NT * TCKC;
      const size_t off = ((size_t)(kl / 8) * (NT / 8) + nl / 8) * 64 + (nl % 8) * 8 + kl % 8;
      for (int j = 0; j < 8; ++j) {
        const int d = (int)((yb >> (7 * (7 - j))) & 127ull) - 64;
        dig[base + (size_t)j * NT * KCc + off] = bf16_bits((float)d);
      }
    }
  }
  return 0;
}

size_t cheb_tc_smem(int NT) { return tc_smem_bytes(NT); }

cudaError_t cheb_tc_prepare(int NT) {
  const size_t smem = tc_smem_bytes(NT);
  cudaError_t e = cudaSuccess;
  if (NT == 48) {
    static int c0 = 0, c1 = 0, c2 = 0;
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, double, 48>, smem, &c0);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<float, double, 48>, smem, &c1);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, float, 48>, smem, &c2);
  } else {
    static int c0 = 0, c1 = 0, c2 = 0;
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, double, 64>, smem, &c0);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<float, double, 64>, smem, &c1);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, float, 64>, smem, &c2);
  }
  return e;
}

cudaError_t launch_cheb_tc(int tin, int tout, const void* in, long long fsi, void* out,
                           long long fso, int nf, int nlines, int Nz, const ChebTc& t, int* err,
                           cudaStream_t s) {
  if (tin == 0 && tout == 0)
    return launch_nt<double, double>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
  if (tin == 1 && tout == 0)
    return launch_nt<float, double>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
  if (tin == 0 && tout == 1)
    return launch_nt<double, float>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace chf
