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
// Tiles and data flow.  A tile is 128 rows (re and im of 64 lines of one field) by all Nz
// outputs, computed as nNt output slices of NT (48 or 64) columns; the eight accumulators
// G_0..G_7 of a slice (8 NT fp32 columns) live in tensor memory.  The eight B digit planes of a
// slice are stacked into one 8 NT-row operand, so A plane i needs a single MMA chain over rows
// 0 .. (8-i) NT with its accumulator starting at column i NT: product (i, j) lands on diagonal
// i + j.  (The MMA issue rate, about one instruction per 50..128 cycles, is what limits the
// kernel; merging the pairs this way cuts 36 small MMAs per k-step to 8..12 large ones.)
// Persistent CTAs (one per SM) walk the tiles with 16 producer warps and one issuer warp: the
// producers convert their rows to fixed point once per tile, write the digit planes of the first
// slice into rotating shared buffers and their 7-bit groups (one byte each) into a per-CTA plane
// cache in global memory, and rebuild the later slices' planes from that cache; the issuer copies
// the digits of B and issues the MMAs.  Rows are split into K chunks of 96 that accumulate into
// the same tensor memory.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ch_internal.h"

namespace chf {

namespace {

constexpr int TCT = 512;          // threads per CTA
constexpr int TCM = 128;          // rows per tile = tensor-memory lanes
constexpr int TCKC = 96;          // K per chunk
constexpr int TCG = TCKC / 8;     // 8-element core-matrix groups per chunk
constexpr int kNA = 4;            // shared buffers of A digit planes (kNA - 1 copied ahead)
constexpr int kNB = 1;            // shared buffers of B digit planes
constexpr int kSmallK = 144;      // K up to which every accumulator stays below 2^22 in magnitude
// 32-bit words of one cached plane (four 7-bit groups per word, TCM x TCKC groups)
constexpr int kCacheWords = TCM * TCKC / 4;
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
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// wait for the phase with the given parity until the global timer passes `deadline`
__device__ __forceinline__ bool mbar_wait_until(uint32_t bar, uint32_t parity,
                                                uint64_t deadline) {
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtime() > deadline) return false;
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;   // the common case: no clock read
  return mbar_wait_until(bar, parity, gtime() + kWaitNs);
}
// The waits of one thread.  The first wait that runs out clears `ok`; every later wait returns
// false at once, so a thread spends at most one bound waiting in vain however many waits follow
// (the transform kernel's issuer then stops issuing and drains, its producers skip their waits).
struct Waiter {
  bool ok = true;
  __device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity) {
    ok = ok && mbar_wait(bar, parity);
    return ok;
  }
};
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
// L2 policy that keeps lines resident (the per-CTA digit-plane cache and the matrix digits,
// re-read for every output slice) ahead of the streamed rows and outputs
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// bulk copy global -> shared with completion on an mbarrier, read under the L2 policy `pol`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar, uint64_t pol) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], "
      "[%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}
// a 32-bit store to global memory under the L2 policy `pol`
__device__ __forceinline__ void st_hint(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}
// streamed (evict-first) loads of the rows' second read and stores of the outputs
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ df ld_stream(const df* p) {
  const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}
__device__ __forceinline__ void st_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(df* p, df v) {
  __stcs(reinterpret_cast<float2*>(p), make_float2(v.h, v.l));
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
  __device__ static int expo(U b) { return (int)((b >> 52) & 0x7FFull); }
};
template <> struct FBits<float> {
  typedef unsigned int U;
  static constexpr int MB = 23, EMAX = 0xFF, SH0 = 30, EOFF = 126;
  __device__ static U bits(float x) { return __float_as_uint(x); }
  __device__ static int expo(U b) { return (int)((b >> 23) & 0xFFu); }
};
// double-float h + l: the bits of h in the low word, of l in the high word; the row scale comes
// from h (|h + l| < 2^E whenever |h| < 2^E, since |l| <= ulp(h) / 2)
template <> struct FBits<df> {
  typedef unsigned long long U;
  static constexpr int EMAX = 0xFF, EOFF = 126;
  __device__ static U bits(df x) {
    return (U)__float_as_uint(x.h) | ((U)__float_as_uint(x.l) << 32);
  }
  __device__ static int expo(U b) { return (int)((b >> 23) & 0xFFull); }
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

// round(f 2^(54-E)) of a float with bit pattern b, E = maxe - 126, as a signed integer
__device__ __forceinline__ long long fixed_f32(unsigned b, int maxe) {
  const int ef = (int)((b >> 23) & 0xFFu);
  unsigned long long mant = b & 0x7FFFFFu;
  if (ef) mant |= 1ull << 23;
  const int s = (ef ? ef : 1) - maxe + 30;
  unsigned long long X;
  if (s >= 0) {
    X = mant << s;
  } else {
    const int sh = -s;
    X = sh >= 64 ? 0ull : (mant + (1ull << (sh - 1))) >> sh;
  }
  return (b >> 31) ? -(long long)X : (long long)X;
}
// X + bias of a double-float: round(h 2^(54-E)) + round(l 2^(54-E)) (one extra unit of error
// at most, 2^-54 of the row scale)
template <>
__device__ __forceinline__ unsigned long long to_biased<df>(unsigned long long b, int maxe) {
  if (maxe >= 0xFF) return kBias;
  return kBias + (unsigned long long)(fixed_f32((unsigned)b, maxe) +
                                      fixed_f32((unsigned)(b >> 32), maxe));
}

// digits at bit offset sh (< 28) of two elements' 28-bit halves, as two bf16 packed in one word
// (first in the low half): u = 7-bit group, value u - 64 through the float 2^23 + u
__device__ __forceinline__ uint32_t digit_pair(uint32_t w0, uint32_t w1, int sh) {
  const float f0 = __uint_as_float(0x4B000000u | ((w0 >> sh) & 127u)) - 8388672.0f;
  const float f1 = __uint_as_float(0x4B000000u | ((w1 >> sh) & 127u)) - 8388672.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// the 7-bit groups at bit offset sh of four elements' 28-bit halves as four bytes (first in the
// lowest byte): the plane cache's format, half the size of the bf16 digits
__device__ __forceinline__ uint32_t pack_groups(uint32_t w0, uint32_t w1, uint32_t w2,
                                                uint32_t w3, int sh) {
  return ((w0 >> sh) & 127u) | (((w1 >> sh) & 127u) << 8) | (((w2 >> sh) & 127u) << 16) |
         (((w3 >> sh) & 127u) << 24);
}
// two bytes of the plane cache (7-bit groups u, digit u - 64) as two bf16 digits in one word
__device__ __forceinline__ uint32_t group_pair(uint32_t b2) {
  const float f0 = __uint_as_float(0x4B000000u | (b2 & 127u)) - 8388672.0f;
  const float f1 = __uint_as_float(0x4B000000u | ((b2 >> 8) & 127u)) - 8388672.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}
// a 32-bit load under the L2 policy `pol`
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// integer value of an fp32 accumulator: exact for integer values of magnitude <= 2^22 through
// the float 1.5 2^23 + v (small K) ...
__device__ __forceinline__ int acc_int_small(uint32_t b) {
  return __float_as_int(__uint_as_float(b) + 12582912.0f) - 0x4B400000;
}
// ... and by one float-to-integer conversion for any integer value below 2^24 (larger K; the
// accumulator holds an exact integer, so the conversion does not round)
__device__ __forceinline__ int acc_int(uint32_t b) { return __float2int_rz(__uint_as_float(b)); }

// T 2^e rounded to nearest even, by integer operations (ldexp fallback outside the normal range)
template <typename TO> __device__ TO scaled(long long T, int e);
template <> __device__ __forceinline__ double scaled<double>(long long T, int e) {
  if (T == 0) return 0.0;
  const unsigned long long sg = (unsigned long long)T & 0x8000000000000000ull;
  unsigned long long a = sg ? 0ull - (unsigned long long)T : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;                                     // leading one at bit 63
  unsigned long long mant = a >> 11;            // 53 bits
  const unsigned rem = (unsigned)(a & 0x7FFull);
  mant += (rem + (unsigned)(mant & 1ull)) > 0x400u ? 1ull : 0ull;   // to nearest, ties to even
  const int be = 63 - lz + e + 1023 + (int)(mant >> 53);
  if (be <= 0 || be >= 2047) return ldexp((double)T, e);
  return __longlong_as_double((long long)(sg | ((unsigned long long)be << 52) |
                                          (mant & 0xFFFFFFFFFFFFFull)));
}
template <> __device__ __forceinline__ float scaled<float>(long long T, int e) {
  if (T == 0) return 0.0f;
  const unsigned long long sg = (unsigned long long)T & 0x8000000000000000ull;
  unsigned long long a = sg ? 0ull - (unsigned long long)T : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mant = a >> 40;            // 24 bits
  const unsigned long long rem = a & 0xFFFFFFFFFFull;
  mant += (rem + (mant & 1ull)) > (1ull << 39) ? 1ull : 0ull;
  const int be = 63 - lz + e + 127 + (int)(mant >> 24);
  if (be <= 0 || be >= 255) return ldexpf((float)T, e);
  return __uint_as_float((unsigned)(sg >> 32) | ((unsigned)be << 23) |
                         (unsigned)(mant & 0x7FFFFFull));
}
// double-float result: the high part rounded to float from the integer, the low part from the
// exact integer remainder
template <> __device__ __forceinline__ df scaled<df>(long long T, int e) {
  if (T == 0) return df(0.0f, 0.0f);
  const bool neg = T < 0;
  unsigned long long a = neg ? 0ull - (unsigned long long)T : (unsigned long long)T;
  const int lz = __clzll((long long)a);   // |T| < 2^62.3: lz >= 1
  const unsigned long long n = a << lz;
  unsigned long long mant = n >> 40;
  const unsigned long long rem = n & 0xFFFFFFFFFFull;
  mant += (rem + (mant & 1ull)) > (1ull << 39) ? 1ull : 0ull;
  // |T| rounded to 24 significant bits; mant may have rounded up to 2^24, so shift by 39 first
  const unsigned long long ahi = (mant << 39) >> (lz - 1);
  const long long Thi = neg ? -(long long)ahi : (long long)ahi;
  return df(scaled<float>(Thi, e), scaled<float>(T - Thi, e));
}
// the forward transform's last output carries the factor 1 / (2N) (forward outputs are float64)
template <typename TO> __device__ __forceinline__ TO last_scale(TO v, double f) { return v; }
template <> __device__ __forceinline__ double last_scale<double>(double v, double f) {
  return v * f;
}
template <typename TO> __device__ __forceinline__ TO qnan();
template <> __device__ __forceinline__ double qnan<double>() {
  return __longlong_as_double(0x7FF8000000000000ll);
}
template <> __device__ __forceinline__ float qnan<float>() { return __uint_as_float(0x7FC00000u); }
template <> __device__ __forceinline__ df qnan<df>() {
  return df(__uint_as_float(0x7FC00000u), __uint_as_float(0x7FC00000u));
}

constexpr int kBars = 2 * kNB + 2 * kNA + 3;   // barriers (see the kernel)
__host__ __device__ constexpr size_t tc_smem_bytes(int NT) {
  // B planes (kNB chunks), A planes (kNA buffers), row exponents, the barriers and the
  // tensor-memory address, output-column exponents (at most 512)
  return (size_t)kNB * 8 * NT * TCKC * 2 + (size_t)kNA * TCM * TCKC * 2 + TCM * sizeof(int) +
         (size_t)(kBars + 1) * 8 + 512 * sizeof(int);
}

// ---- the transform kernel ---------------------------------------------------------------------
// in / out: nf fields of complex lines (re, im interleaved), field stride fsi / fso complex
// elements, line stride Nz; bdig: nNt output slices of 8 NT Kp bf16 digits (per slice and chunk
// of K: the eight digit planes stacked as one 8 NT x KC matrix in the canonical no-swizzle
// K-major core-matrix layout, plane j in rows j NT ..); fexp: F_n; cache: per CTA, nchunk x 8
// A digit planes of one tile as 7-bit groups, four per 32-bit word (kCacheWords words each).
//
// Persistent CTAs (17 warps) walk the tiles of 128 rows; per tile they loop over the nNt output
// slices.  Warps 0..15 turn the rows into fixed-point values and, for the first slice, write the
// eight digit planes into kNA rotating shared buffers and their groups into the CTA's plane cache
// (each thread reads back only what it wrote, so program order orders the two); for each later
// slice they rebuild its first kNA planes as soon as the previous slice's MMAs are done, drain
// the previous slice's accumulators, then rebuild the rest as the MMAs free the buffers.  Lane 0
// of warp 16 allocates the tensor memory and issues the bulk copies of B and the MMAs.  Plane t
// (counted over tiles, slices and chunks) uses shared buffer t % kNA: its producers wait for
// `empty` of that buffer (the MMAs of plane t - kNA completed, signalled by tcgen05.commit) and
// announce it on `full` (one arrival per producer warp).  The digits of B of chunk u (counted
// over tiles, slices and chunks) go to buffer u % kNB once `bfree` of that buffer says the MMAs
// of chunk u - kNB are done.  A slice's MMAs start once every producer warp has arrived on
// `drained` for the previous slice.
template <typename TI, typename TO, int NT>
__global__ void __launch_bounds__(TCT + 32, 1)
    cheb_tc_kernel(const TI* __restrict__ in, long long fsi, TO* __restrict__ out, long long fso,
                   int nlines, int Nz, int Kp, int tpf, int ntiles, int nNt,
                   const uint16_t* __restrict__ bdig, const int* __restrict__ fexp,
                   uint32_t* __restrict__ cache, int fwd, double lastf, int* __restrict__ err) {
  typedef FBits<TI> F;
  typedef typename F::U U;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sB = tsm;
  constexpr uint32_t kBBytes = 8 * NT * TCKC * 2;   // one chunk of B planes
  unsigned char* sA = sB + (size_t)kNB * kBBytes;
  int* sE = reinterpret_cast<int*>(sA + (size_t)kNA * TCM * TCKC * 2);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(sE + TCM);
  uint32_t* sT = reinterpret_cast<uint32_t*>(bars + kBars);
  int* sF = reinterpret_cast<int*>(bars + kBars + 1);   // F_n of every output column (<= 512)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunk = (Kp + TCKC - 1) / TCKC;
  constexpr uint32_t kPlaneBytes = TCM * TCKC * 2;
  // barriers (8 bytes each, buffer b of a kind at + 8 b): bload[kNB] (B chunk copied),
  // bfree[kNB] (MMAs of the chunk done); full[kNA] (16 producer warps); empty[kNA] (MMAs of the
  // plane done); drained (16 producer warps read the accumulators); sliced (every MMA of a slice
  // done: one phase per slice, so the producers' epilogue waits never alias a buffer's phases);
  // fin (the issuer's MMAs in flight, after a wait ran out)
  const uint32_t barB = su32(&bars[0]), barBfree = su32(&bars[kNB]);
  const uint32_t barFull = su32(&bars[2 * kNB]);
  const uint32_t barEmpty = su32(&bars[2 * kNB + kNA]);
  const uint32_t barDrain = su32(&bars[2 * kNB + 2 * kNA]);
  const uint32_t barSlice = barDrain + 8, barFin = barDrain + 16;
  const size_t bslice = (size_t)8 * NT * Kp;
  uint32_t* ccta = cache + (size_t)blockIdx.x * nchunk * 8 * kCacheWords;
  const bool issuer_warp = (warp == TCT / 32);
  const bool issuer = issuer_warp && lane == 0;
  if (issuer) {
    for (int b = 0; b < kNB; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barB + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barBfree + 8 * b));
    }
    for (int b = 0; b < kNA; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 16;" ::"r"(barFull + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barEmpty + 8 * b));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 16;" ::"r"(barDrain));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barSlice));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barFin));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (issuer_warp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(sT)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < TCT)
    for (int c = tid; c < nNt * NT; c += TCT) sF[c] = fexp[c];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();   // barriers, tensor-memory address and sF visible to every warp
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sT;
  const uint32_t sA0 = su32(sA), sB0 = su32(sB);
  const uint64_t keep = policy_evict_last();
  Waiter W;

  if (issuer_warp) {
    if (lane == 0) {
      // bf16 x bf16 -> fp32, both K-major, M = 128 (N added per MMA)
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCM >> 4) << 24);
      int t = 0, u = 0, S = 0;           // plane, B chunk and slice counters (all tiles)
      int nfull[kNA] = {};
      int nbl[kNB] = {}, ibl[kNB] = {};  // B chunks waited for / issued per buffer
      bool any_mma = false;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int sl = 0; sl < nNt; ++sl, ++S) {
          for (int ch = 0; ch < nchunk; ++ch, ++u) {
            const int KCc = min(TCKC, Kp - ch * TCKC);
            const int bb = u % kNB;
            // B buffer bb: the MMAs of chunk u - kNB read it
            if (u >= kNB && !W.wait(barBfree + 8 * bb, ((u - kNB) / kNB) & 1)) goto drain;
            bulk_load(sB0 + (uint32_t)(bb * kBBytes),
                      bdig + (size_t)sl * bslice + (size_t)ch * 8 * NT * TCKC,
                      (uint32_t)(8 * NT * KCc * 2), barB + 8 * bb, keep);
            ++ibl[bb];
            if (!W.wait(barB + 8 * bb, nbl[bb] & 1)) goto drain;
            ++nbl[bb];
            if (ch == 0 && S > 0 && !W.wait(barDrain, (S - 1) & 1)) goto drain;
            for (int i = 0; i < 8; ++i, ++t) {
              const int bf = t % kNA;
              if (!W.wait(barFull + 8 * bf, nfull[bf] & 1)) goto drain;
              ++nfull[bf];
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              // A plane i times B planes 0 .. 7-i at once: the stacked B rows j NT + n land in
              // accumulator columns i NT + j NT + n = (i + j) NT + n, the diagonal of (i, j).
              // N = (8 - i) NT is issued in pieces of at most 256.  A k-step adds 2 core-matrix
              // groups to both start addresses (4096 bytes of A, 2 NT 128 bytes of B).
              const uint64_t ad = sdesc(sA0 + (uint32_t)(bf * kPlaneBytes), 2048, 128);
              const uint32_t sBb = sB0 + (uint32_t)(bb * kBBytes);
              const int ntot = (8 - i) * NT;
              for (int s = 0; s < KCc / 16; ++s)
                for (int n0 = 0; n0 < ntot; n0 += 256) {
                  const int nlen = min(256, ntot - n0);
                  const uint64_t bd = sdesc(sBb + (uint32_t)(n0 / 8 * 128), NT * 128, 128);
                  mma_bf16(tmem + (uint32_t)(i * NT + n0), ad + (uint64_t)(s * 256),
                           bd + (uint64_t)(s * 16 * NT), idesc0 | ((uint32_t)(nlen >> 3) << 17),
                           (uint32_t)((ch | i | s) != 0));
                }
              any_mma = true;
              mma_commit(barEmpty + 8 * bf);
              if (i == 7) mma_commit(barBfree + 8 * bb);
              if (i == 7 && ch == nchunk - 1) mma_commit(barSlice);
            }
          }
        }
      }
    drain:
      if (!W.ok) {
        // A wait ran out: nothing more is issued.  Before the tensor memory is released and the
        // CTA ends, wait (one shared bound for all of them) for the MMAs and the bulk copies
        // still in flight: the MMAs through one last commit, each copy on its own barrier phase.
        const uint64_t dl = gtime() + kWaitNs;
        if (any_mma) {
          mma_commit(barFin);
          mbar_wait_until(barFin, 0, dl);
        }
        for (int b = 0; b < kNB; ++b)
          if (ibl[b] > nbl[b]) mbar_wait_until(barB + 8 * b, nbl[b] & 1, dl);
      }
    }
    __syncwarp();
  } else {
    // producers: warp = 8-row core-matrix group, lane = (row in the group, pair of k)
    const int r = lane >> 2, q = lane & 3;
    const int m = warp * 8 + r;
    constexpr int CW = NT / 4;
    const int qd = warp & 3, cg = warp >> 2;
    const int mm = qd * 32 + lane;
    const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(cg * CW);
    // the largest exponent field of this thread's row of tile `tl` over all of K (the row's
    // first, cold read)
    auto row_exponent = [&](int tl) {
      const int fld = tl / tpf;
      const int line = (tl - fld * tpf) * (TCM / 2) + (m >> 1);
      const bool rowok = line < nlines;
      const TI* src = in + ((size_t)fld * fsi + (size_t)(rowok ? line : 0) * Nz) * 2 + (m & 1);
      int mx = 1;
      for (int ch = 0; ch < nchunk; ++ch) {
        const int ngc = min(TCKC, Kp - ch * TCKC) / 8;
#pragma unroll
        for (int gl = 0; gl < TCG; ++gl)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = ch * TCKC + 8 * gl + 2 * q + e;
            if (gl < ngc && rowok && k < Nz) mx = max(mx, F::expo(F::bits(src[2 * (size_t)k])));
          }
      }
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      return max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    };
    // L2 prefetch (evict-last) of the row elements of chunk ch of tile tl that this thread
    // converts: issued one chunk ahead, so the conversion's loads, which the registers allow only
    // a few at a time, find the rows in L2 instead of DRAM
    auto prefetch_rows = [&](int tl, int ch) {
      const int fld = tl / tpf;
      const int line = (tl - fld * tpf) * (TCM / 2) + (m >> 1);
      if (line >= nlines) return;
      const TI* src = in + ((size_t)fld * fsi + (size_t)line * Nz) * 2 + (m & 1);
      const int ngp = min(TCKC, Kp - ch * TCKC) / 8;
      for (int gl = 0; gl < ngp; ++gl) {
        const int k = ch * TCKC + 8 * gl + 2 * q;
        if (k < Nz)
          asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(src + 2 * (size_t)k));
      }
    };
    int t = 0, S = 0;
    int ahead = -1;   // the next tile's row exponent, read during this tile's last slice
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int fld = tile / tpf;
      const int line0 = (tile - fld * tpf) * (TCM / 2);
      const int line = line0 + (m >> 1);
      const bool rowok = line < nlines;
      const TI* src = in + ((size_t)fld * fsi + (size_t)(rowok ? line : 0) * Nz) * 2 + (m & 1);
      const int maxe = ahead >= 0 ? ahead : row_exponent(tile);
      ahead = -1;
      // sE: every producer warp has read the previous tile's entries (before its slice loop)
      asm volatile("bar.sync 1, %0;" ::"r"(TCT) : "memory");
      if (q == 0) sE[m] = maxe;
      asm volatile("bar.sync 1, %0;" ::"r"(TCT) : "memory");
      const int me = sE[mm];
      // first slice: generate the planes of every chunk (cached for the later slices); the last
      // output n = N, sum_k w_k X_k with w_k = e_k (-1)^k (forward) or (-1)^k (backward), is
      // summed exactly here as S_hi 2^27 + S_lo
      long long s_hi = 0, s_lo = 0;
      for (int ch = 0; ch < nchunk; ++ch) {
        const int ngr = min(TCKC, Kp - ch * TCKC) / 8;
        uint32_t yh[2 * TCG], yl[2 * TCG];   // bits 28..55 and 0..27 of X + bias
#pragma unroll
        for (int gl = 0; gl < TCG; ++gl)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int k = ch * TCKC + 8 * gl + 2 * q + e;
            U b = 0;
            if (gl < ngr && rowok && k < Nz) b = F::bits(ld_stream(src + 2 * (size_t)k));
            const unsigned long long y = to_biased<TI>(b, maxe);
            yh[2 * gl + e] = (uint32_t)(y >> 28);
            yl[2 * gl + e] = (uint32_t)y & 0xFFFFFFFu;
            if (gl < ngr && k < Nz) {
              const long long xs = (long long)(y - kBias);
              const int w = ((k & 1) ? -1 : 1) * ((fwd && k != 0 && k != Nz - 1) ? 2 : 1);
              s_hi += w * (xs >> 27);
              s_lo += w * (xs & 0x7FFFFFFll);
            }
          }
        if (ch + 1 < nchunk) prefetch_rows(tile, ch + 1);
        for (int i = 0; i < 8; ++i, ++t) {
          const int bf = t % kNA;
          if (t >= kNA) W.wait(barEmpty + 8 * bf, ((t - kNA) / kNA) & 1);
          uint32_t* dst = reinterpret_cast<uint32_t*>(sA + (size_t)bf * kPlaneBytes);
          uint32_t* gdst = ccta + (size_t)(ch * 8 + i) * kCacheWords;
          const int sh = 7 * (3 - (i & 3));
#pragma unroll
          for (int g2 = 0; g2 < TCG / 2; ++g2)
            if (2 * g2 < ngr) {
              const int gl = 2 * g2;
              const uint32_t* yy = i < 4 ? yh : yl;
              dst[(gl * 16 + warp) * 32 + lane] = digit_pair(yy[2 * gl], yy[2 * gl + 1], sh);
              dst[((gl + 1) * 16 + warp) * 32 + lane] =
                  digit_pair(yy[2 * gl + 2], yy[2 * gl + 3], sh);
              // the four 7-bit groups as bytes, read back by this same thread for the later
              // slices (program order: no fence)
              st_hint(gdst + (g2 * 16 + warp) * 32 + lane,
                      pack_groups(yy[2 * gl], yy[2 * gl + 1], yy[2 * gl + 2], yy[2 * gl + 3], sh),
                      keep);
            }
          // the shared-memory plane for the MMAs (async proxy)
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(barFull + 8 * bf)
                         : "memory");
        }
      }
      s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 1);
      s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 1);
      s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 2);
      s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 2);
      if (q == 0 && rowok && W.ok) {
        // sum_k w_k x_k = 2^(E - 54) (S_hi 2^27 + S_lo) = T 2^(E - 51), T = S_hi 2^24 + S_lo / 8
        // (|sum w X| < 2 Kp 2^54 < 2^64, so three low bits are dropped: 2^-51 of the row scale)
        const long long T = s_hi * 16777216ll + (s_lo >> 3);
        TO v = maxe >= F::EMAX ? qnan<TO>() : scaled<TO>(T, maxe - F::EOFF - 51);
        if (fwd) v = last_scale<TO>(v, lastf);
        st_stream(out + ((size_t)fld * fso + (size_t)line * Nz) * 2 + (m & 1) + 2 * (size_t)(Nz - 1),
                  v);
      }
      const int oline = line0 + (mm >> 1);
      TO* dstp =
          out + ((size_t)fld * fso + (size_t)(oline < nlines ? oline : 0) * Nz) * 2 + (mm & 1);
      // the later slices' planes, rebuilt from the packed groups of the first slice: plane c
      // (chunk c / 8, plane c % 8) of the slice that starts at plane number t0s
      const int tplanes = 8 * nchunk;
      int tnext = t;                     // next plane to rebuild (the slice after the current)
      auto rebuild = [&](int upto) {
        for (; tnext < upto; ++tnext) {
          const int c = tnext % tplanes;   // planes of a tile are numbered slice by slice
          const int chc = c >> 3;
          const int ngc = min(TCKC, Kp - chc * TCKC) / 8;
          const int bf = tnext % kNA;
          const uint32_t* gsrc = ccta + (size_t)c * kCacheWords;
          uint32_t wv[TCG / 2];
#pragma unroll
          for (int g2 = 0; g2 < TCG / 2; ++g2)
            wv[g2] = (2 * g2 < ngc) ? ld_keep(gsrc + (g2 * 16 + warp) * 32 + lane, keep) : 0u;
          if (tnext >= kNA) W.wait(barEmpty + 8 * bf, ((tnext - kNA) / kNA) & 1);
          uint32_t* dst = reinterpret_cast<uint32_t*>(sA + (size_t)bf * kPlaneBytes);
#pragma unroll
          for (int g2 = 0; g2 < TCG / 2; ++g2)
            if (2 * g2 < ngc) {
              const int gl = 2 * g2;
              dst[(gl * 16 + warp) * 32 + lane] = group_pair(wv[g2] & 0xFFFFu);
              dst[((gl + 1) * 16 + warp) * 32 + lane] = group_pair(wv[g2] >> 16);
            }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(barFull + 8 * bf)
                         : "memory");
        }
      };
      for (int sl = 0; sl < nNt; ++sl, ++S) {
        if (sl == nNt - 1 && tile + (int)gridDim.x < ntiles) prefetch_rows(tile + gridDim.x, 0);
        // every MMA of the slice done
        W.wait(barSlice, S & 1);
        // the next slice's first planes into the buffers its MMAs start with (free now)
        if (sl + 1 < nNt) rebuild(t + min(kNA, tplanes));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its rows), columns
        // (w / 4) NT/4 .. + NT/4 - 1 of each of the eight accumulators, 4 at a time (after a
        // failed wait the producers keep their loop structure, which their named barrier
        // needs, but wait no more and store nothing)
        const bool orow = W.ok && oline < nlines;
        for (int c0 = 0; c0 < CW; c0 += 4) {
          uint32_t v[8][4];
          tmem_ld8x4(tb + (uint32_t)c0, NT, v);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int n = sl * NT + cg * CW + c0 + e;
            if (orow && n < Nz - 1) {
              int g[8];
              if (Kp <= kSmallK) {
#pragma unroll
                for (int d = 0; d < 8; ++d) g[d] = acc_int_small(v[d][e]);
              } else {
#pragma unroll
                for (int d = 0; d < 8; ++d) g[d] = acc_int(v[d][e]);
              }
              const long long H = ((long long)(g[0] * 128 + g[1]) * 128 + g[2]) * 128 + g[3];
              const long long L = ((long long)(g[4] * 128 + g[5]) * 128 + g[6]) * 128 + g[7];
              const long long T = H * 262144ll + (L >> 10);   // (H 2^28 + L) / 2^10
              // sum = 2^(E + F - 108) 2^49 (H 2^28 + L) = T 2^(E + F - 49)
              st_stream(dstp + 2 * (size_t)n,
                        me >= F::EMAX ? qnan<TO>() : scaled<TO>(T, me - F::EOFF - 49 + sF[n]));
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(barDrain) : "memory");
        // the rest of the next slice's planes, as its MMAs free the buffers
        if (sl + 1 < nNt) {
          rebuild(t + tplanes);
          t += tplanes;
        }
        // while the last slice's MMAs run: the next tile's cold row read
        if (sl == nNt - 2 && tile + (int)gridDim.x < ntiles) ahead = row_exponent(tile + gridDim.x);
      }
    }
  }
  if (!W.ok) atomicOr(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (issuer_warp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <typename TI, typename TO, int NT>
cudaError_t launch_t(const void* in, long long fsi, void* out, long long fso, int nf, int nlines,
                     int Nz, const ChebTc& t, int* err, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(NT);
  const int tpf = (nlines + TCM / 2 - 1) / (TCM / 2);
  const long long ntiles = (long long)nf * tpf;
  if (ntiles <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, t.ctas);
  cheb_tc_kernel<TI, TO, NT><<<grid, TCT + 32, smem, s>>>(
      (const TI*)in, fsi, (TO*)out, fso, nlines, Nz, t.Kp, tpf, (int)ntiles, t.nNt, t.dig,
      t.fexp, t.cache, t.dir == 0 ? 1 : 0, t.dir == 0 ? 0.5 / (double)(Nz - 1) : 1.0, err);
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
  // the MMAs produce outputs n < N (the last one, n = N, has the weights +-1, +-2 and is summed
  // exactly by the kernel's producers); output slice width 48 or 64, whichever pads less after
  // weighting 48-wide slices by 5/4 (more MMA instructions per column)
  const int c48 = (N + 47) / 48 * 48, c64 = (N + 63) / 64 * 64;
  NT = (5 * c48 <= 4 * c64) ? 48 : 64;
  nNt = (N + NT - 1) / NT;
  if (nNt * NT > 512) return -1;   // the kernel keeps F_n of at most 512 columns
  dig.assign((size_t)nNt * 8 * NT * Kp, 0);
  fexp.assign((size_t)nNt * NT, 0);
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> row(Nz);
  std::vector<long long> Y(Nz);
  for (int n = 0; n < N; ++n) {
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
      (void)KCc;
      for (int j = 0; j < 8; ++j) {
        // plane j occupies rows j NT .. j NT + NT - 1 of one 8 NT-row K-major matrix
        const int row = j * NT + nl;
        const size_t off = ((size_t)(kl / 8) * NT + row / 8) * 64 + (row % 8) * 8 + kl % 8;
        const int d = (int)((yb >> (7 * (7 - j))) & 127ull) - 64;
        dig[base + off] = bf16_bits((float)d);
      }
    }
  }
  return 0;
}

size_t cheb_tc_smem(int NT) { return tc_smem_bytes(NT); }

size_t cheb_tc_cache_bytes(int Kp) {
  return (size_t)((Kp + TCKC - 1) / TCKC) * 8 * kCacheWords * sizeof(uint32_t);
}

cudaError_t cheb_tc_prepare(int NT) {
  const size_t smem = tc_smem_bytes(NT);
  cudaError_t e = cudaSuccess;
  if (NT == 48) {
    static SmemLimit c0, c1, c2, c3, c4;
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, double, 48>, smem, &c0);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<float, double, 48>, smem, &c1);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, float, 48>, smem, &c2);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<df, double, 48>, smem, &c3);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, df, 48>, smem, &c4);
  } else {
    static SmemLimit c0, c1, c2, c3, c4;
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, double, 64>, smem, &c0);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<float, double, 64>, smem, &c1);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, float, 64>, smem, &c2);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<df, double, 64>, smem, &c3);
    if (e == cudaSuccess) e = ensure_smem(cheb_tc_kernel<double, df, 64>, smem, &c4);
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
  if (tin == 2 && tout == 0)
    return launch_nt<df, double>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
  if (tin == 0 && tout == 2)
    return launch_nt<double, df>(in, fsi, out, fso, nf, nlines, Nz, t, err, s);
  return cudaErrorInvalidValue;
}

// Failure path of the bounded waits, exercised on purpose: one thread runs a loop of `nwaits`
// waits of the transform's shape (the same Waiter, alternating the parities of two mbarriers)
// on barriers that nothing arrives at.  The first wait gives up after kWaitNs and every later
// one returns at once, so the kernel ends after about one bound however long the loop; the
// thread records the failure in err[0] and the number of waits that actually spun in err[1].
// No TMEM and no asynchronous copy is involved, so nothing else is left in flight.
__global__ void __launch_bounds__(32) wait_selftest_kernel(int* __restrict__ err, int nwaits) {
  __shared__ __align__(8) uint64_t bar[2];
  if (threadIdx.x != 0) return;
  const uint32_t b0 = su32(&bar[0]), b1 = su32(&bar[1]);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b1));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  Waiter W;
  int spun = 0;
  for (int i = 0; i < nwaits; ++i) {
    if (W.ok) ++spun;
    W.wait((i & 1) ? b1 : b0, (uint32_t)((i >> 1) & 1));
  }
  if (!W.ok) atomicOr(&err[0], 1);
  atomicAdd(&err[1], spun);
}

// Eight independent float64 FMA chains per thread (enough to cover the pipe's latency): x <- x
// a + b with |a| < 1, so the values stay bounded; the sum is stored so nothing is dead code.
__global__ void __launch_bounds__(256) fma_probe_kernel(double* __restrict__ out, int iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1e-3 * (t + i);
  const double a = 0.999999, b = 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[t] = s;
}

cudaError_t launch_fma_probe(double* out, int blocks, int iters, cudaStream_t s) {
  fma_probe_kernel<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* err, int nwaits, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(err, nwaits);
  return cudaGetLastError();
}

}  // namespace chf
