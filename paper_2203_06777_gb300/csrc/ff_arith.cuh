// Float-float ("double-float") arithmetic for the FP64 kernels: every real carried as an
// unevaluated sum hi + lo of two FP32 numbers, after Dekker ("A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971): sums by Knuth's error-free TwoSum,
// products by the FMA-based TwoProduct (the rounding error of a*b is fma(a, b, -a*b) exactly).
// A value carries about 46-47 significant bits; its exponent range is FP32's.
//
// Also: the FP64 <-> float-float conversions done with integer operations (conversions through
// the FP64 pipe would cost as much as the FP64 arithmetic these kernels avoid), and the spin
// projection / reconstruction tables that let a rolled hop loop run one code path for every
// direction.
#pragma once

#include "dwf_common.cuh"

namespace gdwf {
namespace ffa {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) {
  ff r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// s + e == a + b exactly, for any a, b (Knuth's TwoSum, six additions).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Renormalise hi + lo with |hi| >= |lo| (Dekker's FastTwoSum, three additions).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }

// a + SG b (SG = +1 or -1 at compile time): TwoSum of the leading parts, the trailing parts added
// to its error, one renormalisation (eleven instructions).
template <int SG>
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float bh = SG > 0 ? b.hi : -b.hi, bl = SG > 0 ? b.lo : -b.lo;
  float e;
  const float s = two_sum(a.hi, bh, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, bl));
  return fast_two_sum(s, e);
}

// a * b: TwoProduct of the leading parts plus the two cross terms (seven instructions).
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// Dot-product accumulator S + E: the products' leading parts are summed with TwoSum into S, all
// rounding errors and cross terms in FP32 into E; S + E is passed on unnormalised.
struct ffacc {
  float s, e;
};

__device__ __forceinline__ void dot_first(ffacc& A, ff a, ff b, bool neg) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  A.s = neg ? -p : p;
  A.e = neg ? -e : e;
}

// A += SG a b (twelve instructions).
template <int SG>
__device__ __forceinline__ void dot_add(ffacc& A, ff a, ff b) {
  const float ah = SG > 0 ? a.hi : -a.hi, al = SG > 0 ? a.lo : -a.lo;
  const float p = __fmul_rn(ah, b.hi);
  float e = __fmaf_rn(ah, b.hi, -p);
  e = __fmaf_rn(ah, b.lo, e);
  e = __fmaf_rn(al, b.hi, e);
  float t;
  A.s = two_sum(A.s, p, t);
  A.e = __fadd_rn(A.e, __fadd_rn(t, e));
}

// acc += v for an accumulator kept unnormalised across the eight hops (TwoSum of the leading
// parts, the trailing parts summed in FP32; eight instructions instead of an ff_add's eleven),
// renormalised once at the end. v itself may be unnormalised (a dot product's S and E).
__device__ __forceinline__ void acc_add(ff& acc, ff v) {
  float t;
  acc.hi = two_sum(acc.hi, v.hi, t);
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, v.lo));
}

// FP64 -> float-float with integer operations only (conversions through the FP64 pipe would cost
// as much as the FP64 arithmetic this kernel avoids). hi takes the sign, the exponent and the
// leading 23 stored mantissa bits (truncated); lo the next 23 bits, formed as (1.f x 2^k) - 2^k,
// which is exact. Values of magnitude below 2^-103 give 0; above FP32's range, infinity.
__device__ __forceinline__ ff ff_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t H = (uint32_t)(b >> 32), L = (uint32_t)b;
  const uint32_t sgn = H & 0x80000000u;
  const uint32_t mag = H & 0x7FFFFFFFu;  // exponent and leading 20 mantissa bits
  // mantissa bits 51..29 below a 9-bit window of the exponent; adding 2^30 rebiases that window
  // from FP64 (1023) to FP32 (127) for every exponent in FP32's normal range
  const uint32_t hb = __funnelshift_l(L, H, 3) + 0x40000000u;  // bit 31 clear when in range
  const uint32_t pe = (hb & 0x7F800000u) - (23u << 23);  // 2^k with k = exponent(hi) - 23
  const float lo = __fsub_rn(__uint_as_float(sgn | pe | ((L >> 6) & 0x7FFFFFu)), __uint_as_float(sgn | pe));
  // exponent of x in [920, 1150] (FP64 bias): both parts exact as above
  const bool in_range = mag - (920u << 20) < ((1151u - 920u) << 20);
  const bool big = mag >= (1151u << 20);
  const uint32_t hi_bits = in_range ? (sgn | hb) : (big ? (sgn | 0x7F800000u) : sgn);
  return ff_make(__uint_as_float(hi_bits), in_range ? lo : 0.f);
}

// FP32 -> FP64 with integer operations (exact; FP32 subnormals read as zero).
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sgn = b & 0x80000000u;
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t hb = sgn | ((e + 896u) << 20) | ((b >> 3) & 0xFFFFFu);
  const uint32_t H = e == 0 ? sgn : (e == 255 ? (sgn | 0x7FF00000u | ((b & 0x7FFFFFu) ? 0x80000u : 0u)) : hb);
  const uint32_t L = (e == 0 || e == 255) ? 0u : (b << 29);
  return __hiloint2double((int)H, (int)L);
}

// The value hi + lo rounded to FP64 (one FP64 addition).
__device__ __forceinline__ double ff_to_double(ff v) { return widen(v.hi) + widen(v.lo); }

__device__ __forceinline__ ff ff_const(double x) { return ff_from_double(x); }

// ---------------------------------------------------------------- spin projection tables
// Chiral basis, SIG = +1 applying 1 + gamma_mu (the conventions of project / accumulate in
// dhop_kernel.cuh), written so that one code path serves every direction: the projection is
// h_k = psi_k + w_k psi_{p_k} (k = 0, 1; w_k in {+-1, +-i}, p_k in {2, 3}) and the reconstruction
// of the lower spins acc_{2+j} += w'_j uh_{q_j}; the kernels read the right parts at
// direction-dependent addresses and flip signs by the tables below.

// Multiplication by w in {+1, -1, +i, -i} (codes 0..3; code ^ 1 negates w): w (x + iy) takes
// its real part from x or y (swap) and flips the sign of either part.
struct WMul {
  bool swap;
  uint32_t nr, ni;  // 0x80000000 where the real / imaginary part is negated
};

__device__ __forceinline__ WMul wmul(int code) {
  WMul w;
  w.swap = code >= 2;                                        // +i: (-y, x), -i: (y, -x)
  w.nr = (code == 1 || code == 2) ? 0x80000000u : 0u;
  w.ni = (code == 1 || code == 3) ? 0x80000000u : 0u;
  return w;
}

// Codes of w per (mu, k), two bits each at bit 4 mu + 2 k, for projector sign S = +1 (S = -1: ^ 1).
constexpr uint32_t pack_w(int a0, int a1, int b0, int b1, int c0, int c1, int d0, int d1) {
  return (uint32_t)(a0 | a1 << 2 | b0 << 4 | b1 << 6 | c0 << 8 | c1 << 10 | d0 << 12 | d1 << 14);
}
// projection h_k = psi_k + w_k psi_{p_k}, p = (3, 2) for mu < 2, else (2, 3):
//   mu = 0: (-i, -i); 1: (-1, +1); 2: (-i, +i); 3: (+1, +1)
constexpr uint32_t PROJ_W = pack_w(3, 3, 1, 0, 3, 2, 0, 0);
// reconstruction of the lower spins, acc[2 + j] += w'_j uh_{q_j}, q = (1, 0) for mu < 2, else (0, 1):
//   mu = 0: (+i, +i); 1: (+1, -1); 2: (+i, -i); 3: (+1, +1)
constexpr uint32_t RECON_W = pack_w(2, 2, 0, 1, 2, 3, 0, 0);

__device__ __forceinline__ int w_code(uint32_t table, int mu, int k, int S) {
  return (int)((table >> (4 * mu + 2 * k)) & 3u) ^ (S < 0 ? 1 : 0);
}

__device__ __forceinline__ ff flip(ff v, uint32_t n) {
  return ff_make(__uint_as_float(__float_as_uint(v.hi) ^ n), __uint_as_float(__float_as_uint(v.lo) ^ n));
}

// One real of an FP64 field with its sign bit flipped by `neg` (0 or 0x80000000).
__device__ __forceinline__ double ld64(const char* p, uint32_t neg) {
  const double d = __ldg(reinterpret_cast<const double*>(p));
  return __hiloint2double(__double2hiint(d) ^ (int)neg, __double2loint(d));
}

// h = the two upper spins of (1 + S gamma_mu) psi for one slice of an FP64 field: blk points at
// the slice's first real (site block + 8 s), cs is the byte stride between reals. The
// additions run in FP64 (one instruction each; the stored reals are FP64), then each projected
// real is split once.
__device__ __forceinline__ void project_load_ff(const char* blk, int mu, int S, size_t cs, ff* h) {
  const WMul w0 = wmul(w_code(PROJ_W, mu, 0, S)), w1 = wmul(w_code(PROJ_W, mu, 1, S));
  const int p0 = mu < 2 ? 3 : 2, p1 = 5 - p0;
  // lower spin p_k: the real slot reads the imaginary part when w_k is imaginary, and vice versa
  const char* l0 = blk + (size_t)(p0 * 6 + (w0.swap ? 1 : 0)) * cs;
  const char* l1 = blk + (size_t)(p1 * 6 + (w1.swap ? 1 : 0)) * cs;
  const ptrdiff_t o0 = w0.swap ? -(ptrdiff_t)cs : (ptrdiff_t)cs;
  const ptrdiff_t o1 = w1.swap ? -(ptrdiff_t)cs : (ptrdiff_t)cs;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t cc = (size_t)(2 * c) * cs;
    h[(0 * 3 + c) * 2] = ff_from_double(ld64(blk + cc, 0u) + ld64(l0 + cc, w0.nr));
    h[(0 * 3 + c) * 2 + 1] = ff_from_double(ld64(blk + cc + cs, 0u) + ld64(l0 + cc + o0, w0.ni));
    h[(1 * 3 + c) * 2] = ff_from_double(ld64(blk + 6 * cs + cc, 0u) + ld64(l1 + cc, w1.nr));
    h[(1 * 3 + c) * 2 + 1] = ff_from_double(ld64(blk + 7 * cs + cc, 0u) + ld64(l1 + cc + o1, w1.ni));
  }
}

}  // namespace ffa
}  // namespace gdwf
