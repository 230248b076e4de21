// clmath.cuh -- device arithmetic for the exact skip length of Algorithm 1.
//
// The skip of Algorithm 1 is delta = floor(ln r / ln(1 - p)).  This library
// defines delta as the floor of that exact real number (r = (2k+1)/2^53,
// p = Q/S with integers Q < S), and evaluates it in two tiers:
//
//   1. float-float (pairs of FP32, ~46 bits): x = L_r / L_p with
//      L_r = -ln(r), L_p = -ln(1 - p); accepted when x is farther than
//      2^-40 x from an integer.  FP64 runs at 1/75 of FP32 on this GPU, so the
//      per-candidate path uses only FP32 and integer pipes.
//   2. double-double (~104 bits) when tier 1 cannot decide; accepted when x is
//      farther than 2^-96 x from an integer; otherwise the nearest integer is
//      taken (which is right when x is exactly an integer) and counted.
//
// Both logarithms are of a ratio of integers, -ln(A/B) with 1 <= A < B,
// computed by table-driven argument reduction (Tang, ACM TOMS 15(2), 1989/90)
// and the atanh series:
//   A' = A 2^e near B;  J = round(64 A'/B);
//   -ln(A/B) = e ln2 + ln(64/J) - 2 atanh(s),  s = (64A' - JB) / (64A' + JB),
// where s is formed from exact integers, so no cancellation is lost for
// p -> 0 (A -> B) or p -> 1 (A -> 0), and |s| <= ~1/127.  The float-float
// tier evaluates both logarithms of a skip on one branch-free path (a warp's
// lanes hold very different p, and a branch on p's size would run both sides
// for the whole warp); the table has 97 entries, ~800 bytes, so a warp's
// divergent lookups touch few L1 lines.
//
// Float-float and double-double arithmetic follow Dekker (1971) and Knuth
// (TAOCP vol. 2, 4.2.2): error-free TwoSum, TwoProd via fused multiply-add.
#pragma once
#include <cstdint>

#include "cl_internal.cuh"
#include "ln_tables.h"

namespace cl {

// ----------------------------------------------------------------- float-float
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = ff_two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, p.lo);
  p.lo = fmaf(x.lo, y.hi, p.lo);
  return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  ff p = ff_two_prod(x.hi, y);
  p.lo = fmaf(x.lo, y, p.lo);
  return ff_fast_two_sum(p.hi, p.lo);
}
// 1/y for a normal float y > 0: the hardware approximation (rcp.approx, at
// most one ulp off) refined by one Newton-Raphson step r + r (1 - y r), which
// leaves it within about one ulp of 1/y at the cost of two FMAs.
__device__ __forceinline__ float rcp_nr(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return fmaf(r, fmaf(-y, r, 1.0f), r);
}
// x / y (y > 0): first quotient q1 = x.hi / y.hi from the reciprocal; the
// residual x - q1 y formed with FMAs (x.hi - q1 y.hi is rounded once, at
// ~2^-23 |x|), second quotient from it.  Relative error below ~2^-44.
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  const float r = rcp_nr(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  float e = fmaf(-q1, y.hi, x.hi);
  e = __fadd_rn(e, x.lo);
  e = fmaf(-q1, y.lo, e);
  return ff_fast_two_sum(q1, __fmul_rn(e, r));
}
// ---- integer -> float without conversion instructions.  On this GPU the
// int<->float conversion instructions share the slow FP64-class pipe, so the
// per-candidate path builds floats from integer bits instead: the float with
// biased exponent 150 + k and significand bits x (0 <= x < 2^23) is exactly
// 2^(23+k) + x 2^k, so subtracting 2^(23+k) leaves x 2^k exactly.  For
// u23_to_f (exponent field 150, its lowest bit clear) x = 2^23 works too: the
// or-ed bit lands in the exponent and gives 2^24.
__device__ __forceinline__ float u23_to_f(unsigned x) {
  return __fsub_rn(__int_as_float(0x4B000000u | x), 8388608.0f);
}
__device__ __forceinline__ float u23_to_f_2p23(unsigned x) {  // x 2^23
  return __fsub_rn(__int_as_float(0x56800000u | x), 0x1p46f);
}
__device__ __forceinline__ float u23_to_f_2p46(unsigned x) {  // x 2^46
  return __fsub_rn(__int_as_float(0x62000000u | x), 0x1p69f);
}
// unsigned 64-bit integer to float-float from three exact 23-bit chunks: the
// top two sum exactly (FastTwoSum, the larger first), the third is added with
// one rounding.  Exact below 2^46; relative error below 2^-46.4 above.
__device__ __forceinline__ ff ff_from_u64(unsigned long long x) {
  const float f2 = u23_to_f_2p46((unsigned)(x >> 46));
  const float f1 = u23_to_f_2p23((unsigned)(x >> 23) & 0x7FFFFFu);
  const float f0 = u23_to_f((unsigned)x & 0x7FFFFFu);
  ff s = ff_fast_two_sum(f2, f1);
  s.lo = __fadd_rn(s.lo, f0);
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_from_i64(long long v) {
  ff r = ff_from_u64((unsigned long long)(v < 0 ? -v : v));
  return v < 0 ? ff{-r.hi, -r.lo} : r;
}

// a + b + c for the three terms of a reduced logarithm: a = e ln2 >= 0,
// b = a table entry in [0, ln2] (so a >= b or a = 0), c = -2 atanh(s) with
// |c| < a + b unless a + b = 0 (then the result is c): the leading parts sum
// exactly in two FastTwoSum steps, all trailing parts and errors are added
// once, one renormalization; the sum loses at most a bit to cancellation.
__device__ __forceinline__ ff ff_sum3(ff a, ff b, ff c) {
  const ff h = ff_fast_two_sum(a.hi, b.hi);
  const ff h2 = ff_fast_two_sum(h.hi, c.hi);
  const float lo = __fadd_rn(__fadd_rn(h.lo, h2.lo), __fadd_rn(__fadd_rn(a.lo, b.lo), c.lo));
  return ff_fast_two_sum(h2.hi, lo);
}

// e ln2 + ln(64/J) - 2 atanh(s) for |s| <= 1/127, J in [32, 128], e >= 1 when
// J > 64 (then written (e - 1) ln2 + ln(128/J), so both leading terms are
// non-negative and are added without cancellation; with |2 atanh s| at most
// about half of ln(64/J) or ln(128/J) for J != 64, 128, the last sum loses at
// most one bit).
//   atanh(s) = s + s m,  m = z (1/3 + z/5 + z^2/7),  z = s^2,
// dropped terms below 2^-59 |s|; |m| < 2^-15.6, so m is needed to ~2^-32 only:
// z/3 as a pair (exact product error, the lo parts of z and 1/3), the rest in
// float.
__device__ __forceinline__ ff ff_log_tail(ff s, int e, int J) {
  const float z = __fmul_rn(s.hi, s.hi);
  const float zl = fmaf(2.0f * s.hi, s.lo, fmaf(s.hi, s.hi, -z));
  const float tail = __fmul_rn(z, fmaf(z, 1.0f / 7.0f, 1.0f / 5.0f));
  const float mh = __fmul_rn(z, CL_THIRD_FF_HI);
  float ml = fmaf(z, CL_THIRD_FF_HI, -mh);
  ml = fmaf(z, __fadd_rn(CL_THIRD_FF_LO, tail), ml);
  ml = fmaf(zl, CL_THIRD_FF_HI, ml);
  const float ch = __fmul_rn(s.hi, mh);
  float cl = fmaf(s.hi, mh, -ch);
  cl = fmaf(s.hi, ml, cl);
  cl = fmaf(s.lo, mh, cl);
  ff at = ff_fast_two_sum(s.hi, ch);  // |ch| < 2^-15 |s.hi|
  at.lo = __fadd_rn(at.lo, __fadd_rn(s.lo, cl));
  const float2 t = __ldg(&CL_LNT2_FF[J - 32]);
  const float2 le = __ldg(&CL_ELN2_FF[e - (J > 64 ? 1 : 0)]);  // (e or e - 1) ln2, below 53 ln2
  return ff_sum3(ff{le.x, le.y}, ff{t.x, t.y}, ff{-2.0f * at.hi, -2.0f * at.lo});
}

// -ln r for r = A / 2^53, A odd in [1, 2^53) (Tang's reduction with a
// power-of-two denominator and a 513-entry table): A' = A 2^e in [2^52, 2^53),
// J = round(A' / 2^43) in [512, 1024], N = A' - J 2^43 in [-2^42, 2^42)
// (exact as float-float),
//   -ln r = e ln2 + ln(1024/J) - 2 atanh(s),  s = N / (J 2^44 + N),  |s| < 2^-11,
// so atanh(s) = s + s z (1/3 + z/5), z = s^2, needs float only past s itself
// (the next term is below 2^-66 |s|).  ln(1024/J) - 2 atanh(s) loses at most
// one bit to cancellation for J < 1024; J = 1024 has no table term.
__device__ __forceinline__ ff ff_neglog_r53(unsigned long long A) {
  const int e = __clzll(A) - 11;
  const unsigned long long Ap = A << e;
  const int J = (int)((Ap + (1ull << 42)) >> 43);
  const long long N = (long long)Ap - ((long long)J << 43);
  const unsigned long long a = (unsigned long long)(N < 0 ? -N : N);  // <= 2^42: 21-bit chunks
  ff Nf = ff_fast_two_sum(__fmul_rn(u23_to_f((unsigned)(a >> 21)), 0x1p21f), u23_to_f((unsigned)a & 0x1FFFFFu));
  if (N < 0) Nf = ff{-Nf.hi, -Nf.lo};
  // J 2^44 + N: the first sum is exact (|N| <= 2^42 < J 2^44), the second rounds once,
  // below 2^-47 of the total
  ff Df = ff_fast_two_sum(__fmul_rn(u23_to_f((unsigned)J), 0x1p44f), Nf.hi);
  Df.lo = __fadd_rn(Df.lo, Nf.lo);
  const ff s = ff_div(Nf, Df);
  const float z = __fmul_rn(s.hi, s.hi);
  const float poly = __fmul_rn(z, fmaf(z, 0.2f, 1.0f / 3.0f));
  const ff at{s.hi, fmaf(s.hi, poly, s.lo)};
  const float2 t = __ldg(&CL_LNR_FF[J - 512]);
  const float2 le = __ldg(&CL_ELN2_FF[e]);  // e ln2, e <= 52
  return ff_sum3(ff{le.x, le.y}, ff{t.x, t.y}, ff{-2.0f * at.hi, -2.0f * at.lo});
}

// -ln r for r = (2k+1)/2^53 with k the top 52 bits of the word pair (hi:lo), the
// same reduction on 32-bit pieces: A = 2k+1 = hi 2^21 + a21 with a21 = ((lo >>
// 12) << 1) | 1 (21 bits); for hi >= 2^10 (all but 2^-22 of the draws) A' = A 2^e,
// e = clz(hi) <= 21, has its 32 top bits t = (hi << e) | (a21 >> (21 - e)) and low
// 21 bits l = (a21 << e) mod 2^21; J = round(A' / 2^43) = (t >> 22) + bit 21 of t;
// N = A' - J 2^43 = Nh 2^21 + l with Nh = t - J 2^22 in [-2^21, 2^21] (wrapping
// 32-bit arithmetic gives it exactly), which is exact as float-float.  The rest is
// that of ff_neglog_r53; smaller hi takes ff_neglog_r53 itself.
__device__ __forceinline__ ff ff_neglog_r53_w(unsigned lo, unsigned hi) {
  if (hi < (1u << 10)) return ff_neglog_r53(2ull * ((((unsigned long long)hi << 32) | lo) >> 12) + 1ull);
  const int e = __clz(hi);
  const unsigned a21 = ((lo >> 12) << 1) | 1u;
  const unsigned t = (hi << e) | (a21 >> (21 - e));
  const unsigned l = (a21 << e) & 0x1FFFFFu;
  const unsigned J = (t >> 22) + ((t >> 21) & 1u);  // in [512, 1024]
  const int Nh = (int)(t - (J << 22));               // in [-2^21, 2^21]
  const float nh = __fmul_rn(__fsub_rn(u23_to_f((unsigned)(Nh + (1 << 22))), 4194304.0f), 0x1p21f);  // Nh 2^21, exact
  const ff Nf = ff_fast_two_sum(nh, u23_to_f(l));  // |nh| >= 2^21 > l, or nh = 0
  // J 2^44 + N: the first sum is exact (|N| <= 2^42 < J 2^44), the second rounds once
  ff Df = ff_fast_two_sum(__fmul_rn(u23_to_f(J), 0x1p44f), Nf.hi);
  Df.lo = __fadd_rn(Df.lo, Nf.lo);
  const ff s = ff_div(Nf, Df);
  const float z = __fmul_rn(s.hi, s.hi);
  const float poly = __fmul_rn(z, fmaf(z, 0.2f, 1.0f / 3.0f));
  const ff at{s.hi, fmaf(s.hi, poly, s.lo)};
  const float2 tb = __ldg(&CL_LNR_FF[J - 512]);
  const float2 le = __ldg(&CL_ELN2_FF[e]);
  return ff_sum3(ff{le.x, le.y}, ff{tb.x, tb.y}, ff{-2.0f * at.hi, -2.0f * at.lo});
}

// -ln(1 - Q/S) = -ln(A/S), A = S - Q, for integers 0 < Q < S < 2^53; one path
// for every p (no branch on its size, so lanes of a warp stay converged):
//   A' = A 2^e with S's leading bit, A'/S in (1/2, 2);  J = round(64 A'/S)
//   in [32, 128] (from 23-bit leading parts, off by at most 2^-13.7 before
//   rounding);  N = 64 A' - J S, D = 64 A' + J S exactly in 64-bit integers;
//   -ln(A/S) = e ln2 + ln(64/J) - 2 atanh(N/D).
// For p < 1/2048 this is e = 0, J = 64, N = -64 Q: the pure atanh series,
// with full relative precision however small p is.
// e ln2 - ln(Ap / B) for integers Ap, B < 2^53 of the same bit length (Ap / B in
// (1/2, 2)), e >= 0, and e >= 1 when Ap > B: J = round(64 Ap / B) from the
// 23-bit leading part (B >> sh) and cB = 64 / (B >> sh); N = 64 Ap - J B and
// D = 64 Ap + J B exact in 64-bit integers; the tail as described above.
__device__ __forceinline__ ff ff_neglog_reduced(unsigned long long Ap, unsigned long long B, int e, int sh, float cB) {
  const float q = __fmul_rn(u23_to_f((unsigned)(Ap >> sh)), cB);
  int J = __float_as_int(__fadd_rn(q, 12582912.0f)) - 0x4B400000;  // round to nearest
  J = J < 32 ? 32 : (J > 128 ? 128 : J);
  const unsigned long long JB = (unsigned long long)(unsigned)J * B;
  const unsigned long long A64 = Ap << 6;
  return ff_log_tail(ff_div(ff_from_i64((long long)(A64 - JB)), ff_from_u64(A64 + JB)), e, J);
}

__device__ __forceinline__ ff ff_neglog1m_table(unsigned long long Q, unsigned long long S, const LpConst& c) {
  const unsigned long long A = S - Q;
  const int e = __clzll(A) - c.zS;
  return ff_neglog_reduced(A << e, S, e, c.sh, c.cS);
}

// ------------------------------------------------------------- double-double
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd dd_fast_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  dd t = dd_two_sum(x.lo, y.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return dd_fast_two_sum(s.hi, s.lo);
}
// Dekker's double-double sum: one TwoSum of the leading parts, the trailing
// parts added with one rounding (relative error about 2^-104 of |x| + |y|: as
// accurate as dd_add for terms of one sign, with half its operations).
__device__ __forceinline__ dd dd_add_dekker(dd x, dd y) {
  dd s = dd_two_sum(x.hi, y.hi);
  s.lo = __dadd_rn(s.lo, __dadd_rn(x.lo, y.lo));
  return dd_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  dd p = dd_two_prod(x.hi, y.hi);
  p.lo = fma(x.hi, y.lo, p.lo);
  p.lo = fma(x.lo, y.hi, p.lo);
  return dd_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd x, double y) {
  dd p = dd_two_prod(x.hi, y);
  p.lo = fma(x.lo, y, p.lo);
  return dd_fast_two_sum(p.hi, p.lo);
}
// x / y with three quotient digits (each from the exact residual)
__device__ __forceinline__ dd dd_div(dd x, dd y) {
  double q1 = __ddiv_rn(x.hi, y.hi);
  dd r = dd_add(x, dd_mul_d(y, -q1));
  double q2 = __ddiv_rn(r.hi, y.hi);
  r = dd_add(r, dd_mul_d(y, -q2));
  double q3 = __ddiv_rn(r.hi, y.hi);
  dd q = dd_fast_two_sum(q1, q2);
  return dd_add(q, dd{q3, 0.0});
}
__device__ __forceinline__ dd dd_from_i64(long long v) {
  double hi = __ll2double_rn(v);
  return {hi, __ll2double_rn(v - __double2ll_rz(hi))};
}

// -ln(A / B) for integers 1 <= A < B <= 2^55, as double-double.
__device__ __forceinline__ dd dd_neglog_ratio(unsigned long long A, unsigned long long B) {
  int e = __clzll(A) - __clzll(B);
  unsigned long long Ap = A << e;
  if (Ap >= B) {
    Ap >>= 1;
    e -= 1;
  }
  int J = __double2int_rn(64.0 * __ull2double_rn(Ap) / __ull2double_rn(B));
  J = J < 32 ? 32 : (J > 64 ? 64 : J);
  long long N = (long long)(Ap << 6) - (long long)J * (long long)B;
  long long D = (long long)(Ap << 6) + (long long)J * (long long)B;
  dd s = dd_div(dd_from_i64(N), dd_from_i64(D));
  dd z = dd_mul(s, s);
  // sum_{k=0}^{9} z^k / (2k+1), Horner from the top
  dd p = dd{__ldg(&CL_ATANH_DD[9][0]), __ldg(&CL_ATANH_DD[9][1])};
  for (int k = 8; k >= 0; --k) p = dd_add(dd_mul(p, z), dd{__ldg(&CL_ATANH_DD[k][0]), __ldg(&CL_ATANH_DD[k][1])});
  dd at = dd_mul(s, p);
  dd t = dd{__ldg(&CL_LNT_DD[J - 32][0]), __ldg(&CL_LNT_DD[J - 32][1])};
  dd le = dd_mul_d(dd{CL_LN2_DD_HI, CL_LN2_DD_LO}, (double)e);
  dd r = dd_add(le, t);
  return dd_add(r, dd{-2.0 * at.hi, -2.0 * at.lo});
}

// ------------------------------------------------------------ skip decision
// Outcome of one tier: the floor of x clamped at R, or "undecided".
static constexpr long long SKIP_UNDECIDED = -1;

// x = hi + lo >= 0 (a normalized pair, evaluation error below 2^-41 x):
// floor(x) clamped at R, or SKIP_UNDECIDED when x may lie within tau x =
// 2^-40 x of an integer.
//  * hi < 2^23 not an integer: hi is at least ulp(hi) >= 2^-24 hi from every
//    integer while |lo| <= ulp(hi)/2 and the error is far below that, so
//    floor(x) = floor(hi) with no window test (the common case);
//  * hi < 2^23 an integer k: x = k + lo, decided by the sign of lo when
//    |lo| > tau x;
//  * 2^23 <= hi < 2^33: hi is an integer and |lo| <= 2^9; floor(x) =
//    hi + floor(lo), and the fractional part of lo (exact) must be farther than
//    tau x from 0 and 1.
// Floors come from the rounded-down sum with 2^23 or 1.5 2^23 (whose ulp is 1)
// and its bits; no conversion instruction.
__device__ __forceinline__ long long floor_decide_ff(ff x, long long R) {
  if (!(x.hi < 0x1p33f)) return R;  // x >= 2^33 > R for sure
  const float margin = 0x1p-40f * x.hi;
  long long k;
  if (x.hi < 0x1p23f) {
    const float t = __fadd_rd(x.hi, 0x1p23f);  // 2^23 + floor(hi), exact
    k = (long long)(__float_as_int(t) - 0x4B000000);
    if (__fsub_rn(t, 0x1p23f) == x.hi) {  // hi is an integer
      if (x.lo < -margin)
        k -= 1;
      else if (!(x.lo > margin))
        return SKIP_UNDECIDED;
    }
  } else {
    const unsigned b = __float_as_uint(x.hi);
    k = (long long)((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 150u);
    const float tl = __fadd_rd(x.lo, 12582912.0f);  // 1.5 2^23 + floor(lo), exact for |lo| <= 2^9
    const float d = __fsub_rn(x.lo, __fsub_rn(tl, 12582912.0f));  // lo - floor(lo) in [0, 1]
    if (!(d > margin) || !(__fsub_rn(1.0f, d) > margin)) return SKIP_UNDECIDED;
    k += (long long)(__float_as_int(tl) - 0x4B400000);
  }
  return k < R ? k : R;
}

// floor_decide_ff for 1 <= R < 2^31 on 32-bit integers: x_hi < 2^23, nearly every
// skip, is decided here; larger x takes the 64-bit path.
__device__ __forceinline__ int floor_decide_ff32(ff x, int R) {
  if (x.hi < 0x1p23f) {
    const float margin = 0x1p-40f * x.hi;
    const float t = __fadd_rd(x.hi, 0x1p23f);  // 2^23 + floor(hi), exact
    int k = __float_as_int(t) - 0x4B000000;
    if (__fsub_rn(t, 0x1p23f) == x.hi) {  // hi is an integer
      if (x.lo < -margin)
        k -= 1;
      else if (!(x.lo > margin))
        return (int)SKIP_UNDECIDED;
    }
    return k < R ? k : R;
  }
  return (int)floor_decide_ff(x, (long long)R);
}

// Same for double-double with tau = 2^-92 (the tier's evaluation error is below
// 2^-96); an undecided x takes the nearest integer (*tie = true), which is the
// exact floor when x is an integer.
__device__ __forceinline__ long long floor_decide_dd(dd x, long long R, bool* tie) {
  const double tau = 0x1p-92;
  *tie = false;
  if (x.hi > 0x1p40 || x.hi > (double)R * (1.0 + 0x1p-40)) return R;
  double k0 = floor(x.hi);
  dd r = dd_two_sum(__dsub_rn(x.hi, k0), x.lo);
  long long k;
  double dlo, dhi;
  if (r.hi < 0.0) {
    k = (long long)k0 - 1;
    dhi = __dsub_rn(-r.hi, r.lo);
    dlo = __dadd_rn(1.0, r.hi);
  } else if (r.hi > 1.0 || (r.hi == 1.0 && r.lo >= 0.0)) {
    k = (long long)k0 + 1;
    dlo = __dadd_rn(__dsub_rn(r.hi, 1.0), r.lo);
    dhi = __dsub_rn(1.0, dlo);
  } else {
    k = (long long)k0;
    dlo = __dadd_rn(r.hi, r.lo);
    dhi = __dsub_rn(__dsub_rn(1.0, r.hi), r.lo);
  }
  double margin = tau * x.hi;
  if (!(dlo > margin) || !(dhi > margin)) {
    *tie = true;
    if (dhi < dlo) k += 1;  // nearest integer
  }
  return k < R ? k : R;
}

// Tier 1 for double weights: x = L_r / L_p as one double (L_r from float-float,
// L_p from the double logarithm), window 2^-40 x as for float-float.
__device__ __forceinline__ long long floor_decide_d(double x, long long R) {
  const double tau = 0x1p-40;
  if (!(x < 0x1p33)) return R;
  double k0 = floor(x);
  long long k = (long long)k0;
  if (k > R) return R;
  double dlo = x - k0;          // exact
  double dhi = 1.0 - dlo;       // one rounding
  double margin = tau * x;
  if (k >= R) return dlo > margin ? R : SKIP_UNDECIDED;
  if (!(dlo > margin) || !(dhi > margin)) return SKIP_UNDECIDED;
  return k;
}

// -ln(1 - Q/S) for doubles 0 < Q < S, in double: log1p(-Q/S) while Q/S <= 1/2,
// else log((S - Q)/S) with S - Q exact (Sterbenz' lemma).
__device__ __forceinline__ double d_neglog1m(double Q, double S) {
  if (2.0 * Q <= S) return -log1p(-(Q / S));
  return -log((S - Q) / S);
}

// sum_{k=0}^{9} z^k / (2k+1) times s: atanh(s) in double-double, |s| <~ 2^-7
__device__ __forceinline__ dd dd_atanh_small(dd s) {
  dd z = dd_mul(s, s);
  dd p = dd{__ldg(&CL_ATANH_DD[9][0]), __ldg(&CL_ATANH_DD[9][1])};
  for (int k = 8; k >= 0; --k) p = dd_add(dd_mul(p, z), dd{__ldg(&CL_ATANH_DD[k][0]), __ldg(&CL_ATANH_DD[k][1])});
  return dd_mul(s, p);
}

// -ln(1 - Q/S) for doubles 0 < Q < S, in double-double: y = 1 - Q/S (formed as
// (1 - c) - Q/S when Q/S <= 1/2, else as (S - Q)/S with S - Q exact), reduced
// to m = y 2^e in [1/2, 1) and c = J/64, then ln(64/J) + e ln2 - 2 atanh((m-c)/(m+c)).
static __device__ __noinline__ dd dd_neglog1m_f64(double Q, double S) {
  int e = 0;
  int J;
  dd d, den;
  if (2.0 * Q <= S) {
    dd p = dd_div(dd{Q, 0.0}, dd{S, 0.0});
    J = __double2int_rn(64.0 * (1.0 - p.hi));
    J = J < 32 ? 32 : (J > 64 ? 64 : J);
    double c = J / 64.0;
    d = dd_add(dd{1.0 - c, 0.0}, dd{-p.hi, -p.lo});
    den = dd_add(dd{2.0 * c, 0.0}, d);
  } else {
    dd y = dd_div(dd{S - Q, 0.0}, dd{S, 0.0});
    int ex;
    frexp(y.hi, &ex);  // y.hi = f 2^ex, f in [1/2, 1)
    e = -ex;
    dd m = dd{ldexp(y.hi, e), ldexp(y.lo, e)};
    J = __double2int_rn(64.0 * m.hi);
    J = J < 32 ? 32 : (J > 64 ? 64 : J);
    double c = J / 64.0;
    d = dd_add(m, dd{-c, 0.0});
    den = dd_add(m, dd{c, 0.0});
  }
  dd at = dd_atanh_small(dd_div(d, den));
  dd t = dd{__ldg(&CL_LNT_DD[J - 32][0]), __ldg(&CL_LNT_DD[J - 32][1])};
  dd le = dd_mul_d(dd{CL_LN2_DD_HI, CL_LN2_DD_LO}, (double)e);
  return dd_add(dd_add(le, t), dd{-2.0 * at.hi, -2.0 * at.lo});
}

// Tier-2 skip for double weights.
static __device__ __noinline__ long long skip_fallback_dd_f64(unsigned long long Ar, double Q, double S, long long R,
                                                              bool* tie) {
  dd Lr = dd_neglog_ratio(Ar, 1ull << 53);
  dd Lp = dd_neglog1m_f64(Q, S);
  return floor_decide_dd(dd_div(Lr, Lp), R, tie);
}

// Tier-2 skip: x = -ln(Ar / 2^53) / -ln(Ap / S) in double-double.
static __device__ __noinline__ long long skip_fallback_dd(unsigned long long Ar, unsigned long long Ap,
                                                   unsigned long long S, long long R, bool* tie) {
  dd Lr = dd_neglog_ratio(Ar, 1ull << 53);
  dd Lp = dd_neglog_ratio(Ap, S);
  return floor_decide_dd(dd_div(Lr, Lp), R, tie);
}

// -ln(1 - p) for p < 2^-12 (float-float, relative error ~2^-46) by its series
// p (1 + c), c = p/2 + p^2/3 + p^3/4 (the next term, p^4/5, is below 2^-50 p):
// c as a float pair (p/2 exactly, the rest rounded at ~2^-50), p c with an
// exact product of the leading parts.
__device__ __forceinline__ ff ff_neglog1m_series(ff p) {
  const float ch = 0.5f * p.hi;
  const float cl = fmaf(p.hi * p.hi, fmaf(p.hi, 0.25f, 1.0f / 3.0f), 0.5f * p.lo);
  ff pc = ff_two_prod(p.hi, ch);
  pc.lo = fmaf(p.hi, cl, fmaf(p.lo, ch, pc.lo));
  ff L = ff_fast_two_sum(p.hi, pc.hi);
  L.lo = __fadd_rn(L.lo, __fadd_rn(p.lo, pc.lo));
  return L;
}

// -ln(1 - Q/S), 0 < Q < S < 2^53: the series for p < 2^-12 (most candidates
// of a power-law graph; lanes of a warp mostly agree), with p = Q (1/S) as
// float-float (Q exact, 1/S to ~2^-48); the table otherwise.
__device__ __forceinline__ ff ff_neglog1m(unsigned long long Q, unsigned long long S, const LpConst& c) {
  if (Q < c.Ssmall) {  // Q < S / 4096 < 2^41: two exact 23-bit chunks
    const ff q = ff_fast_two_sum(u23_to_f_2p23((unsigned)(Q >> 23)), u23_to_f((unsigned)Q & 0x7FFFFFu));
    return ff_neglog1m_series(ff_mul(q, ff{c.iS_hi, c.iS_lo}));
  }
  return ff_neglog1m_table(Q, S, c);
}

// A positive normal double as float-float: its 53-bit significand m = 1.f 2^52
// cut into the leading 24 bits (hi, exact) and the next 23 (lo, exact), the last
// 6 bits dropped: relative error below 2^-47.  Requires the binary exponent E
// (x = m 2^(E - 52)) in [-80, 100], so that hi and lo are normal floats.
__device__ __forceinline__ ff ff_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const float hi = __int_as_float((unsigned)((E + 127) << 23) | (unsigned)((m >> 29) & 0x7FFFFFu));
  const float scale = __int_as_float((unsigned)((E - 46 + 127) << 23));  // 2^(E - 46)
  return ff{hi, __fmul_rn(u23_to_f((unsigned)(m >> 6) & 0x7FFFFFu), scale)};
}

// -ln(1 - Q/S) for doubles 0 < Q < S (double weights): the series of
// ff_neglog1m_series for p < 2^-12 with p = Q (1/S) (Q from its leading 47
// significand bits, 1/S a float-float pair: relative error ~2^-46); otherwise
// the reduced logarithm of A / S from the two significands and the exponent
// difference, A = S - Q rounded to double, and the rounding error c = S - Q - A
// (exact by Dekker's FastTwoSum, S > Q) put back to first order:
// -ln((A + c)/S) = -ln(A/S) - c/A + O(2^-106).  Without it the 2^-53 relative
// error of A would be 2^-53 / p of the result, 2^-41 at p = 2^-12.  Outside the
// float range of the series' conversion (Q below 2^-80 or above 2^100) the
// double logarithm is used.
__device__ __forceinline__ ff ff_neglog1m_d(double Q, double S, const LpConstD& c) {
  if (Q < c.S_small) {
    const int E = (int)(((unsigned long long)__double_as_longlong(Q) >> 52) & 0x7FF) - 1023;
    if (E >= -80 && E <= 100) return ff_neglog1m_series(ff_mul(ff_from_double(Q), ff{c.iS_hi, c.iS_lo}));
    const double L = d_neglog1m(Q, S);
    const float h = (float)L;
    return ff{h, (float)(L - (double)h)};
  }
  const double A = __dsub_rn(S, Q);
  const double cA = __dsub_rn(__dsub_rn(S, A), Q);
  const unsigned long long b = (unsigned long long)__double_as_longlong(A);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int e = c.s_e - eb;  // >= 0: A < S
  const unsigned long long a = (b & ((1ull << 52) - 1)) | (1ull << 52);  // A = a 2^(eb - 1075)
  // c/A = (c 2^(1075 - eb)) / a with |c 2^(1075 - eb)| <= 1/2; below eb = 53 (A under
  // 2^-970, the result above 670) the term is left out
  const double sc = __longlong_as_double((long long)(eb >= 53 ? 2098 - eb : 0) << 52);
  const float t = (float)__dmul_rn(cA, sc);
  const float corr = __fmul_rn(__fmul_rn(t, 0x1p-30f), rcp_nr(u23_to_f((unsigned)(a >> 30))));
  ff L = ff_neglog_reduced(a, c.s_m, e, 30, c.cS);
  L.lo = __fsub_rn(L.lo, corr);
  return L;
}

}  // namespace cl
