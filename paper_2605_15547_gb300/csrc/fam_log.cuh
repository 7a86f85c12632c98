// fam_log.cuh -- logf, log2f, log10f, log1pf.
//
// Following the paper's log2f scheme (Fig. 2, Sec. II.A): split x = 2^e m with m in
// [3/4, 3/2) (so that the result near x = 1 comes from the polynomial alone, without
// cancellation), pick a table point near m, and write log x = e log 2 + log c + log1p(r).
// The FP64 and double-double tiers use c_j = j/128 and r = (m - c_j)/c_j, |r| <= 2^-7.58,
// with (1/c_j, log c_j) from a 97-entry table; the double-float tier uses a short
// reciprocal R_j of j/256 (the paper's cr_log idea, Sec. II.B), so that r = m R_j - 1 is
// exact.  log2 and log10 use tables of log2 / log10 and scale log1p(r) by 1/ln 2 or
// 1/ln 10.  log1p(x) evaluates the polynomial on x itself for |x| < 2^-7 and otherwise
// works on u = 1 + x = uh + ul (exact pair), adding ul/uh.
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"
#include "fam_f64.cuh"

namespace crm {

// KIND 0: ln, 1: log2, 2: log10, 3: log1p (ln of 1 + x)
template <int KIND> struct LogK;
template <> struct LogK<0> {
  static constexpr float KH = CRM_LN2_F16_HI, KL = CRM_LN2_F16_LO;
};
template <> struct LogK<1> {
  static constexpr float KH = 1.0f, KL = 0.0f;
};
template <> struct LogK<2> {
  static constexpr float KH = CRM_LOG10_2_F16_HI, KL = CRM_LOG10_2_F16_LO;
};
template <> struct LogK<3> : LogK<0> {};

// Table per kind: log1p uses the natural-log table.
template <int KIND> CRM_DEV const float *log_tab_df() {
  return KIND == 1 ? CRM_LOG2_T193R_DF : (KIND == 2 ? CRM_LOG10_T193R_DF : CRM_LN_T193R_DF);
}
template <int KIND> CRM_DEV const double *log_tab_dd() {
  return KIND == 1 ? CRM_LOG2_T97_DD : (KIND == 2 ? CRM_LOG10_T97_DD : CRM_LN_T97_DD);
}

// Decompose a positive normal double u = 2^e m, m in [3/4, 3/2); j = round(128 m) and
// c = j/128 with integer operations only.
struct DecD {
  double m, c;
  int e, j;
};
CRM_DEV DecD decompose_d(double u) {
  uint64_t b = dbits(u);
  uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
  bool big = mant >= (1ull << 51);  // m in [1.5, 2): halve
  DecD r;
  r.e = (int)(b >> 52) - 1023 + (big ? 1 : 0);
  r.m = bitsd(mant | (big ? 0x3FE0000000000000ull : 0x3FF0000000000000ull));
  if (big) {
    r.j = 64 + (int)((mant + (1ull << 45)) >> 46);
    r.c = bitsd(0x3FE0000000000000ull + ((uint64_t)(r.j - 64) << 46));
  } else {
    r.j = 128 + (int)((mant + (1ull << 44)) >> 45);
    r.c = bitsd(0x3FF0000000000000ull + ((uint64_t)(r.j - 128) << 45));
  }
  return r;
}

// ------------------------------------------------------------------ plain (FP64) tier
// r = (m - c) / c: m - c exact, times the double 1/c (relative error 2^-52).
// log1p(r) by Taylor to degree 7 (remainder r^8/8 <= 2^-63.6, i.e. 2^-56 relative to r),
// Horner in FP64.  ln u = e ln2_hi + L + (p + e ln2_lo) (e ln2_hi exact: 42-bit split).
// Error: p relative 2^-51.5 (remainder + 8 roundings at |r|-scaled weight), L 2^-53 |L|,
// final two sums 2^-53 |y| each, optional scaling by 1/ln 2 or 1/ln 10 2^-53: < 2^-49.7
// relative to |y| (|p| <= |L|/2 or L = 0, so there is no cancellation).
// eps = 2^-48 -> D = ceil(2^-48 2^53) + 1 = 33.
constexpr uint32_t LOG_PLAIN_D = 33;

template <int KIND> CRM_DEV double log_plain_y(float x, const double2 *T97) {
  double xd = (double)x;
  bool pathA = false;
  double u = xd;
  if (KIND == 3) {
    pathA = fabsf(x) < 0x1p-7f;
    u = pathA ? 1.0 : 1.0 + xd;  // 1 + x: exact for |x| < 2^29, else within 2^-53
  }
  DecD D = decompose_d(u);
  double2 T = T97[D.j - 96];
  double r = (D.m - D.c) * T.x;
  double L = T.y;
  double ef = (double)D.e;
  if (KIND == 3) r = pathA ? xd : r;
  const double *c = CRM_LOG1P_TAYLOR_D;  // c[k-1] = (-1)^(k+1)/k
  double p = fma_(r, c[6], c[5]);
  p = fma_(r, p, c[4]);
  p = fma_(r, p, c[3]);
  p = fma_(r, p, c[2]);
  p = fma_(r, p, c[1]);
  p = fma_(r, p, c[0]);
  p = p * r;
  double y = fma_(ef, CRM_LN2_D42_HI, L) + fma_(ef, CRM_LN2_D42_LO, p);
  if (KIND == 1) y = y * CRM_INV_LN2_D_HI;
  if (KIND == 2) y = y * CRM_INV_LN10_D_HI;
  return y;
}

// Lanes outside the finite positive domain (NaN, 0, negative, inf; for log1p also
// x <= -1 and x == 0) are returned through special_log.
template <int KIND> CRM_DEV float special_log(float x) {
  if (x != x) return qnan_of(x);
  if (KIND == 3) {
    if (x == 0.0f) return x;
    if (x == -1.0f) return -CRM_INF_F;
    if (x < -1.0f) return CRM_QNAN_F;
    return CRM_INF_F;  // +inf
  }
  if (x == 0.0f) return -CRM_INF_F;
  if (x < 0.0f) return CRM_QNAN_F;
  return CRM_INF_F;
}
template <int KIND> CRM_DEV bool log_ok(float x) {
  if (KIND == 3) return (x > -1.0f) && (x < CRM_INF_F) && (x != 0.0f);
  return (x > 0.0f) && (x < CRM_INF_F);
}

template <int KIND> CRM_DEV float log_plain(float x, const double2 *T97, bool &hard) {
  bool ok = log_ok<KIND>(x);
  double y = log_plain_y<KIND>(ok ? x : 2.0f, T97);
  hard = ok && hard_d_to_f(y, LOG_PLAIN_D);
  return ok ? __double2float_rn(y) : special_log<KIND>(x);
}

// ------------------------------------------------------------------ double-float tier
// Decomposition in binary32 (subnormal inputs are scaled by 2^24 first), x = 2^e m with
// m in [3/4, 3/2), j = rint(256 m), and R_j = 1/(j/256) rounded to 9 significant bits
// (a 193-entry table with -log_b R_j as a float pair): r = m R_j - 1 is one exact FMA
// (m R_j is a multiple of 2^-32 and |r| <= 2^-8.008 < 2^-8), and
//   log_b x = e log_b 2 - log_b R_j + log_b(1 + r)
// (the reduction of the paper's cr_log, Sec. II.B, with a short reciprocal).
// log1p(r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5): r - r^2/2 by Fast2Sum on the exact
// square (split by FMA), the r^3 tail in float.  For log2 / log10 the pair is multiplied
// by the float pair 1/ln 2 or 1/ln 10.  B = e K_hi - log_b R_j by one FMA (e K_hi is exact:
// K_hi has 16 significant bits) with its rounding error recovered exactly as in Fast2Sum
// (e == 0, or |e K_hi| > |log_b R_j|), then Fast2Sum(B, q); the sum goes to the rounding
// test unnormalised.  Error budget, relative to the result:
//   r^6/6 remainder 2^-50.6 abs, tail rounding 2^-49.6 abs, the table pair and the K split
//   <= 2^-48 abs, with |result| >= 2^-9 unless e = 0 and j = 256 (then R_j = 1, all terms
//   scale with r and the bound is 2^-40 relative); e K_lo rounding and the K split
//   <= 2^-42 relative.  Total < 2^-39; the test allows 2^-37 (round_df: the low word is
//   below 2^-15 of the high one).
//
// us = 2^(e - eadj) m for a positive normal float us (any bit pattern gives an in-range
// table index; the result is then meaningless and discarded), plus, for log1p, the low
// word ul of 1 + x and the direct path for |x| < 2^-7.  Returns the unnormalised sum.
// With EXACT_T the correction ul/us is a correctly rounded division (for callers whose result
// can consist of that term alone, e.g. log(x^2 + y^2) with x^2 + y^2 within 2^-24 of a power
// of two); otherwise the fast reciprocal suffices (log1pf: the term is below 2^-24 of r).
template <int KIND, bool EXACT_T = false>
CRM_DEV Pair<float> log_df_core(float us, int eadj, float ul, bool pathA, float x, const float4 *T193) {
  using K = LogK<KIND>;
  // us = 2^e m, m in [3/4, 3/2), from one integer subtraction: the exponent field of
  // us / (3/4) rounded down is floor(log2(us / (3/4)))
  const uint32_t b = fbits(us);
  const int32_t ee = (int32_t)(b - 0x3F400000u) >> 23;
  const float m = bitsf(b - ((uint32_t)ee << 23));
  const float sh = fma_(m, 256.0f, CRM_SHIFTER_F);
  const float4 T = T193[fbits(sh) - (fbits(CRM_SHIFTER_F) + 192u)];  // (R_j, 0, L hi, lo)
  float rh = fma_(m, T.x, -1.0f);  // exact
  float Lh = T.z, Ll = T.w, ef = (float)(ee + eadj);
  float t = 0.0f;
  if (KIND == 3) {
    t = EXACT_T ? ul / us : __fdividef(ul, us);  // ul/uh with |ul| <= 2^-24 uh
    rh = pathA ? x : rh;
    Lh = pathA ? 0.0f : Lh;
    Ll = pathA ? 0.0f : Ll;
    ef = pathA ? 0.0f : ef;
    t = pathA ? 0.0f : t;
  }
  // log1p(r)
  float h2 = rh * rh;
  float h2l = fma_(rh, rh, -h2);
  float q3 = fma_(rh, 0.2f, -0.25f);
  q3 = fma_(rh, q3, 0x1.555556p-2f);
  float P = (h2 * rh) * q3;
  float s = fma_(h2, -0.5f, rh);
  float z = fma_(h2, -0.5f, rh - s);
  float rest = fma_(h2l, -0.5f, P);
  rest = rest + (KIND == 3 ? z + t : z);
  float qh = s, ql = rest;
  if (KIND == 1 || KIND == 2) {
    const float IH = KIND == 1 ? CRM_INV_LN2_F_HI : CRM_INV_LN10_F_HI;
    const float IL = KIND == 1 ? CRM_INV_LN2_F_LO : CRM_INV_LN10_F_LO;
    qh = s * IH;
    ql = fma_(s, IH, -qh);
    ql = fma_(s, IL, ql);
    ql = fma_(rest, IH, ql);
  }
  // B = e K + L: B = RN(e K_hi + L_hi), e K_hi - B exact, Bz = L_hi - (B - e K_hi)
  float B = fma_(ef, K::KH, Lh);
  float Bz = Lh + fma_(ef, K::KH, -B);
  float Bl = Bz + fma_(ef, K::KL, Ll);
  // |B| > |qh| unless B = 0: with e != 0, |e K + L| >= 0.125 (log10; more for ln, log2);
  // with e = 0 and j != 256, |log_b R_j| >= 1.97 |log_b(1 + r)| (checked over every j when
  // the table is generated); so Fast2Sum is exact here
  Pair<float> S = fast_two_sum(B, qh);
  return {S.hi, S.lo + (Bl + ql)};
}

template <int KIND> CRM_DEV float log_df(float x, const float4 *T193, bool &hard, int *sg = nullptr) {
  if (KIND == 3 && sg && fabsf(x) < 0x1p-25f && x != 0.0f) {  // log1p x = x - x^2/2 + ...: just below x
    hard = false;
    *sg = -1;
    return x;
  }
  const bool ok = log_ok<KIND>(x);
  float us = x, ul = 0.0f;
  int eadj = 0;
  bool pathA = false;
  if (KIND == 3) {  // 1 + x is never subnormal for x > -1
    pathA = fabsf(x) < 0x1p-7f;
    Pair<float> u = two_sum(1.0f, x);
    us = u.hi;
    ul = u.lo;
  } else {  // subnormal inputs by selects: they are common in bit-pattern inputs
    const bool sub = x < 0x1p-126f;
    us = sub ? x * 0x1p24f : x;
    eadj = sub ? -24 : 0;
  }
  Pair<float> y = log_df_core<KIND>(us, eadj, ul, pathA, x, T193);
  if (__builtin_expect(ok, 1)) return round_df(y.hi, y.lo, hard, sg);
  hard = false;  // NaN, zero, negative, infinite (rare: a branch, not selects)
  put_sg(sg, 0);  // exact results
  return special_log<KIND>(x);
}

// ------------------------------------------------------------------ double-double tier
// Same decomposition in binary64 on u = uh + ul (exact), d = (m - c) + ul 2^-e as a
// double-double, r = d (1/c)_dd, log1p(r) by Taylor to degree 14 in double-double Horner
// form (remainder < 2^-110), ln u = e ln2_dd + L_dd + log1p(r), scaled by 1/ln2_dd or
// 1/ln10_dd.  Error < 2^-98 relative.
constexpr double LOG_DD_EPS = 0x1p-92;

template <int KIND> CRM_DEV Pair<double> log_dd_core(float x) {
  double xd = (double)x;
  Pair<double> u = {xd, 0.0};
  bool pathA = false;
  if (KIND == 3) {
    pathA = fabsf(x) < 0x1p-7f;
    u = pathA ? Pair<double>{1.0, 0.0} : two_sum(1.0, xd);
  }
  DecD D = decompose_d(u.hi);
  const double *T = log_tab_dd<KIND == 3 ? 0 : KIND>() + 4 * (D.j - 96);
  double sc = pow2d(-D.e);
  Pair<double> dd_ = two_sum(D.m - D.c, u.lo * sc);
  Pair<double> r = dd_mul(dd_, dd(T[0], T[1]));
  if (KIND == 3 && pathA) r = {xd, 0.0};
  const double *c = CRM_LOG1P_TAYLOR_DD;  // pairs, k = 1..17
  Pair<double> p = dd(c[2 * 13], c[2 * 13 + 1]);
  for (int k = 12; k >= 0; k--) p = dd_add(dd_mul(p, r), dd(c[2 * k], c[2 * k + 1]));
  p = dd_mul(p, r);
  Pair<double> y;
  if (KIND == 1) {
    // log2: e + (log2 c + log1p(r)/ln 2)
    Pair<double> q = dd_mul(p, dd(CRM_INV_LN2_D_HI, CRM_INV_LN2_D_LO));
    y = dd_add(dd_add(q, dd(T[2], T[3])), dd((double)D.e, 0.0));
  } else {
    Pair<double> eK = KIND == 2 ? dd_mul_d(dd(CRM_LOG10_2_DD_HI, CRM_LOG10_2_DD_LO), (double)D.e)
                                : dd_mul_d(dd(CRM_LN2_DD_HI, CRM_LN2_DD_LO), (double)D.e);
    if (KIND == 2) p = dd_mul(p, dd(CRM_INV_LN10_D_HI, CRM_INV_LN10_D_LO));
    if (KIND == 3 && pathA) {
      y = p;
    } else {
      y = dd_add(dd_add(eK, dd(T[2], T[3])), p);
    }
  }
  return y;
}

template <int KIND> CRM_DEV float log_dd(float x, bool &hard, int *sg = nullptr) {
  Pair<double> y = log_dd_core<KIND>(x);
  return round_dd_to_f(y.hi, y.lo, LOG_DD_EPS * fabs(y.hi), hard, sg);
}

// ------------------------------------------------------------------ FP64-free middle tier
// logf, log2f, log10f of a positive finite x: the binary64 path's fixed-point core
// (logz_q116: Z = ln x in Q116 with an error bound, 128-bit integer arithmetic, Sec. II.B's
// short-reciprocal reduction) on the exact binary64 value of x, times 1/ln 2 or 1/ln 10
// in Q126 for log2 / log10 (W = Z C 2^-126 truncated: the constant's rounding adds 2^-4 of
// a unit, the truncations 1 unit, and Z's error grows by C <= 1.443), then rounded to 24
// bits with an integer test: hard only when the discarded part lies within the bound of
// half an ulp (|log_b x| >= 2^-25 for x != 1, so the bound, a few hundred units of
// 2^-116, is below 2^-70 of the result).  On GB300 the FP64 pipe runs one warp
// instruction every few dozen cycles, so this tier replaces the FP64 tier for the lanes
// the double-float test sends to the slow path.
template <int KIND> CRM_DEV float logq_round(U128 Z, uint64_t err, bool &hard, int *sg = nullptr) {
  const bool neg = (int64_t)Z.hi < 0;
  U128 A = neg ? neg128(Z) : Z;  // |Z| < 2^123
  if (KIND == 1 || KIND == 2) {
    const uint64_t ch = KIND == 1 ? CRM_LOGI_INV_LN2_Q126_HI : CRM_LOGI_INV_LN10_Q126_HI;
    const uint64_t cl = KIND == 1 ? CRM_LOGI_INV_LN2_Q126_LO : CRM_LOGI_INV_LN10_Q126_LO;
    // A C as 256 bits (limbs w0..w3), then W = A C >> 126
    const U128 hh = mul64w(A.hi, ch), hl = mul64w(A.hi, cl), lh = mul64w(A.lo, ch);
    const uint64_t ll_hi = __umul64hi(A.lo, cl);
    U128 mid = add128(hl, lh);  // may carry into bit 128 of the middle sum
    const uint64_t c1 = (mid.hi < hl.hi || (mid.hi == hl.hi && mid.lo < hl.lo)) ? 1ull : 0ull;
    mid = add128_64(mid, ll_hi);
    const uint64_t c2 = (mid.hi == 0 && mid.lo < ll_hi) ? 1ull : 0ull;
    // limbs: w1 = mid.lo, w2 = hh.lo + mid.hi, w3 = hh.hi + carries
    const uint64_t w2 = hh.lo + mid.hi;
    const uint64_t w3 = hh.hi + c1 + c2 + (w2 < hh.lo ? 1ull : 0ull);
    const uint64_t w1 = mid.lo;
    // >> 126: W = (w3:w2:w1) >> 62 within 128 bits
    A.lo = (w2 << 2) | (w1 >> 62);
    A.hi = (w3 << 2) | (w2 >> 62);
    err = err + (err >> 1) + 3ull;
  }
  // round |W| (Q116; 2^-25.3 <= |W| < 2^8 unless x == 1) to 24 bits: sh = p - 23 discarded
  // bits, p the leading bit's position (90 .. 123, so sh in 67 .. 100; s64 guards the
  // shifts of the x == 1 lane)
  const bool zero = (A.hi | A.lo) == 0;
  const int p = A.hi ? 127 - __clzll(A.hi) : 63 - __clzll(A.lo | 1ull);
  const int sh = p - 23;
  const int s64 = sh < 64 ? 0 : sh - 64;
  const uint64_t mant = A.hi >> s64;  // 24 bits
  const U128 rem = {A.lo, A.hi & ((1ull << s64) - 1ull)};
  const U128 half = s64 == 0 ? U128{1ull << 63, 0ull} : U128{0ull, 1ull << (s64 - 1)};
  const U128 dlt = sub128(rem, half);
  const bool near = (dlt.hi == 0 && dlt.lo <= err) || (dlt.hi == ~0ull && dlt.lo >= 0ull - err);
  const bool up = (int64_t)dlt.hi > 0 || (dlt.hi == 0 && dlt.lo != 0);
  // value mant 2^(sh - 116): exponent field sh - 116 + 23 + 127, the leading bit adds 1
  const uint32_t bits = ((uint32_t)(sh + 33) << 23) + (uint32_t)mant + (up ? 1u : 0u);
  hard = !zero && (near || sh < 64);
  if (sg) {  // sign of v - y: decided unless the discarded part is within err of 0 or of a unit
    const U128 unit = s64 == 0 ? U128{0ull, 1ull} : U128{0ull, 1ull << s64};
    const U128 E = {err, 0ull};
    hard = !zero && (sh < 64 || le128(rem, E) || le128(sub128(unit, rem), E));
    *sg = zero ? 0 : ((up != neg) ? -1 : 1);  // |v| below |y| when rounded up; negated for v < 0
  }
  return zero ? 0.0f : bitsf(bits | (neg ? 0x80000000u : 0u));
}

// The binary64 bit pattern of a positive finite binary32 x, by integer operations.
CRM_DEV uint64_t f2d_bits_pos(float x) {
  const uint32_t b = fbits(x), m = b & 0x007FFFFFu;
  const uint32_t E = b >> 23;
  if (E != 0) return ((uint64_t)(E + 896u) << 52) | ((uint64_t)m << 29);
  const int p = 31 - __clz(m);  // subnormal: x = m 2^-149, leading bit p in [0, 22]
  return ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0x000FFFFFFFFFFFFFull);
}

template <int KIND> CRM_DEV float logf_int(float x, bool &hard, int *sg = nullptr) {
  uint64_t err;
  const U128 Z = logz_q116(f2d_bits_pos(x), (const ulonglong2 *)CRM_LOGI_L, CRM_LOGI_R, err);
  return logq_round<KIND>(Z, err, hard, sg);
}

// log1pf of x > -1, x != 0, finite: |x| < 2^-25 gives x (x^2/2 is below half an ulp of x,
// on either side, and log1p x is never a midpoint).  Otherwise 1 + x is exact in binary64
// for x < 2^53 (x's last bit is at least 2^-48, and 1 + x spans at most 53 bits), and the
// same core gives ln(1 + x) (|ln(1 + x)| >= 2^-25.1, inside the rounding's range).  For x >=
// 2^53, ln(1 + x) = ln x + 1/x - 1/(2x^2) + ...: 1/x <= 2^-53 is added in Q116 from a
// binary32 reciprocal (relative 2^-24: at most 2^40 units, bounded by c 2^-23 + 2 units),
// the rest is below 2^-105 (2^11 units).  These bounds are far below an ulp of the result
// (ln x >= 36, ulp 2^98 units): hard lanes stay rare.
CRM_DEV float log1pf_int(float x, bool &hard, int *sg = nullptr) {
  hard = false;
  put_sg(sg, -1);  // log1p x < x for x != 0
  if (fabsf(x) < 0x1p-25f) return x;
  uint64_t err;
  const ulonglong2 *LT = (const ulonglong2 *)CRM_LOGI_L;
  if (x < 0x1p53f) return logq_round<0>(logz_q116(dbits((double)x + 1.0), LT, CRM_LOGI_R, err), err, hard, sg);
  U128 Z = logz_q116(f2d_bits_pos(x), LT, CRM_LOGI_R, err);
  const uint32_t rb = fbits(1.0f / (x * 0x1p-100f));  // 2^100/x in [2^-28, 2^47], normal
  const uint64_t Mr = (rb & 0x007FFFFFu) | 0x00800000u;
  const int s = (int)(rb >> 23) - 134;  // 2^116/x = Mr 2^(Er - 150 - 100 + 116)
  const uint64_t c = s >= 0 ? Mr << s : Mr >> (-s);
  Z = add128_64(Z, c);
  err += (c >> 23) + 2ull + 2048ull;
  return logq_round<0>(Z, err, hard, sg);
}

// Slow path: the FP64-free tier, then double-double.
// With sg: the exact results log2(2^k) = k and log10(10^k) = k (k = 1..10) are returned
// directly (an error bound cannot decide a result that is a binary32 number).
template <int KIND> CRM_DEV float log_slow(float x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = false;
  if (!log_ok<KIND>(x)) {
    put_sg(sg, 0);
    return special_log<KIND>(x);
  }
  float r = KIND == 3 ? log1pf_int(x, hard, sg) : logf_int<KIND>(x, hard, sg);
  if (!hard && !force) return r;
  // exact zero (x = 1) and log1p's shortcut (|x| < 2^-25: log1p x < x) are final
  if (sg && !hard && (*sg == 0 || (KIND == 3 && fabsf(x) < 0x1p-25f))) return r;
  if (sg && KIND == 1) {
    const uint32_t b = fbits(x);
    const uint32_t m = b & 0x007FFFFFu, E = b >> 23;
    if ((E != 0 && m == 0) || (E == 0 && (m & (m - 1u)) == 0)) {  // a power of two
      *sg = 0;
      return E != 0 ? (float)((int)E - 127) : (float)(31 - __clz(m) - 149);
    }
  }
  if (sg && KIND == 2) {
    float p = 1.0f;
    for (int k = 1; k <= 10; k++) {
      p *= 10.0f;  // exact
      if (x == p) {
        *sg = 0;
        return (float)k;
      }
    }
  }
  r = log_dd<KIND>(x, hard, sg);
  unresolved = hard ? 3 : 2;  // the double-double tier ran
  return r;
}

}  // namespace crm
