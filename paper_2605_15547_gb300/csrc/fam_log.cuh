// fam_log.cuh -- logf, log2f, log10f, log1pf.
//
// Following the paper's log2f scheme (Fig. 2, Sec. II.A): split x = 2^e m with m in
// [3/4, 3/2) (so that the result near x = 1 comes from the polynomial alone, without
// cancellation), pick a table point near m, and write log x = e log 2 + log c + log1p(r).
// The FP64 and double-double tiers use c_j = j/128 and r = (m - c_j)/c_j, |r| <= 2^-7.58,
// with (1/c_j, log c_j) from a 97-entry table; the double-float tier uses a short
// reciprocal R_j of j/256 (the paper's cr_log idea, Sec. II.B), so that r = m R_j - 1 is
// exact.  For log2 and log10 the FP64 and double-double tiers use tables of log2 / log10
// and scale log1p(r) by 1/ln 2 or 1/ln 10; the double-float tier scales the natural
// logarithm.  log1p(x) evaluates the polynomial on x itself for |x| < 2^-7 and otherwise
// works on u = 1 + x = uh + ul (exact pair), adding ul/uh.
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"
#include "fam_f64.cuh"

namespace crm {

// KIND 0: ln, 1: log2, 2: log10, 3: log1p (ln of 1 + x)
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
// Decomposition in binary32, x = 2^e m with m in [3/4, 3/2), j = rint(256 m), and R_j =
// 1/(j/256) rounded to 9 significant bits: r = m R_j - 1 is one exact FMA (m R_j is a
// multiple of 2^-32 and |r| <= 2^-8.008), and
//   ln x = e ln 2 - ln R_j + log1p(r)
// (the reduction of the paper's cr_log, Sec. II.B, with a short reciprocal).  The table
// (CRM_LN_T193M_DF) splits L = -ln R_j into L_hi on the grid 2^-17, L_mid on the grid
// 2^-32 (|L_mid| <= 2^-18) and L_lo, so that two sums are exact without error terms:
//   B = e ln2_hi + L_hi (one FMA: a multiple of 2^-17 below 2^7 for |e| <= 149), and
//   r' = r + L_mid (a multiple of 2^-32 below 2^-8).
// log1p(r) + L_mid = r' - r^2/2 + r^3/3 - r^4/4 + r^5/5 (remainder r^6/6 <= 2^-50.6):
//   s = RN(r' - r^2/2) by one FMA on the exact product (-r/2) r, its error z exactly
//   (r' - s is exact, s being within a factor 2 of r'), and the tail
//   P = (-r^2/2) r (-2/3 + r/2 - 2r^2/5) in float, added to z by one FMA.
// Then hi = RN(B + s) by Fast2Sum (|B| >= |s| unless B = 0: with e = 0 and j != 256,
// |L_hi| > |r| + |L_mid| + r^2, checked for every j when the table is generated) and
// lo = (s - (hi - B)) + ((z + P) + (e ln2_lo + L_lo)).  log2 and log10 multiply the pair by
// the float pair 1/ln 2 or 1/ln 10 (four operations).  Error budget, relative to the result:
//   with e = 0 and j = 256 (L = 0) the terms scale with r: tail roundings 5 2^-24 r^2/3 <=
//   2^-39.3, s's error term 2^-48; otherwise |result| >= 2^-9: tail 2^-47.3 + 2^-49.6
//   abs, the three sums of lo 2^-24 |lo| with |lo| < 2^-25.5 (e = 0) or below 2^-24 of the
//   result (e != 0: e ln2_lo <= |e| 2^-18), ln 2 split 2^-43 |e| abs, the table 2^-57 abs;
//   the 1/ln b product 2^-47.  Total < 2^-38.5; the rounding test allows 2^-37.
// Exhaustively checked: every binary32 input that passes the test returns RN(f(x)).
//
// tb = the bit pattern of us with the exponent offset eadj folded into its exponent field
// (fbits(us) + eadj 2^23, modulo 2^32: a subnormal input scaled by 2^24 passes eadj = -24;
// any tb gives an in-range table index, the result is then meaningless and discarded),
// plus, for log1p, the low word ul of 1 + x and the direct path for |x| < 2^-7 (r = x, the
// entry of R = 1).  Returns the unnormalised pair.  With EXACT_T the correction ul/us is a
// correctly rounded division (for callers whose result can consist of that term alone, e.g.
// log(x^2 + y^2) with x^2 + y^2 within 2^-24 of a power of two); otherwise the fast
// reciprocal suffices (log1pf: the term is below 2^-24 of r).
template <int KIND, bool EXACT_T = false>
CRM_DEV Pair<float> log_df_core(uint32_t tb, float us, float ul, bool pathA, float x, const float4 *T193) {
  // m = 2^-e us in [3/4, 3/2) from one subtraction: the exponent field of us / (3/4)
  // rounded down is floor(log2(us / (3/4)))
  const uint32_t t = tb - 0x3F400000u;
  const int32_t ee = (int32_t)t >> 23;
  const float m = bitsf(t - ((uint32_t)ee << 23) + 0x3F400000u);
  const float sh = fma_(m, 256.0f, CRM_SHIFTER_F);
  uint32_t j = fbits(sh) - (fbits(CRM_SHIFTER_F) + 192u);
  if (KIND == 3) j = pathA ? 64u : j;  // the entry of R = 1: every L word zero
  const float4 E = T193[j];            // (R_j, L_hi, L_mid, L_lo)
  float r = fma_(m, E.x, -1.0f);       // exact
  float tc = 0.0f;
  if (KIND == 3) {  // pathA: us within 2^-7 of 1, so e = 0
    tc = EXACT_T ? ul / us : __fdividef(ul, us);  // ul/us with |ul| <= 2^-24 us
    r = pathA ? x : r;
    tc = pathA ? 0.0f : tc;
  }
  const float rp = r + E.z;  // exact
  const float hr = -0.5f * r;
  const float s = fma_(hr, r, rp);
  const float z = fma_(hr, r, rp - s);
  float g = fma_(r, -0.4f, 0.5f);
  g = fma_(r, g, -0x1.555556p-1f);
  g = r * g;
  float zp = fma_(hr * r, g, z);
  if (KIND == 3) zp = zp + tc;
  const float ef = (float)ee;
  const float B = fma_(ef, CRM_LN2_F16_HI, E.y);  // exact
  const float Bl = fma_(ef, CRM_LN2_F16_LO, E.w);
  const float hi = B + s;
  const float lo = (s - (hi - B)) + (zp + Bl);
  if (KIND == 1 || KIND == 2) {
    const float IH = KIND == 1 ? CRM_INV_LN2_F_HI : CRM_INV_LN10_F_HI;
    const float IL = KIND == 1 ? CRM_INV_LN2_F_LO : CRM_INV_LN10_F_LO;
    const float qh = hi * IH;
    float ql = fma_(hi, IH, -qh);
    ql = fma_(hi, IL, ql);
    ql = fma_(lo, IH, ql);
    return {qh, ql};
  }
  return {hi, lo};
}

// Specials: lanes outside the finite positive domain (log1p: outside (-1, inf) minus 0)
// take the result of special_log.  The common one, a negative argument (log1p: below -1),
// whose result is the default NaN, is a select; the rare ones (NaN, zeros, +inf; log1p
// also -1) a branch.
template <int KIND> CRM_DEV float log_df(float x, const float4 *T193, bool &hard, int *sg = nullptr) {
  if (KIND == 3 && sg && fabsf(x) < 0x1p-25f && x != 0.0f) {  // log1p x = x - x^2/2 + ...: just below x
    hard = false;
    *sg = -1;
    return x;
  }
  float us, ul = 0.0f;
  uint32_t tb;
  bool pathA = false, ok, rare;
  if (KIND == 3) {  // 1 + x is never subnormal for x > -1
    pathA = fabsf(x) < 0x1p-7f;
    const Pair<float> u = two_sum(1.0f, x);
    us = u.hi;
    ul = u.lo;
    tb = fbits(us);
    ok = (x > -1.0f) && (fabsf(x) < CRM_INF_F) && (x != 0.0f);
    rare = !ok && !(x < -1.0f);
  } else {  // subnormal inputs scaled by 2^24 (a select: they are common in bit-pattern inputs)
    const uint32_t bx = fbits(x);
    const float sc = bx < 0x00800000u ? 0x1p24f : 1.0f;
    us = x * sc;
    tb = fbits(us) - fbits(sc) + fbits(1.0f);
    ok = (bx - 1u) < 0x7F7FFFFFu;  // positive, finite, nonzero
    rare = !ok && !(x < 0.0f);
  }
  const Pair<float> y = log_df_core<KIND>(tb, us, ul, pathA, x, T193);
  if (sg) {  // directed rounding: a branch
    if (__builtin_expect(ok, 1)) return round_df(y.hi, y.lo, hard, sg);
    hard = false;
    *sg = 0;  // exact results
    return special_log<KIND>(x);
  }
  bool h;
  const float v = round_df(y.hi, y.lo, h);
  hard = ok && h;
  float res = ok ? v : CRM_QNAN_F;
  if (__builtin_expect(rare, 0)) res = special_log<KIND>(x);
  return res;
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
