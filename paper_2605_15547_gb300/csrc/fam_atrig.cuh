// fam_atrig.cuh -- atanf, asinf, acosf through one core, atan(a/b) for a, b >= 0.
//
//   atan x = sign(x) atan(|x| / 1),
//   asin x = sign(x) atan(|x| / s),           s = sqrt((1 - x)(1 + x)),
//   acos x = atan(s / x) (x > 0),  pi - atan(s / |x|) (x < 0),
// so that small results (atan and asin near 0, acos near 1) come out of the core with
// full relative accuracy.  The core swaps a and b when a > b (atan(a/b) = pi/2 -
// atan(b/a)), picks c_j = j/16 nearest to p/q (p <= q), and uses
//   atan(p/q) = atan(c_j) + atan(t),   t = (p - c_j q) / (q + c_j p),   |t| <= 1/32,
// with a 17-entry table of atan(j/16) (the paper's atanf uses a 0.125 KB table, Table I)
// and an odd polynomial for atan(t).  One division per evaluation.
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"
#include "fam_f64.cuh"

namespace crm {

enum { AT_ATAN = 0, AT_ASIN = 1, AT_ACOS = 2 };

// ------------------------------------------------------------------ plain (FP64) tier
// t: exact numerator when c_j = 0 (then t = p/q to 2^-53), else absolute error <= 2^-52
// (rounding of s and of the division); polynomial to degree 9 (remainder t^11/11 <=
// 2^-58.5); table 2^-53; the sum atan(c_j) + atan(t) is at least half of atan(c_j), so
// errors grow at most twice.  atan: eps = 2^-47 (D = 65); asin, acos: eps = 2^-46 (129).
CRM_DEV double atan_ratio_d(double a, double b, const double *AT) {
  bool sw = a > b;
  double p = sw ? b : a, q = sw ? a : b;
  float rf = __fdividef(__double2float_rn(p), __double2float_rn(q));  // only picks j
  int j = __float2int_rn(rf * 16.0f);
  j = j < 0 ? 0 : (j > 16 ? 16 : j);
  double c = (double)j * 0.0625;
  double t = fma_(-c, q, p) / fma_(c, p, q);
  double t2 = t * t;
  const double *k = CRM_ATAN_TAYLOR_D;
  double at = fma_(t2, fma_(t2, fma_(t2, fma_(t2, k[4], k[3]), k[2]), k[1]), k[0]) * t;
  double r = AT[j] + at;
  return sw ? (CRM_PIO2_D_HI - r) + CRM_PIO2_D_LO : r;
}

template <int KIND> CRM_DEV bool atrig_special(float x, float &r) {
  bool nan = x != x;
  float ax = fabsf(x);
  if (KIND == AT_ATAN) {
    r = nan ? qnan_of(x) : x;  // +-0 -> +-0 (infinities are not special: atan(1/0))
    return nan || x == 0.0f;
  }
  if (KIND == AT_ASIN) {
    r = nan ? qnan_of(x) : (ax > 1.0f ? CRM_QNAN_F : x);
    return nan || ax > 1.0f || x == 0.0f;
  }
  r = nan ? qnan_of(x) : (ax > 1.0f ? CRM_QNAN_F : 0.0f);  // acos(1) = +0
  return nan || ax > 1.0f || x == 1.0f;
}

// (a, b) for atan(a/b) and whether to take pi - result (acos of a negative x)
template <int KIND> CRM_DEV void atrig_args(float x, double &a, double &b, bool &flip) {
  double ax = fabs((double)x);
  flip = false;
  if (KIND == AT_ATAN) {
    bool inf = fabsf(x) == CRM_INF_F;
    a = inf ? 1.0 : ax;
    b = inf ? 0.0 : 1.0;
    return;
  }
  double s = sqrt((1.0 - ax) * (1.0 + ax));  // 1 - x^2 is exact in binary64
  if (KIND == AT_ASIN) {
    a = ax;
    b = s;
  } else {
    a = s;
    b = ax;
    flip = x < 0.0f;
  }
}

template <int KIND> CRM_DEV float atrig_plain(float x, const double *AT, bool &hard) {
  float rsp;
  bool sp = atrig_special<KIND>(x, rsp);
  double a, b;
  bool flip;
  atrig_args<KIND>(sp ? 0.5f : x, a, b, flip);
  double r = atan_ratio_d(a, b, AT);
  if (KIND == AT_ACOS) r = flip ? (CRM_PI_D_HI - r) + CRM_PI_D_LO : r;
  if (KIND != AT_ACOS && x < 0.0f) r = -r;
  hard = !sp && hard_d_to_f(r, KIND == AT_ATAN ? 65u : 129u);
  return sp ? rsp : __double2float_rn(r);
}

// ------------------------------------------------------------------ double-float tier
// The same core on float pairs.  c_j q.hi is split exactly by FMA so that p - c_j q is
// exact in its leading word (Sterbenz: p/(c_j q) is within [1/2, 2] when j >= 1);
// t = num/den by df_div; atan t = t - t^3/3 + t^5 (1/5 - t^2/7) with t^3/3 as a pair.
// s = sqrt(1 - x^2): 1 - x^2 as an exact pair d, s0 = RN(d y0) with y0 the hardware
// reciprocal square root (s0 within delta < 2^-21.7 of sqrt(d)), and one Newton
// correction (d - s0^2) y0 / 2 from the residual: y0 in place of 1/s0 costs 2 delta of
// the correction (2^-42.2 of s), the truncation delta^2 / 2 (2^-44.4), the residual's
// roundings 2^-45.7: s to 2^-41.8 of itself, which moves the result by at most 1.3 times
// that (atan(u)/u >= pi/4 on [0, 1]).
// Error: t to 2^-43 (2^-43 of t when j = 0), atan t to 2^-45 of itself, table and pi
// pairs 2^-48, the sum at most doubles the errors: < 2^-41; with s (asin, acos) < 2^-40,
// inside the rounding test's 2^-37.  The result pair is left unnormalised (|lo| < 2^-21 |hi|) for round_df.
CRM_DEV Pair<float> atan_ratio_df(Pair<float> a, Pair<float> b, const float2 *AT) {
  bool sw = a.hi > b.hi;
  Pair<float> p = sw ? b : a, q = sw ? a : b;
  // j = rint(16 p/q) in [0, 16] by the 1.5 2^23 shifter (p/q <= 1: clamped, which also
  // maps a NaN quotient to 1); c = j/16 exactly
  const float rf = fminf(__fdividef(p.hi, q.hi), 1.0f);  // only picks j
  const float jsh = fma_(rf, 16.0f, CRM_SHIFTER_F);
  const int j = (int)(fbits(jsh) - fbits(CRM_SHIFTER_F));
  const float c = (jsh - CRM_SHIFTER_F) * 0.0625f;
  float m = c * q.hi;
  float ml = fma_(c, q.hi, -m);
  float nh = p.hi - m;  // exact
  float nl = (p.lo - ml) - c * q.lo;
  Pair<float> num = fast_two_sum(nh, nl);
  float d = c * p.hi;
  float dl = fma_(c, p.hi, -d);
  Pair<float> den = fast_two_sum(q.hi, d);
  den.lo = den.lo + (q.lo + dl + c * p.lo);
  Pair<float> t = df_div_raw(num, den);  // |t.lo| < 2^-20 |t.hi|: t^2 as below loses 2^-40
  // atan t
  float u = t.hi * t.hi;
  float ul = fma_(t.hi, t.hi, -u);
  ul = fma_(2.0f * t.hi, t.lo, ul);
  float w = t.hi * u;
  float wl = fma_(t.hi, u, -w);
  wl = fma_(t.hi, ul, wl);
  wl = fma_(t.lo, u, wl);
  float s3 = w * CRM_INV3_F_HI;
  float s3l = fma_(w, CRM_INV3_F_HI, -s3);
  s3l = fma_(w, CRM_INV3_F_LO, s3l);
  s3l = fma_(wl, CRM_INV3_F_HI, s3l);
  float ah = t.hi - s3;
  float al = (t.hi - ah) - s3;
  al = al + (t.lo - s3l);
  al = fma_(w * u, fma_(u, -0x1.249250p-3f, 0x1.99999ap-3f), al);  // t^5 (1/5 - t^2/7)
  float2 A = AT[j];
  // atan(j/16) >= atan(1/16) > |atan t| for j >= 1 (A = 0 for j = 0), and pi/2 > atan(a/b)
  // for the swapped case: both sums are ordered (Fast2Sum)
  Pair<float> r = df_add_ordered_raw({A.x, A.y}, {ah, al});
  if (sw) r = df_add_ordered_raw({CRM_PIO2_F_HI, CRM_PIO2_F_LO}, -r);
  return r;
}

template <int KIND> CRM_DEV float atrig_df(float x, const float2 *AT, bool &hard, int *sg = nullptr) {
  if (sg && fabsf(x) < (KIND == AT_ACOS ? 0x1p-27f : 0x1p-12f) && x == x) {
    // atan x just below x, asin x just above it (x^3/6 below half an ulp); acos x within
    // 2^-27 of pi/2, below RN(pi/2) = 0x1.921fb6p+0
    hard = false;
    *sg = KIND == AT_ATAN ? -sgnf(x) : (KIND == AT_ASIN ? sgnf(x) : -1);
    return KIND == AT_ACOS ? 0x1.921fb6p+0f : x;
  }
  float rsp;
  bool sp = atrig_special<KIND>(x, rsp);
  float xs = sp ? 0.5f : x;
  float ax = fabsf(xs);
  Pair<float> a, b;
  bool flip = false;
  if (KIND == AT_ATAN) {
    bool inf = ax == CRM_INF_F;
    a = {inf ? 1.0f : ax, 0.0f};
    b = {inf ? 0.0f : 1.0f, 0.0f};
  } else {
    // 1 - x^2 exactly as a pair, then its square root as a pair
    float p = ax * ax;
    float pl = fma_(ax, ax, -p);
    Pair<float> d1 = fast_two_sum(1.0f, -p);  // 1 >= p
    Pair<float> dd_ = fast_two_sum(d1.hi, d1.lo - pl);
    // d >= 2^-23 unless x = +-1 (d = 0: the floor keeps y0 finite and s = 0)
    const float y0 = rsqrt_hw(fmaxf(dd_.hi, 0x1p-126f));
    float s0 = dd_.hi * y0;
    float s2 = s0 * s0;
    float s2l = fma_(s0, s0, -s2);
    float res = ((dd_.hi - s2) - s2l) + dd_.lo;
    float corr = res * (0.5f * y0);
    Pair<float> s = fast_two_sum(s0, corr);
    if (KIND == AT_ASIN) {
      a = {ax, 0.0f};
      b = s;
    } else {
      a = s;
      b = {ax, 0.0f};
      flip = xs < 0.0f;
    }
  }
  Pair<float> r = atan_ratio_df(a, b, AT);
  if (KIND == AT_ACOS && flip) r = df_add_ordered_raw({CRM_PI_F_HI, CRM_PI_F_LO}, -r);  // pi > r
  if (__builtin_expect(sp, 0)) {
    hard = false;
    put_sg(sg, 0);  // NaN, +-0, acos(1) = +0: exact
    return rsp;
  }
  const float y = round_df(r.hi, r.lo, hard, sg);
  if (sg && KIND != AT_ACOS && x < 0.0f) *sg = -*sg;
  return (KIND != AT_ACOS && x < 0.0f) ? -y : y;
}

// ------------------------------------------------------------------ double-double tier
// s by one Newton step in double-double, t by a double-double division, atan(t) to
// degree 25 (remainder < 2^-130), double-double table and pi/2.  Error < 2^-96.
constexpr double ATRIG_DD_EPS = 0x1p-88;

CRM_DEV Pair<double> dd_sqrt(Pair<double> a) {
  if (a.hi <= 0.0) return {0.0, 0.0};
  double s0 = sqrt(a.hi);
  Pair<double> sq = two_prod(s0, s0);
  Pair<double> r = dd_add(a, dd_neg(sq));
  double corr = r.hi / (2.0 * s0);
  return fast_two_sum(s0, corr);
}

CRM_DEV Pair<double> atan_ratio_dd(Pair<double> a, Pair<double> b) {
  bool sw = a.hi > b.hi;
  Pair<double> p = sw ? b : a, q = sw ? a : b;
  double rq = q.hi == 0.0 ? 0.0 : p.hi / q.hi;
  int j = (int)rint(rq * 16.0);
  j = j < 0 ? 0 : (j > 16 ? 16 : j);
  double c = (double)j * 0.0625;
  Pair<double> num = dd_add(p, dd_mul_d(q, -c));
  Pair<double> den = dd_add(q, dd_mul_d(p, c));
  Pair<double> t = dd_div(num, den);
  Pair<double> t2 = dd_sqr(t);
  const double *k = CRM_ATAN_TAYLOR_DD;
  Pair<double> at = dd(k[2 * 13], k[2 * 13 + 1]);
  for (int i = 12; i >= 0; i--) at = dd_add(dd_mul(at, t2), dd(k[2 * i], k[2 * i + 1]));
  at = dd_mul(at, t);
  Pair<double> r = dd_add(dd(CRM_ATAN_T17_DD[2 * j], CRM_ATAN_T17_DD[2 * j + 1]), at);
  return sw ? dd_add(dd(CRM_PIO2_D_HI, CRM_PIO2_D_LO), dd_neg(r)) : r;
}

// ------------------------------------------------------------------ FP64-free middle tier
// atanf, asinf and acosf in signed Q126 fixed point.  atan r for 0 <= r <= 1: j =
// rint(16 r), t = (r - j/16)/(1 + (j/16) r) by q_div (|t| <= 1/32), atan t by its Taylor
// series to degree 23 (remainder t^25/25 < 2^-129), atan(j/16) from a Q126 table.
// Products truncate by less than a unit and the constants by half a unit: atan r is
// within 2^10 units of 2^-126.
CRM_DEV U128 atan_q126(U128 R) {
  const int j = (int)(((R.hi >> 57) + 1) >> 1);  // rint(16 r): 16 r = R 2^-122
  const U128 N = sub128(R, U128{0ull, (uint64_t)j << 58});  // r - j/16, exact
  U128 t = {0ull, 0ull};
  if (N.hi | N.lo) {
    const U128 Rs = {(R.lo >> 4) | (R.hi << 60), R.hi >> 4};  // r/16, truncated
    U128 D = {0ull, 1ull << 62};                              // 1 + j r/16
    for (int i = 0; i < j; i++) D = add128(D, Rs);
    int es;
    t = q_div(N, D, es);  // D in [1, 2): es = 0
  }
  const U128 u = q_mul(t, t);
  U128 p = q_ld(CRM_ATANI_C + 20);
#pragma unroll
  for (int k = 9; k >= 0; k--) p = add128(q_ld(CRM_ATANI_C + 2 * k), q_mul(u, p));
  return add128(q_ld(CRM_ATANI_T + 2 * j), add128(t, q_mul(t, q_mul(u, p))));
}

// atan(a/b) for Q126 values a, b >= 0 with max(a, b) >= 2^-12: the smaller over the larger
// by q_div (relative 2^-118; w 2^es is the quotient, es <= 12, so its truncation is at most
// 2^12 units), pi/2 - atan(b/a) when a > b.  An error of e units in a or b moves the result
// by at most e 2^12 units (|d atan(a/b)/da| = b/(a^2 + b^2) <= 1/max(a, b)).
CRM_DEV U128 atan2_q126(U128 a, U128 b) {
  const bool sw = !le128(a, b);
  int es;
  const U128 w = q_div(sw ? b : a, sw ? a : b, es);
  const U128 v = atan_q126(q_shl(w, es));
  return sw ? sub128(q_ld(CRM_ATANI_PIO2), v) : v;
}

// sqrt d for a Q126 value 2^-24 <= d <= 1: s and k with sqrt d = s 2^-k, s in [1/2, 2).
// D = d 4^k in [1/2, 2) (exact), y = 1/sqrt D by three Newton steps y += y (1 - D y^2)/2
// from a binary32 seed (relative error 2^-21, then 2^-41, 2^-81, the truncation limit
// near 2^-123), s = D y.
CRM_DEV U128 q_sqrt(U128 d, int &k) {
  const int p = 127 - __clzll(d.hi);  // d.hi != 0 since d >= 2^-24
  k = (126 - p) >> 1;
  const U128 D = q_shl(d, 2 * k);
  const float y0 = rsqrtf((float)(D.hi >> 39) * 0x1p-23f);
  U128 y = {0ull, (uint64_t)(y0 * 0x1p38f) << 24};
  const U128 ONE = {0ull, 1ull << 62};
#pragma unroll
  for (int it = 0; it < 3; it++) {
    const U128 e = sub128(ONE, q_mul(q_mul(D, y), y));                   // 1 - D y^2, signed
    const U128 h = {(e.lo >> 1) | (e.hi << 63), (uint64_t)((int64_t)e.hi >> 1)};  // e / 2
    y = add128(y, q_mul(y, h));
  }
  return q_mul(D, y);
}

// atanf: r = |x| (exact) or 1/|x| (q_div, then shifted; 1/|x| is within 2^2 units) for
// |x| > 1, pi/2 minus the core for |x| > 1; error bound 2^11 units against results of at
// least 2^-12.  |x| < 2^-12 gives x (x^3/3 is below half an ulp), +-inf RN(+-pi/2).
CRM_DEV float atanf_int(float x, bool &hard, int *sg = nullptr) {
  hard = false;
  const float ax = fabsf(x);
  // atan x - x has the sign of -x; RN(pi/2) = 0x1.921fb6p+0 lies above pi/2
  put_sg(sg, -sgnf(x));
  if (ax < 0x1p-12f) return x;
  if (ax == CRM_INF_F) return copysignf(0x1.921fb6p+0f, x);
  const bool sw = ax > 1.0f;
  U128 R;  // r in Q126
  if (!sw) {
    R = q_of_f(ax);
  } else {  // 1/|x| = (1/m) 2^-(E - 127), m = M 2^-23 in [1, 2): 1/m from q_div, then shifted
    const uint32_t b = fbits(ax);
    int es;
    const U128 w = q_div(U128{0ull, 1ull << 62}, U128{0ull, (uint64_t)((b & 0x007FFFFFu) | 0x00800000u) << 39},
                         es);  // 1 / m in Q126 (es = 0)
    R = q_shr(w, (int)(b >> 23) - 127);
  }
  U128 v = atan_q126(R);
  if (sw) v = sub128(q_ld(CRM_ATANI_PIO2), v);
  const float y = q_round_f(v, U128{2048ull, 0ull}, hard, 0, sg);
  if (sg && x < 0.0f) *sg = -*sg;
  return x < 0.0f ? -y : y;
}

// asinf = sign(x) atan(|x| / s), acosf = atan(s / x) (x > 0), pi - atan(s / |x|) (x < 0),
// s = sqrt(1 - x^2) with 1 - x^2 exact in Q126 (|x| >= 2^-27 has its square's bits above
// 2^-126) and s within 2^-114 of itself relative (after the shift by k <= 12).  The
// errors: a, b exact or relative 2^-114 (2^12 units of 2^-126 on the quotient), q_div 2^12
// units, the core 2^10 units: bound 2^16 units against results of at least 2^-12.  acos of
// a negative x is formed as (pi - theta)/2 = pi/2 - theta/2 and rounded with es = 1.
// |x| = 1 and the tiny ranges (asin x = x below 2^-12, x + x^3/6 being within half an
// ulp; acos x = RN(pi/2) below 2^-27, pi/2 being 2^-25.8 from a midpoint) are direct.
template <int KIND> CRM_DEV float asincosf_int(float x, bool &hard, int *sg = nullptr) {
  hard = false;
  const float ax = fabsf(x);
  // asin x - x has the sign of x, RN(pi/2) = 0x1.921fb6p+0 and RN(pi) = 0x1.921fb6p+1 lie
  // above pi/2 and pi (and acos x < pi/2 + 2^-27 < RN(pi/2) for |x| < 2^-27)
  if (KIND == AT_ASIN) {
    put_sg(sg, sgnf(x));
    if (ax < 0x1p-12f) return x;
    put_sg(sg, -sgnf(x));
    if (ax == 1.0f) return copysignf(0x1.921fb6p+0f, x);
  } else {
    put_sg(sg, -1);
    if (ax < 0x1p-27f) return 0x1.921fb6p+0f;
    if (x == -1.0f) return 0x1.921fb6p+1f;
  }
  const U128 a = q_of_f(ax);
  int k;
  const U128 s = q_sqrt(sub128(U128{0ull, 1ull << 62}, q_mul(a, a)), k);
  const U128 sq = q_shr(s, k);
  if (KIND == AT_ASIN) {
    const float y = q_round_f(atan2_q126(a, sq), U128{1ull << 16, 0ull}, hard, 0, sg);
    if (sg && x < 0.0f) *sg = -*sg;
    return x < 0.0f ? -y : y;
  }
  const U128 th = atan2_q126(sq, a);
  if (x > 0.0f) return q_round_f(th, U128{1ull << 16, 0ull}, hard, 0, sg);
  return q_round_f(sub128(q_ld(CRM_ATANI_PIO2), q_shr(th, 1)), U128{1ull << 16, 0ull}, hard, 1, sg);
}

template <int KIND> CRM_DEV float atrig_slow(float x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = false;
  float sp;
  if (atrig_special<KIND>(x, sp)) {
    put_sg(sg, 0);
    return sp;
  }
  float r = KIND == AT_ATAN ? atanf_int(x, hard, sg) : asincosf_int<KIND>(x, hard, sg);
  if (!hard && !force) return r;
  if (sg) {  // the tiny ranges and the +-1 / +-inf ends are exact statements above
    const float ax = fabsf(x);
    if ((KIND == AT_ATAN && (ax < 0x1p-12f || ax == CRM_INF_F)) ||
        (KIND == AT_ASIN && (ax < 0x1p-12f || ax == 1.0f)) || (KIND == AT_ACOS && (ax < 0x1p-27f || x == -1.0f)))
      return r;
  }
  double ax = fabs((double)x);
  Pair<double> a, b;
  bool flip = false;
  if (KIND == AT_ATAN) {
    bool inf = fabsf(x) == CRM_INF_F;
    a = {inf ? 1.0 : ax, 0.0};
    b = {inf ? 0.0 : 1.0, 0.0};
  } else {
    Pair<double> s = dd_sqrt(dd((1.0 - ax) * (1.0 + ax), 0.0));
    if (KIND == AT_ASIN) {
      a = {ax, 0.0};
      b = s;
    } else {
      a = s;
      b = {ax, 0.0};
      flip = x < 0.0f;
    }
  }
  Pair<double> y = atan_ratio_dd(a, b);
  if (flip) y = dd_add(dd(CRM_PI_D_HI, CRM_PI_D_LO), dd_neg(y));
  if (KIND != AT_ACOS && x < 0.0f) y = dd_neg(y);
  r = round_dd_to_f(y.hi, y.lo, ATRIG_DD_EPS * fabs(y.hi), hard, sg);
  unresolved = hard ? 3 : 2;  // the double-double tier ran
  return r;
}

}  // namespace crm
