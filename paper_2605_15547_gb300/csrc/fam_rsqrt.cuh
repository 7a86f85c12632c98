// fam_rsqrt.cuh -- rsqrtf.
//
// 1/sqrt(x) is algebraic, so a hard case can be decided exactly: the binary32 midpoint
// m next to the approximation has at most 25 significant bits, m^2 is exact in binary64,
// and the sign of x m^2 - 1 (one FMA, exact before its single rounding, never zero
// because 1/sqrt(x) is never a midpoint) tells on which side of m the true value lies.
#pragma once
#include "crm_common.cuh"

namespace crm {

CRM_DEV bool rsqrt_special(float x, float &r) {
  bool nan = x != x;
  r = nan ? qnan_of(x) : (x == 0.0f ? copysignf(CRM_INF_F, x) : (x < 0.0f ? CRM_QNAN_F : 0.0f));
  return nan || x <= 0.0f || x == CRM_INF_F;
}

// ------------------------------------------------------------------ plain (FP64) tier
// y0 from the hardware reciprocal square root on a normal binary32 (subnormal x is
// scaled by 2^48 first, the result by 2^24), then one Newton step in binary64 with the
// residual e = 1 - x y0^2 from an FMA: y = y0 + y0 e (1/2 + 3e/8).  |e| <= 2^-21 so the
// truncation is 2^-66 and the roundings give a relative error below 2^-51.5:
// eps = 2^-50 (D = 9).
CRM_DEV double rsqrt_plain_y(float x) {
  bool sub = x < 0x1p-126f;
  float xs = sub ? x * 0x1p48f : x;
  double xd = (double)xs;
  double y0 = (double)rsqrtf(xs);
  double h = xd * y0;
  double e = fma_(-h, y0, 1.0);
  double corr = fma_(e, 0.375, 0.5) * e;
  double y = fma_(y0, corr, y0);
  return sub ? y * 0x1p24 : y;
}

CRM_DEV float rsqrt_plain(float x, bool &hard) {
  float r;
  bool sp = rsqrt_special(x, r);
  double y = rsqrt_plain_y(sp ? 1.0f : x);
  hard = !sp && hard_d_to_f(y, 9);
  return sp ? r : __double2float_rn(y);
}

// ------------------------------------------------------------------ double-float tier
// y0 = hardware reciprocal square root (relative error below 2^-21; subnormal x scaled
// by 2^24 and x >= 2^64 by 2^-64, the result back by 2^12 or 2^-32), the residual e = 1 - x y0^2 from exact pair products
// (1 - p is exact by Sterbenz since x y0^2 is within 2^-20 of 1), and one Newton step
// kept as a pair: y = y0 + y0 e (1/2 + 3e/8).  |e| < 2^-20: the truncation is
// (5/16) e^3 < 2^-61, the residual is good to 2^-48 absolute, the correction product to
// 2^-24 of itself (2^-45 of y): relative error < 2^-44.5, inside the rounding test's
// 2^-37; the pair (y0, c), |c| < 2^-21 y0, goes to round_df unnormalised.
CRM_DEV float rsqrt_df(float x, bool &hard) {
  float r;
  bool sp = rsqrt_special(x, r);
  bool sub = x < 0x1p-126f, big = x >= 0x1p64f;  // keep y0^2 and its error normal
  float xs = sp ? 1.0f : (sub ? x * 0x1p24f : (big ? x * 0x1p-64f : x));
  float y0 = rsqrtf(xs);
  float s = y0 * y0;
  float sl = fma_(y0, y0, -s);
  float p = xs * s;
  float pl = fma_(xs, s, -p);
  float e = (1.0f - p) - fma_(xs, sl, pl);
  float corr = fma_(e, 0.375f, 0.5f) * e;
  float c = y0 * corr;
  bool h;
  const float yh = round_df(y0, c, h);
  // special inputs (x <= 0, NaN, +inf) by selects: they are common in real data (half of
  // a symmetric input range), so a branch would diverge in most warps
  hard = !sp && h;
  float out = sub ? yh * 0x1p12f : (big ? yh * 0x1p-32f : yh);
  return sp ? r : out;
}

// ------------------------------------------------------------------ exact slow tier
// Exact decision: the binary32 neighbours dn <= y <= up of the approximation and their
// midpoint m; RN(1/sqrt(x)) is up when x m^2 < 1, dn otherwise.  If y is itself a
// binary32 value (dn == up) it lies within 2^-50 of 1/sqrt(x) while the midpoints are
// 2^-25 away, so it is the answer.
CRM_DEV float rsqrt_slow(float x, bool &unresolved, bool force) {
  bool hard;
  float r = rsqrt_plain(x, hard);
  unresolved = false;
  float sp;
  if ((!hard && !force) || rsqrt_special(x, sp)) return r;
  double y = rsqrt_plain_y(x);
  float dn = __double2float_rd(y), up = __double2float_ru(y);
  if (dn == up) return dn;
  double m = 0.5 * ((double)dn + (double)up);  // 25 significant bits at most
  double m2 = m * m;                           // exact
  double v = fma_((double)x, m2, -1.0);        // sign of x m^2 - 1, exactly
  return v < 0.0 ? up : dn;
}

}  // namespace crm
