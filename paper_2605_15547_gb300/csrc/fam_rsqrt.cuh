// fam_rsqrt.cuh -- rsqrtf.
//
// 1/sqrt(x) is algebraic, so a hard case can be decided exactly: a binary32 midpoint m
// has at most 25 significant bits, so x m^2 is an integer of at most 74 bits times a
// power of two, and its comparison with 1 (never equal: 1/sqrt(x) is never a midpoint)
// tells on which side of m the true value lies.
#pragma once
#include "crm_common.cuh"
#include "fam_f64.cuh"

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
// y0 = the hardware reciprocal square root, rsqrt.approx.ftz (relative error below
// 2^-22.9 for a normal argument; subnormal x is scaled by 2^24, the result back by 2^12),
// the residual e = 1 - x y0^2 as 1 - h y0 - hl y0 with h + hl = x y0 exactly (h is about
// sqrt(x), normal for every normal x): two FMAs, each rounding at most 2^-24 of a value
// below 2^-20, so e is good to 2^-43 absolute; then one Newton step kept as a pair:
// y = y0 + y0 e (1/2 + 3e/8).  The truncation is (5/16) e^3 < 2^-61, the correction's
// roundings 2^-44 of y: relative error < 2^-42.5, inside the rounding test's 2^-37; the
// pair (y0, c), |c| < 2^-21 y0, goes to round_df unnormalised.
// Specials: a negative argument (half of a symmetric input range) takes the default NaN
// by a select; NaN, zeros and +inf (rare) a branch.
CRM_DEV float rsqrt_df(float x, bool &hard, int *sg = nullptr) {
  const uint32_t bx = fbits(x);
  const bool sub = bx < 0x00800000u;
  const float xs = x * (sub ? 0x1p24f : 1.0f);
  const float y0 = rsqrt_hw(xs);
  const float h = xs * y0;
  const float hl = fma_(xs, y0, -h);
  const float e = fma_(-hl, y0, fma_(-h, y0, 1.0f));
  const float corr = fma_(e, 0.375f, 0.5f) * e;
  const float c = y0 * corr;
  bool hh;
  const float yh = round_df(y0, c, hh, sg);
  const bool ok = (bx - 1u) < 0x7F7FFFFFu;  // positive, finite, nonzero
  hard = ok && hh;
  float res = ok ? yh * (sub ? 0x1p12f : 1.0f) : CRM_QNAN_F;
  if (sg && !ok) *sg = 0;  // +-inf, NaN, +0: exact
  if (__builtin_expect(!ok && !(x < 0.0f), 0)) rsqrt_special(x, res);
  return res;
}

// ------------------------------------------------------------------ exact slow tier
// Exact decision in integer arithmetic (no FP64): x is scaled into the normal range as in
// the double-float tier and y = that tier's rounded result, which is RN(1/sqrt(x)) or one
// of its two neighbours (the pair is within 2^-44.5, the rounding test's window 2^-36, of
// 1/sqrt(x), far less than an ulp).  With a = Ma 2^(Ea - 150) (Ma the 24-bit significand,
// Ea the exponent field) the midpoint between a and its successor is m = (2 Ma + 1)
// 2^(Ea - 151), and x m^2 = Mx Mm^2 2^(Ex + 2 Ea - 452) with Mx Mm^2 < 2^74: one 128-bit
// product against a power of two says whether m lies above 1/sqrt(x) (x m^2 > 1; never
// equal, 1/sqrt(x) is never a midpoint).  The answer is y's successor when 1/sqrt(x) lies
// above y's upper midpoint, its predecessor when below the lower one, else y.
CRM_DEV bool rsqrt_mid_above(uint32_t xb, uint32_t ab) {
  const uint64_t Mx = (xb & 0x007FFFFFu) | 0x00800000u;
  const uint64_t Mm = 2ull * ((ab & 0x007FFFFFu) | 0x00800000u) + 1ull;
  const int P = 452 - (int)(xb >> 23) - 2 * (int)(ab >> 23);  // x m^2 > 1 iff Mx Mm^2 > 2^P
  if (P < 0) return true;
  if (P >= 128) return false;
  const U128 prod = mul64w(Mx * Mm, Mm);
  return !le128(prod, P < 64 ? U128{1ull << P, 0ull} : U128{0ull, 1ull << (P - 64)});
}

// The sign of 1/sqrt(x) - y for a positive binary32 y (x scaled as above): the sign of
// 1 - x y^2, exactly, from Mx My^2 (< 2^72) against a power of two; 0 when x = 4^k / y^2.
CRM_DEV int rsqrt_cmp(uint32_t xb, uint32_t yb) {
  const uint64_t Mx = (xb & 0x007FFFFFu) | 0x00800000u;
  const uint64_t My = (yb & 0x007FFFFFu) | 0x00800000u;
  const int P = 450 - (int)(xb >> 23) - 2 * (int)(yb >> 23);  // x y^2 = Mx My^2 2^-P
  if (P < 0) return -1;
  if (P >= 128) return 1;
  const U128 prod = mul64w(Mx * My, My);
  const U128 one = P < 64 ? U128{1ull << P, 0ull} : U128{0ull, 1ull << (P - 64)};
  if (prod.hi == one.hi && prod.lo == one.lo) return 0;
  return le128(prod, one) ? 1 : -1;
}

CRM_DEV float rsqrt_slow(float x, int &unresolved, bool force, int *sg = nullptr) {
  (void)force;  // the exact decision is the only tier
  unresolved = false;
  float sp;
  if (rsqrt_special(x, sp)) {
    put_sg(sg, 0);
    return sp;
  }
  const bool sub = x < 0x1p-126f, big = x >= 0x1p64f;
  const float xs = sub ? x * 0x1p24f : (big ? x * 0x1p-64f : x);  // normal, in [2^-125, 2^64)
  bool h;
  const uint32_t xb = fbits(xs), yb = fbits(rsqrt_df(xs, h));
  uint32_t rb;
  if (sg) {  // the double-float result is within a fraction of an ulp: its exact side
    rb = yb;
    *sg = rsqrt_cmp(xb, yb);
  } else {
    rb = !rsqrt_mid_above(xb, yb) ? yb + 1u : (rsqrt_mid_above(xb, yb - 1u) ? yb - 1u : yb);
  }
  const float r = bitsf(rb);
  return sub ? r * 0x1p12f : (big ? r * 0x1p-32f : r);
}

}  // namespace crm
