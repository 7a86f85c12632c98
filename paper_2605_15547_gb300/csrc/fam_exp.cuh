// fam_exp.cuh -- b^x for b in {e, 2, 10} (expf, exp2f, exp10f).
//
// Every tier follows the paper's exp2f scheme (Fig. 1, Sec. II.A): write the argument in
// base 2, t = x log2(b), split t = k + j/2^J + g with a small table of 2^(j/2^J) (at most
// 16 entries in the FP64 and double-double tiers, 64 in the double-float tier), evaluate
// 2^g by a polynomial, and scale by 2^k with integer exponent arithmetic.  Infinite and
// NaN inputs and the saturated ranges are handled in the same pass.
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"
#include "fam_f64.cuh"

namespace crm {

// KIND 0: e^x, 1: 2^x, 2: 10^x
template <int KIND> struct ExpK;
template <> struct ExpK<0> {
  static constexpr float C16 = CRM_LOG2E_X16_F, C64 = CRM_LOG2E_X64_F;
  static constexpr double D0 = CRM_LOG2E_D0, D1 = CRM_LOG2E_D1, D2 = CRM_LOG2E_D2;
  static constexpr float F0 = CRM_LOG2E_F0, F1 = CRM_LOG2E_F1;
  static constexpr float OVF = 89.0f, UNF = -104.0f;  // beyond: +inf / +0 for certain
  static constexpr float XOVF = CRM_EXPF_X_OVF, XZERO = CRM_EXPF_X_ZERO, XSUB = CRM_EXPF_X_SUB;
};
template <> struct ExpK<1> {
  static constexpr float C16 = 16.0f, C64 = 64.0f;
  static constexpr double D0 = 1.0, D1 = 0.0, D2 = 0.0;
  static constexpr float F0 = 1.0f, F1 = 0.0f;
  // 2^-150 is the exact midpoint between +0 and 2^-149: ties to even give +0
  static constexpr float OVF = 128.0f, UNF = -150.0f;
  static constexpr float XOVF = CRM_EXP2F_X_OVF, XZERO = CRM_EXP2F_X_ZERO, XSUB = CRM_EXP2F_X_SUB;
};
template <> struct ExpK<2> {
  static constexpr float C16 = CRM_LOG2_10_X16_F, C64 = CRM_LOG2_10_X64_F;
  static constexpr double D0 = CRM_LOG2_10_D0, D1 = CRM_LOG2_10_D1, D2 = CRM_LOG2_10_D2;
  static constexpr float F0 = CRM_LOG2_10_F0, F1 = CRM_LOG2_10_F1;
  static constexpr float OVF = 38.6f, UNF = -45.5f;
  static constexpr float XOVF = CRM_EXP10F_X_OVF, XZERO = CRM_EXP10F_X_ZERO, XSUB = CRM_EXP10F_X_SUB;
};



// Special inputs: returns true and the result when x is NaN or saturated.
template <int KIND> CRM_DEV bool exp_special(float x, float &r) {
  using K = ExpK<KIND>;
  r = (x != x) ? qnan_of(x) : (x >= K::OVF ? CRM_INF_F : 0.0f);
  return (x != x) || x >= K::OVF || x <= K::UNF;
}

// ------------------------------------------------------------------ plain (FP64) tier
// t = x log2 b = k + j/16 + g, |g| <= 1/32 + 2^-17.  2^g by its degree-6 Taylor
// polynomial (remainder <= 2^-51).  y = T[j] (1 + p) with one FMA, then y 2^k.
// Error budget (relative): table 2^-53, remainder 2^-51, reduction (two FMA roundings of
// g, constant split) 2^-57, polynomial roundings 2^-57, final FMA 2^-53: below 2^-50.4.
// eps = 2^-49, i.e. 16 units of y's last place: D = 17.
constexpr uint32_t EXP_PLAIN_D = 17;

template <int KIND> CRM_DEV double exp_plain_y(float x, const double *T16) {
  using K = ExpK<KIND>;
  float sh = fma_(x, K::C16, CRM_SHIFTER_F);
  int N = (int)(fbits(sh) - fbits(CRM_SHIFTER_F));
  float nf = sh - CRM_SHIFTER_F;  // N exactly
  double g;
  if (KIND == 1) {
    g = (double)fma_(nf, -0.0625f, x);  // x - N/16, exact (Sterbenz)
  } else {
    double xd = (double)x;
    g = fma_(xd, K::D0, (double)(nf * -0.0625f));
    g = fma_(xd, K::D1, g);
  }
  const double *a = CRM_EXP2_TAYLOR_D;
  double p = fma_(g, a[6], a[5]);
  p = fma_(g, p, a[4]);
  p = fma_(g, p, a[3]);
  p = fma_(g, p, a[2]);
  p = fma_(g, p, a[1]);
  p = p * g;
  double T = T16[N & 15];
  double y = fma_(T, p, T);
  return scale_d(y, N >> 4);
}

template <int KIND> CRM_DEV float exp_plain(float x, const double *T16, bool &hard) {
  float r;
  bool sp = exp_special<KIND>(x, r);
  double y = exp_plain_y<KIND>(x, T16);
  hard = !sp && hard_d_to_f(y, EXP_PLAIN_D);
  return sp ? r : __double2float_rn(y);
}

// ------------------------------------------------------------------ double-float tier
// t = th + tl (exact product x*C0 split by FMA, plus x*C1), N = rint(64 th),
// f = th - N/64 (exact), g = gh + gl = f + tl (Fast2Sum: f is 0 or a multiple of
// ulp(th) >= |tl|/2 in exponent), |g| <= 2^-7 + 2^-16.  With T = 2^(j/64) and
// U = T ln2 from a 64-entry float4 table (Th, Tl, Uh, Ul):
//   2^g T = Th + Uh gh + [Tl + Uh gl + Ul gh + T Q(gh) + ...],
//   Q(g) = g^2 (a2 + a3 g + a4 g^2),  a_k = (ln 2)^k / k!.
// The leading sum s = RN(Th + Uh gh) is one FMA; Th - s is exact (s lies within 2^-7 of
// Th >= 1), so a second FMA, Uh gh + (Th - s), gives its rounding error to 2^-24 of
// itself (2^-48 |s|); the bracket and that error are summed in float into r, and the
// pair (s, r), |r| < 2^-15 |s|, goes to the rounding test unnormalised (round_df).
// Error budget (relative to T): rounding of Q 2^-38.8, the dropped cross term
// 2 a2 gh gl 2^-39.1, t from x*C1 and the split of C 2^-40.7, a5 g^5 remainder 2^-44.6,
// tables 2^-48, the error term and the bracket roundings 2^-47: total < 2^-37.7, inside
// the test's 2^-37.
// Inputs outside [X_SUB, X_OVF]: +inf above X_OVF and +0 below X_ZERO (selects), a quiet
// NaN for NaN; results in the subnormal band [X_ZERO, X_SUB) are rounded to the subnormal grid
// from the same pair (below).
// b^x = 2^k (s + r) to 2^-37.7 of itself (budget above); sb is the shifter's bit pattern
// (k and the table index are read from it).
template <int KIND> CRM_DEV void exp_df_core(float x, const float4 *T64U, float &s, float &r, uint32_t &sb) {
  using K = ExpK<KIND>;
  float th, tl;
  if (KIND == 1) {
    th = x;
    tl = 0.0f;
  } else {
    th = x * K::F0;
    tl = fma_(x, K::F0, -th);
    tl = fma_(x, K::F1, tl);
  }
  float sh = fma_(th, 64.0f, CRM_SHIFTER_F);
  // N = rint(64 t) sits in the low bits of sh's pattern 0x4B400000 + N (0x4B400000 is 0
  // modulo 64): the table index is the pattern's low 6 bits
  sb = fbits(sh);
  float nf = sh - CRM_SHIFTER_F;
  float f = fma_(nf, -0.015625f, th);
  float gh, gl;
  if (KIND == 1) {
    gh = f;
    gl = 0.0f;
  } else {
    gh = f + tl;
    gl = tl - (gh - f);
  }
  float4 T = T64U[sb & 63u];
  float q = fma_(gh, CRM_EXP2_A4_F, CRM_EXP2_A3_F);
  q = fma_(gh, q, CRM_EXP2_A2_F);
  float Q = (gh * gh) * q;
  s = fma_(T.z, gh, T.x);
  const float z = fma_(T.z, gh, T.x - s);
  float b = (KIND == 1) ? T.y : fma_(T.z, gl, T.y);
  b = fma_(T.w, gh, b);
  b = fma_(T.x, Q, b);
  r = b + z;
}

// With sg (the directed-rounding kernels) the lane also reports the sign of b^x - y: the
// saturated results lie below +inf and above +0 (equal for x = +-inf), and the subnormal
// band's integer is compared with u itself.
template <int KIND> CRM_DEV float exp_df(float x, const float4 *T64U, bool &hard, int *sg = nullptr) {
  using K = ExpK<KIND>;
  if (sg && fabsf(x) < 0x1p-26f) {  // b^x - 1 has the sign of x and is below 2^-24: 1 or a neighbour
    hard = false;
    *sg = sgnf(x);
    return 1.0f;
  }
  float s, r;
  uint32_t sb;
  exp_df_core<KIND>(x, T64U, s, r, sb);
  // the exponent increment (N >> 6) << 23: sb >> 6 is N >> 6 plus 0x12D0000 (borrow
  // included), whose shift by 23 vanishes modulo 2^32
  const bool ok = (x >= K::XSUB) && (x <= K::XOVF);  // false for NaN
  if (!sg) {
    // round to nearest: overflow (+inf) and underflow to +0, common in inputs with a wide
    // range, by selects (measured: a branch there, or a warp-uniform in-range path, loses
    // on such inputs more than it gains on in-range ones); NaN and the subnormal band on
    // the rare branch below
    bool h;
    const float y = bitsf(fbits(round_df(s, r, h)) + ((sb >> 6) << 23));
    hard = ok && h;
    if (__builtin_expect(ok || x > K::XOVF || x < K::XZERO, 1)) return ok ? y : (x > 0.0f ? CRM_INF_F : 0.0f);
  } else if (__builtin_expect(ok, 1)) {
    const float y = round_df(s, r, hard, sg);
    const float out = bitsf(fbits(y) + ((sb >> 6) << 23));
    // e^x lies above 1 + x for x != 0 by x^2/2 + ..., which for |x| < 2^-12 is below the
    // error bound when x is small; when 1 + x is a binary32 number and the candidate, f(x)
    // is decided above it (arguments with few significant bits, e.g. binary16 inputs)
    if (KIND == 0 && sg && hard && fabsf(x) < 0x1p-12f) {
      const float u = 1.0f + x;
      if (u - 1.0f == x && out == u) {
        hard = false;
        *sg = 1;
      }
    }
    return out;
  }
  // Out of range (round to nearest: NaN or the subnormal band): +inf, +0, a quiet NaN, or
  // a subnormal result.
  hard = false;
  float y = x != x ? qnan_of(x) : (x > 0.0f ? CRM_INF_F : 0.0f);
  put_sg(sg, (x != x || fabsf(x) == CRM_INF_F) ? 0 : (x > 0.0f ? -1 : 1));
  if ((x >= K::XZERO) && (x < K::XSUB)) {
    // The result is the integer nearest to u = (s2 + l2) 2^(k + 149) times 2^-149, with
    // (s2, l2) the normalised pair (k + 149 in [-2, 23], the scaling exact).  With
    // q = rint(u_hi) and d = (u_hi - q) + u_lo, the nearest integer is q, q + 1
    // (d > 1/2) or q - 1 (d < -1/2); the pair's error (2^-37 of u < 2^-13) and d's
    // rounding (2^-24) can move u across a half-integer only when ||d| - 1/2| <= 2^-12:
    // those lanes go slow.
    const Pair<float> p = fast_two_sum(s, r);
    const int N = (int)(sb - fbits(CRM_SHIFTER_F));
    const float sc = bitsf((uint32_t)((N >> 6) + 149 + 127) << 23);
    const float uh = p.hi * sc, ul = p.lo * sc;
    const float q = rintf(uh);
    const float d = (uh - q) + ul;
    const float qi = q + (d > 0.5f ? 1.0f : (d < -0.5f ? -1.0f : 0.0f));
    hard = fabsf(fabsf(d) - 0.5f) <= 0x1p-12f;
    if (sg) {  // u - qi, decided unless u is within the error of the integer qi
      const float dq = d - (qi - q);
      hard = !(fabsf(dq) > 0x1p-12f);
      *sg = dq > 0.0f ? 1 : -1;
    }
    y = qi * 0x1p-149f;
  }
  return y;
}

// ------------------------------------------------------------------ register-table variant
// The double-float tier with a 16-entry table kept in registers instead of the 64-entry
// shared-memory table: lane l of every warp holds entry l mod 16 of (2^(j/16) hi, lo,
// 2^(j/16) ln2 hi, lo), and each lane fetches its entry with four warp shuffles (the
// paper's tables of at most 16 entries read by permutes instead of gathers, Sec. II.A).
// t = k + j/16 + g, |g| <= 2^-4.99, so the polynomial gains a degree and its quadratic
// term, up to 2^-12 of the result, is formed with exact products:
//   2^g T = Th + Uh gh + Th c2 + [Tl + Uh gl + Ul gh + Tl c2
//           + Th (c2l + a2 gh^2 - c2 - c2l + 2 a2 gh gl + g^3 (a3 + a4 g + a5 g^2 + a6 g^3))]
// with c2 + c2l = a2_hi gh^2 exactly.  s0 = RN(Th + Uh gh) and its error z (one FMA each),
// Th c2 = w + wl exactly, s = s0 + w by Fast2Sum (|w| <= 2^-12 |s0|) with error z2; the
// bracket, z, z2 and wl are summed in float into r.  Error budget, relative to the result:
// Taylor remainder a7 g^7 2^-50.9; the cubic tail's roundings 2^-41.6; the bracket's
// roundings (|bracket| <= 2^-19) 2^-41; the sum into r 2^-41.2; t from x C1 and the split of
// C 2^-40.7; tables and the dropped cross terms 2^-43: total < 2^-38, inside the test's
// 2^-37.
template <int KIND> CRM_DEV void exp_df16_core(float x, const float4 &R, float &s, float &r, uint32_t &sb) {
  using K = ExpK<KIND>;
  float th, tl;
  if (KIND == 1) {
    th = x;
    tl = 0.0f;
  } else {
    th = x * K::F0;
    tl = fma_(x, K::F0, -th);
    tl = fma_(x, K::F1, tl);
  }
  const float sh = fma_(th, 16.0f, CRM_SHIFTER_F);
  sb = fbits(sh);  // 0x4B400000 + N, N = rint(16 t); 0x4B400000 is 0 modulo 16
  const float nf = sh - CRM_SHIFTER_F;
  const float f = fma_(nf, -0.0625f, th);
  float gh, gl;
  if (KIND == 1) {
    gh = f;
    gl = 0.0f;
  } else {
    gh = f + tl;
    gl = tl - (gh - f);
  }
  const int j = (int)(sb & 15u);
  float4 T;
  T.x = __shfl_sync(0xFFFFFFFFu, R.x, j);
  T.y = __shfl_sync(0xFFFFFFFFu, R.y, j);
  T.z = __shfl_sync(0xFFFFFFFFu, R.z, j);
  T.w = __shfl_sync(0xFFFFFFFFu, R.w, j);
  float q = fma_(gh, CRM_EXP2_A6_F, CRM_EXP2_A5_F);
  q = fma_(gh, q, CRM_EXP2_A4_F);
  q = fma_(gh, q, CRM_EXP2_A3_F);
  const float g2 = gh * gh;
  const float g2l = fma_(gh, gh, -g2);
  const float c2 = CRM_EXP2_A2_HI_F * g2;
  const float c2l = fma_(CRM_EXP2_A2_HI_F, g2, -c2);
  const float w = T.x * c2;
  const float wl = fma_(T.x, c2, -w);
  const float s0 = fma_(T.z, gh, T.x);
  const float z = fma_(T.z, gh, T.x - s0);
  s = s0 + w;
  const float z2 = w - (s - s0);
  float tq = fma_(CRM_EXP2_A2_HI_F, g2l, CRM_EXP2_A2_LO_F * g2) + c2l;
  if (KIND != 1) tq = fma_((2.0f * CRM_EXP2_A2_F) * gh, gl, tq);
  tq = fma_(g2 * gh, q, tq);
  float b = (KIND == 1) ? T.y : fma_(T.z, gl, T.y);
  b = fma_(T.w, gh, b);
  b = fma_(T.y, c2, b);
  b = fma_(T.x, tq, b);
  r = ((b + z) + z2) + wl;
}

template <int KIND> CRM_DEV float exp_df16(float x, const float4 &R, bool &hard) {
  using K = ExpK<KIND>;
  float s, r;
  uint32_t sb;
  exp_df16_core<KIND>(x, R, s, r, sb);
  const bool ok = (x >= K::XSUB) && (x <= K::XOVF);  // false for NaN
  bool h;
  const float y0 = bitsf(fbits(round_df(s, r, h)) + ((sb >> 4) << 23));  // exponent increment N >> 4
  hard = ok && h;
  // out of range as in exp_df's general path (k = N >> 4)
  if (__builtin_expect(ok || x > K::XOVF || x < K::XZERO, 1)) return ok ? y0 : (x > 0.0f ? CRM_INF_F : 0.0f);
  hard = false;
  float y = x != x ? qnan_of(x) : (x > 0.0f ? CRM_INF_F : 0.0f);
  if ((x >= K::XZERO) && (x < K::XSUB)) {
    const Pair<float> p = fast_two_sum(s, r);
    const int N = (int)(sb - fbits(CRM_SHIFTER_F));
    const float sc = bitsf((uint32_t)((N >> 4) + 149 + 127) << 23);
    const float uh = p.hi * sc, ul = p.lo * sc;
    const float q = rintf(uh);
    const float d = (uh - q) + ul;
    const float qi = q + (d > 0.5f ? 1.0f : (d < -0.5f ? -1.0f : 0.0f));
    hard = fabsf(fabsf(d) - 0.5f) <= 0x1p-12f;
    y = qi * 0x1p-149f;
  }
  return y;
}

// ------------------------------------------------------------------ double-double tier
// t = x log2 b in double-double (x times a three-double constant), N = rint(16 t),
// g = t - N/16 (|g| <= 1/32 + tiny), 2^g by its degree-12 Taylor polynomial in
// double-double Horner form (remainder < 2^-104), times the double-double T[j].
// Error: 13 Horner steps at <= 8u^2 each plus the table and reduction: < 2^-98.
constexpr double EXP_DD_EPS = 0x1p-92;

template <int KIND> CRM_DEV Pair<double> exp_dd_core(float x, int &k) {
  using K = ExpK<KIND>;
  double xd = (double)x;
  Pair<double> t;
  if (KIND == 1) {
    t = {xd, 0.0};
  } else {
    t = two_prod(xd, K::D0);
    t.lo = fma_(xd, K::D1, t.lo);
    t.lo = fma_(xd, K::D2, t.lo);
  }
  double nd = rint(16.0 * t.hi);
  int N = (int)nd;
  double f = fma_(nd, -0.0625, t.hi);  // exact
  Pair<double> g = two_sum(f, t.lo);
  const double *c = CRM_EXP2_TAYLOR_DD;
  Pair<double> p = dd(c[24], c[25]);
  for (int i = 11; i >= 0; i--) p = dd_add(dd_mul(p, g), dd(c[2 * i], c[2 * i + 1]));
  int j = N & 15;
  Pair<double> T = dd(CRM_EXP2_T16_DD[2 * j], CRM_EXP2_T16_DD[2 * j + 1]);
  k = N >> 4;
  return dd_mul(T, p);
}

template <int KIND> CRM_DEV float exp_dd(float x, bool &hard, int *sg = nullptr) {
  int k;
  Pair<double> y = exp_dd_core<KIND>(x, k);
  double s = y.hi * pow2d(k), t = y.lo * pow2d(k);  // exact: results stay in double range
  return round_dd_to_f(s, t, EXP_DD_EPS * fabs(s), hard, sg);
}

// ------------------------------------------------------------------ FP64-free middle tier
// b^x = 2^(x log2 b) with the binary64 path's fixed-point core (exp2q_core: Y = 2^(x' - k)
// in Q124 to 2^54 units, 128-bit integer arithmetic): x' 2^96 is formed exactly for
// exp2f and, for e^x and 10^x, from the 24-bit significand times log2 e in Q125 or log2 10
// in Q124, truncated (argument error below 2 units of 2^-96, i.e. 2^29 units of Y: the
// bound is taken as 2^55).  Y is rounded to 24 bits (fewer for subnormal results) with an
// integer test against half an ulp; |x| < 2^-60 gives 1.  x is not special (no NaN, no
// saturation: those are resolved before).  Replaces the FP64 tier for the lanes the
// double-float test sends to the slow path (see logf_int).
// |x| log2(b) 2^96 for 2^-60 <= |x| < 2^8 (exact for b = 2, else truncated: below 2
// units), from the bit pattern ax of |x|
template <int KIND> CRM_DEV U128 expq_arg(uint32_t ax) {
  const int E = (int)(ax >> 23);
  const uint64_t M = (ax & 0x007FFFFFu) | 0x00800000u;  // |x| = M 2^(E - 150)
  U128 X;
  if (KIND == 1) {
    const int s = E - 54;  // M 2^s, s in [13, 80] for 2^-60 <= |x| < 2^8
    X.lo = s < 64 ? (M << s) : 0ull;
    X.hi = s < 64 ? (M >> (64 - s)) : (M << (s - 64));
  } else {
    const uint64_t ch = KIND == 0 ? CRM_EXPI_LOG2E_Q125_HI : CRM_EXPI_LOG2_10_Q124_HI;
    const uint64_t cl = KIND == 0 ? CRM_EXPI_LOG2E_Q125_LO : CRM_EXPI_LOG2_10_Q124_LO;
    const int F = KIND == 0 ? 125 : 124;
    const U128 ml = mul64w(M, cl), mh = mul64w(M, ch);  // M C as 192 bits p2:p1:p0
    const uint64_t p0 = ml.lo, p1 = ml.hi + mh.lo;
    const uint64_t p2 = mh.hi + (p1 < ml.hi ? 1ull : 0ull);
    const int sft = F - 96 - (E - 150);  // X = M C >> sft, sft in [45, 112]
    if (sft < 64) {
      X.lo = (p0 >> sft) | (p1 << (64 - sft));
      X.hi = (p1 >> sft) | (p2 << (64 - sft));
    } else {
      const int s2 = sft - 64;
      X.lo = s2 ? ((p1 >> s2) | (p2 << (64 - s2))) : p1;
      X.hi = p2 >> s2;
    }
  }
  return X;
}

template <int KIND> CRM_DEV float expf_int(float x, bool &hard, int *sg = nullptr) {
  const uint32_t ax = fbits(x) & 0x7FFFFFFFu;
  hard = false;
  put_sg(sg, sgnf(x));  // b^x - 1 has the sign of x
  if ((int)(ax >> 23) < 127 - 60) return 1.0f;
  U128 X = expq_arg<KIND>(ax);  // |x| log2(b) 2^96
  if (x < 0.0f) X = neg128(X);
  int k;
  const U128 Y = exp2q_core(X, (const ulonglong2 *)CRM_EXP2I_T, k);  // [2^124, 2^125)
  put_sg(sg, k >= 128 ? -1 : 1);
  if (k >= 128) return CRM_INF_F;  // b^x >= 2^128
  if (k < -150) return 0.0f;       // b^x < 2^-150
  // discard sh bits: 101 for a normal result, 101 + (-126 - k) <= 125 for a subnormal one
  const int sh = 101 + (k < -126 ? -126 - k : 0);
  const int s64 = sh - 64;  // 37 .. 61
  const uint64_t mant = Y.hi >> s64;
  const U128 rem = {Y.lo, Y.hi & ((1ull << s64) - 1ull)};
  const U128 dlt = sub128(rem, U128{0ull, 1ull << (s64 - 1)});
  const uint64_t ERR = 1ull << 55;
  hard = (dlt.hi == 0 && dlt.lo <= ERR) || (dlt.hi == ~0ull && dlt.lo >= 0ull - ERR);
  const uint32_t up = ((int64_t)dlt.hi > 0 || (dlt.hi == 0 && dlt.lo != 0)) ? 1u : 0u;
  if (sg) {  // the sign of v - y: decided unless the discarded part is within ERR of 0 or of a unit
    hard = le128(rem, U128{ERR, 0ull}) || le128(sub128(U128{0ull, 1ull << s64}, rem), U128{ERR, 0ull});
    *sg = up ? -1 : 1;
  }
  const uint32_t bits = k < -126 ? (uint32_t)mant + up : ((uint32_t)(k + 126) << 23) + (uint32_t)mant + up;
  return bitsf(bits);
}

// Slow path used for lanes whose fast-path test failed: the FP64-free tier, then
// double-double.
// With sg: the exact results, which no tier can decide by an error bound, are returned
// directly (2^x for integer x >= -149, 10^x for integer x in [1, 10], whose 5^x fits 24 bits).
template <int KIND> CRM_DEV float exp_slow(float x, int &unresolved, bool force, int *sg = nullptr) {
  unresolved = false;
  float sp;
  if (exp_special<KIND>(x, sp)) {
    put_sg(sg, (x != x || fabsf(x) == CRM_INF_F) ? 0 : (x > 0.0f ? -1 : 1));
    return sp;
  }
  bool hard;
  float r = expf_int<KIND>(x, hard, sg);
  if (!hard && !force) return r;
  // a sign stated by the first tier's shortcut (|x| < 2^-60: b^x - 1 has the sign of x) is
  // final: a deeper tier cannot decide a result that close to 1
  if (sg && !hard && fabsf(x) < 0x1p-60f) return r;
  if (sg && x == rintf(x)) {
    if (KIND == 1 && x >= -149.0f) {
      *sg = 0;
      return x >= -126.0f ? bitsf((uint32_t)((int)x + 127) << 23) : bitsf(1u << ((int)x + 149));
    }
    if (KIND == 2 && x >= 1.0f && x <= 10.0f) {
      float p = 1.0f;
      for (int i = 0; i < (int)x; i++) p *= 10.0f;  // exact: 10^10 < 2^34, 5^10 < 2^24
      *sg = 0;
      return p;
    }
  }
  r = exp_dd<KIND>(x, hard, sg);
  unresolved = hard ? 3 : 2;  // the double-double tier ran
  return r;
}

}  // namespace crm
