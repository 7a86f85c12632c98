// fam_hyp.cuh -- expm1f, sinhf, coshf, tanhf.
//
// All four reuse the exp reduction x log2(e) = k + j/16 + g of fam_exp.cuh (the
// paper's Fig. 1 scheme) and arrange the reconstruction so that no leading 1 cancels:
//   expm1: e^x - 1 = 2^k [ (T_j - 2^-k) + T_j p(g) ],    p(g) = 2^g - 1;
//   sinh, cosh: with A = 2^(k-1) T_j and B = 2^(-k-1) / T_j (the table entry of -x),
//     2 sinh|x| = (A - B)(1 + Ev) + (A + B) O,   2 cosh x = (A + B)(1 + Ev) + (A - B) O,
//     where 2^g = 1 + O + Ev splits the polynomial into odd and even parts; for j = k = 0
//     A - B is exactly 0 and sinh keeps full relative accuracy near 0;
//   tanh = sinh / cosh from the same pieces.
#pragma once
#include "fam_exp.cuh"

namespace crm {

enum { HYP_EXPM1 = 0, HYP_SINH = 1, HYP_COSH = 2, HYP_TANH = 3 };

struct ExpRedD {
  double g;
  int k, j;
};
// x log2 e = 16 k + j + 16 g (|g| <= 1/32 + 2^-17), g from two FMAs (error 2^-57 abs)
CRM_DEV ExpRedD exp_reduce_d(float x) {
  float sh = fma_(x, CRM_LOG2E_X16_F, CRM_SHIFTER_F);
  int N = (int)(fbits(sh) - fbits(CRM_SHIFTER_F));
  float nf = sh - CRM_SHIFTER_F;
  double xd = (double)x;
  double g = fma_(xd, CRM_LOG2E_D0, (double)(nf * -0.0625f));
  g = fma_(xd, CRM_LOG2E_D1, g);
  return {g, N >> 4, N & 15};
}

// Special inputs: returns true with the result in r.
template <int H> CRM_DEV bool hyp_special(float x, float &r) {
  float ax = fabsf(x);
  bool nan = x != x;
  if (H == HYP_EXPM1) {
    const bool st = x >= CRM_EXPM1F_X_MONE && x <= CRM_EXPM1F_X_M2;  // -1 + 2^-24
    r = nan ? qnan_of(x) : (x == 0.0f ? x : (st ? -0x1.fffffep-1f : (x > 0.0f ? CRM_INF_F : -1.0f)));
    return nan || x == 0.0f || x > CRM_EXPF_X_OVF || x < CRM_EXPM1F_X_MONE || st;
  }
  if (H == HYP_SINH) {
    r = nan ? qnan_of(x) : (x == 0.0f ? x : copysignf(CRM_INF_F, x));
    return nan || x == 0.0f || ax > CRM_SINHF_X_OVF;
  }
  if (H == HYP_COSH) {
    r = nan ? qnan_of(x) : CRM_INF_F;
    return nan || ax > CRM_SINHF_X_OVF;
  }
  const bool st = ax > CRM_TANHF_X_NEXT && ax <= CRM_TANHF_X_ONE;  // +-(1 - 2^-24)
  r = nan ? qnan_of(x) : (x == 0.0f ? x : copysignf(st ? 0x1.fffffep-1f : 1.0f, x));
  return nan || x == 0.0f || ax > CRM_TANHF_X_NEXT;
}

// The sign of f(x) - r for the results of the special branches (0 for exact ones); the
// first saturation steps (expm1 -1 + 2^-24, tanh +-(1 - 2^-24)) lie on either side of f(x)
// and are left to the slow path (hard).  Tiny |x| < 2^-25: expm1 x - x = x^2/2 + ... > 0,
// sinh x - x has the sign of x, tanh x - x the opposite, cosh x - 1 > 0; saturated
// results are +-inf or +-1 beyond f(x), f(x) -1 above -1.
template <int H> CRM_DEV int hyp_special_sg(float x, bool &hard) {
  const float ax = fabsf(x);
  if (x != x || x == 0.0f || ax == CRM_INF_F) return 0;
  if (ax < 0x1p-25f) return H == HYP_EXPM1 || H == HYP_COSH ? 1 : (H == HYP_SINH ? sgnf(x) : -sgnf(x));
  if (H == HYP_EXPM1) {
    if (x > 0.0f) return -1;  // +inf beyond
    if (x < CRM_EXPM1F_X_MONE) return 1;  // -1 below
    hard = true;  // the -1 + 2^-24 step
    return 0;
  }
  if (H == HYP_TANH && ax <= CRM_TANHF_X_ONE) {
    hard = true;  // the 1 - 2^-24 step
    return 0;
  }
  return H == HYP_COSH ? -1 : -sgnf(x);  // +-inf, or +-1 for tanh
}

// ------------------------------------------------------------------ plain (FP64) tier
// Errors (relative to the result): table entries 2^-53 each, amplified by at most
// (A + B)/|result| <= 46 where A and B do not cancel exactly (j or k nonzero means
// |x| >= ln2/32); polynomial remainders <= 2^-51 relative to their leading term;
// roundings 2^-53 per operation.  expm1, sinh, cosh: eps = 2^-46 (D = 129);
// tanh adds a division: eps = 2^-45 (D = 257).
template <int H> CRM_DEV double hyp_plain_y(float x, const double *T16) {
  const double *a = CRM_EXP2_TAYLOR_D;  // a_k = (ln 2)^k / k!
  if (H == HYP_EXPM1) {
    ExpRedD R = exp_reduce_d(x);
    double p = fma_(R.g, a[6], a[5]);
    p = fma_(R.g, p, a[4]);
    p = fma_(R.g, p, a[3]);
    p = fma_(R.g, p, a[2]);
    p = fma_(R.g, p, a[1]);
    p = p * R.g;
    double T = T16[R.j];
    double y = fma_(T, p, T - pow2d(-R.k));
    return scale_d(y, R.k);
  }
  ExpRedD R = exp_reduce_d(fabsf(x));
  double g2 = R.g * R.g;
  // odd part: a1 g + a3 g^3 + a5 g^5 + a7 g^7 ; even part: a2 g^2 + a4 g^4 + a6 g^6
  double O = R.g * fma_(g2, fma_(g2, fma_(g2, a[7], a[5]), a[3]), a[1]);
  double Ev = g2 * fma_(g2, fma_(g2, a[6], a[4]), a[2]);
  int jb = (16 - R.j) & 15;
  int kb = -R.k - (R.j != 0 ? 1 : 0);
  double A = scale_d(T16[R.j], R.k - 1);
  double B = scale_d(T16[jb], kb - 1);
  double D = A - B, S = A + B;
  double sh = fma_(S, O, fma_(D, Ev, D));
  double ch = fma_(D, O, fma_(S, Ev, S));
  if (H == HYP_SINH) return x < 0.0f ? -sh : sh;
  if (H == HYP_COSH) return ch;
  double t = sh / ch;
  return x < 0.0f ? -t : t;
}

template <int H> constexpr uint32_t hyp_plain_D() { return H == HYP_TANH ? 257u : 129u; }

template <int H> CRM_DEV float hyp_plain(float x, const double *T16, bool &hard) {
  float r;
  bool sp = hyp_special<H>(x, r);
  double y = hyp_plain_y<H>(sp ? 0.5f : x, T16);
  hard = !sp && hard_d_to_f(y, hyp_plain_D<H>());
  return sp ? r : __double2float_rn(y);
}

// ------------------------------------------------------------------ double-float tier
// Precise expm1 core: x log2 e = k + j/64 + g (as in exp_df) and, with T = 2^(j/64) and
// U = T ln 2 from the 64-entry float4 table,
//     Y = 2^-k (e^x - 1) = (T - 2^-k) + U g + T Q(g),   Q = a2 g^2 + a3 g^3 + a4 g^4 + a5 g^5,
// where g^2 is an exact pair and a2 g^2 a pair product, so that Q is good to 2^-46 of
// itself; T - 2^-k is an exact pair (TwoSum).  (T - 2^-k) + U g cancels exactly when
// j = k = 0 and by at most a factor 4 otherwise.  Error (relative to Y): 2^-48 |t| from
// the reduction of t = x log2 e (below 2^-41 at |t| = 128, where nothing cancels),
// 2^-44 elsewhere after cancellation; the a6 g^6 remainder 2^-51.7.  The derived
// functions add one pair division or product (2^-43): all stay below 2^-40, within the
// 2^-37 that the rounding test (round_df) allows.
struct DFY {
  float s, l;  // Y = s + l unnormalised, |l| < 2^-20 |s| (or Y = 0)
  int k;       // e^x - 1 = 2^k Y
};

CRM_DEV DFY expm1_df_core(float x, const float4 *T64U) {
  float th = x * CRM_LOG2E_F0;
  float tl = fma_(x, CRM_LOG2E_F0, -th);
  tl = fma_(x, CRM_LOG2E_F1, tl);
  float sh = fma_(th, 64.0f, CRM_SHIFTER_F);
  int N = (int)(fbits(sh) - fbits(CRM_SHIFTER_F));
  float nf = sh - CRM_SHIFTER_F;
  float f = fma_(nf, -0.015625f, th);
  float gh = f + tl;
  float gl = tl - (gh - f);
  float4 T = T64U[N & 63];
  int k = N >> 6;
  // Q(g) as a pair
  float q2 = gh * gh;
  float q2l = fma_(gh, gh, -q2);
  q2l = fma_(2.0f * gh, gl, q2l);
  float Qh = CRM_EXP2_A2_HI_F * q2;
  float Ql = fma_(CRM_EXP2_A2_HI_F, q2, -Qh);
  Ql = fma_(CRM_EXP2_A2_HI_F, q2l, Ql);
  Ql = fma_(CRM_EXP2_A2_LO_F, q2, Ql);
  float tail = fma_(gh, fma_(gh, CRM_EXP2_A5_F, CRM_EXP2_A4_F), CRM_EXP2_A3_F);
  Ql = fma_(q2 * gh, tail, Ql);
  // T - 2^-k (2^-k negligible against T >= 1 when k > 100)
  float m = k > 100 ? 0.0f : -bitsf((uint32_t)(127 - k) << 23);
  Pair<float> c = two_sum(T.x, m);
  float cl = c.lo + T.y;
  // U g
  float u = T.z * gh;
  float ul = fma_(T.z, gh, -u);
  ul = fma_(T.z, gl, ul);
  ul = fma_(T.w, gh, ul);
  // T Q
  float tq = T.x * Qh;
  float tql = fma_(T.x, Qh, -tq);
  tql = fma_(T.x, Ql, tql);
  tql = fma_(T.y, Qh, tql);
  // T - 2^-k is 0 (j = k = 0) or at least 0.0107 T in magnitude (2^(j/64) - 1 for k = 0,
  // 2 - 2^(j/64) for k = -1, more for other k), while |U g| <= T ln2 (2^-7 + 2^-16) <
  // 0.0055 T: Fast2Sum applies
  Pair<float> s1 = fast_two_sum(c.hi, u);
  Pair<float> s2 = fast_two_sum(s1.hi, tq);  // |s1| >= |tq| (see above)
  float lo = (s1.lo + s2.lo) + (cl + (ul + tql));
  return {s2.hi, lo, k};
}

CRM_DEV float pow2f_exact(int k) { return bitsf((uint32_t)(k + 127) << 23); }  // k in [-126, 127]
CRM_DEV float scale_f(float y, int k) { return bitsf(fbits(y) + ((uint32_t)k << 23)); }

// The unrounded double-float result and its scale, f = 2^sc (r.hi + r.lo), for arg = x
// (expm1), |x| (sinh, cosh) or 2|x| (tanh), arg not special (hyp_df handles those).
template <int H> CRM_DEV Pair<float> hyp_df_core(float arg, const float4 *T64U, int &sc) {
  Pair<float> r;
  sc = 0;
  if (H == HYP_COSH) {
    // cosh a = (e^a + e^-a)/2 never cancels, so the exp core suffices (no expm1 care):
    // e^a = 2^k P with P to 2^-37.7 (exp_df_core), R = 2^-k / P by a pair division, and
    // cosh a = 2^(k-1) (P + 2^-k R): the two terms keep P's relative error, the division
    // and the sums add 2^-43: below the 2^-37 of the rounding test.
    float ps, pr;
    uint32_t sb;
    exp_df_core<0>(arg, T64U, ps, pr, sb);
    const int k = (int)(sb - fbits(CRM_SHIFTER_F)) >> 6;
    const Pair<float> P = fast_two_sum(ps, pr);  // normalised for the division
    const float pk = k > 100 ? 0.0f : pow2f_exact(-k);
    Pair<float> R = df_div({pk, 0.0f}, P);
    float rk = R.hi * pk, rkl = R.lo * pk;
    r = fast_two_sum(P.hi, rk);
    r.lo = r.lo + (P.lo + rkl);  // unnormalised, |r.lo| < 2^-22 |r.hi|
    sc = k - 1;
  } else {
  DFY Y = expm1_df_core(arg, T64U);
  if (H == HYP_EXPM1) {
    r = {Y.s, Y.l};
    sc = Y.k;
  } else if (H == HYP_TANH) {
    // tanh a = Y / (Y + 2^(1-k)) with e^(2a) - 1 = 2^k Y (Y normalised for the division)
    const Pair<float> Yn = fast_two_sum(Y.s, Y.l);
    Pair<float> d = two_sum(Yn.hi, pow2f_exact(1 - Y.k));
    d.lo = d.lo + Yn.lo;
    r = df_div_raw(Yn, d);
  } else {
    const Pair<float> Yn = fast_two_sum(Y.s, Y.l);
    float pk = Y.k > 100 ? 0.0f : pow2f_exact(-Y.k);
    Pair<float> P = two_sum(Yn.hi, pk);  // P = 2^-k e^a
    P.lo = P.lo + Yn.lo;
    Pair<float> R = df_div({pk, 0.0f}, P);  // 2^-2k e^-a ... = 2^-k / P
    // sinh a = 2^(k-1) Y (1 + R)
    Pair<float> onep = fast_two_sum(1.0f, R.hi);  // 1 + R as a pair (R <= 1)
    onep.lo = onep.lo + R.lo;
    r = df_mul_raw(Yn, onep);
    sc = Y.k - 1;
  }
  }
  return r;
}

template <int H> CRM_DEV float hyp_df(float x, const float4 *T64U, bool &hard, int *sg = nullptr) {
  float ax = fabsf(x);
  if (sg && H != HYP_EXPM1 && ax < 0x1p-12f) {
    // sinh x, tanh x within |x|^3/3 of x (above, below), cosh x within x^2/2 above 1
    hard = false;
    *sg = H == HYP_COSH ? (x == 0.0f ? 0 : 1) : (H == HYP_SINH ? sgnf(x) : -sgnf(x));
    return H == HYP_COSH ? 1.0f : x;
  }
  bool tiny = ax < 0x1p-25f;  // the correctly rounded result is x itself (or 1 for cosh)
  bool sp;                    // NaN, tiny, saturated (results by selects; a branch with sg)
  if (H == HYP_EXPM1) {
    // below X_MONE: -1; in [X_MONE, X_M2]: -1 + 2^-24 (the first step of the staircase)
    sp = !(x > CRM_EXPM1F_X_M2 && x <= CRM_EXPF_X_OVF) || tiny;
  } else if (H == HYP_SINH || H == HYP_COSH) {
    sp = !(ax <= CRM_SINHF_X_OVF) || tiny;
  } else {
    // above X_ONE: +-1; in (X_NEXT, X_ONE]: +-(1 - 2^-24)
    sp = !(ax <= CRM_TANHF_X_NEXT) || tiny;
  }
  float arg = H == HYP_EXPM1 ? x : (H == HYP_TANH ? 2.0f * ax : ax);
  arg = sp ? 0.5f : arg;
  int sc = 0;
  const Pair<float> r = hyp_df_core<H>(arg, T64U, sc);
  if (!sg) {
    // round to nearest: tiny and saturated arguments (common: tiny bit patterns, |x| > 9
    // for tanh on a symmetric range) and NaN by selects
    bool h;
    float y = scale_f(round_df(r.hi, r.lo, h), sc);
    if (H == HYP_SINH || H == HYP_TANH) y = x < 0.0f ? -y : y;
    hard = !sp && h;
    float v;
    if (H == HYP_EXPM1)
      v = tiny ? x : (x > 0.0f ? CRM_INF_F : (x < CRM_EXPM1F_X_MONE ? -1.0f : -0x1.fffffep-1f));
    else if (H == HYP_SINH)
      v = tiny ? x : copysignf(CRM_INF_F, x);
    else if (H == HYP_COSH)
      v = tiny ? 1.0f : CRM_INF_F;
    else
      v = tiny ? x : copysignf(ax > CRM_TANHF_X_ONE ? 1.0f : 0x1.fffffep-1f, x);
    return x != x ? qnan_of(x) : (sp ? v : y);
  }
  if (__builtin_expect(!sp, 1)) {
    // r unnormalised: |r.lo| < 2^-20 |r.hi| in every branch above
    float y = scale_f(round_df(r.hi, r.lo, hard, sg), sc);
    if (H == HYP_SINH || H == HYP_TANH) {
      if (sg && x < 0.0f) *sg = -*sg;
      y = x < 0.0f ? -y : y;
    }
    return y;
  }
  hard = false;
  if (sg) *sg = hyp_special_sg<H>(x, hard);
  if (x != x) return qnan_of(x);
  if (H == HYP_EXPM1)
    return tiny ? x : (x > 0.0f ? CRM_INF_F : (x < CRM_EXPM1F_X_MONE ? -1.0f : -0x1.fffffep-1f));
  if (H == HYP_SINH) return tiny ? x : copysignf(CRM_INF_F, x);
  if (H == HYP_COSH) return tiny ? 1.0f : CRM_INF_F;
  return tiny ? x : copysignf(ax > CRM_TANHF_X_ONE ? 1.0f : 0x1.fffffep-1f, x);
}

// ------------------------------------------------------------------ double-double tier
// The same formulas in double-double: g to 2^-106 (x times a three-double log2 e), the
// double-double table, Taylor polynomials to degree 12 (2^g - 1) or 13 / 12 (odd /
// even parts), remainders below 2^-104.  Error < 2^-97 relative (the table and product
// errors are amplified by at most 46 as above).
constexpr double HYP_DD_EPS = 0x1p-90;

struct ExpRedDD {
  Pair<double> g;
  int k, j;
};
CRM_DEV ExpRedDD exp_reduce_dd(float x) {
  double xd = (double)x;
  Pair<double> t = two_prod(xd, CRM_LOG2E_D0);
  t.lo = fma_(xd, CRM_LOG2E_D1, t.lo);
  t.lo = fma_(xd, CRM_LOG2E_D2, t.lo);
  double nd = rint(16.0 * t.hi);
  int N = (int)nd;
  double f = fma_(nd, -0.0625, t.hi);
  return {two_sum(f, t.lo), N >> 4, N & 15};
}
CRM_DEV Pair<double> ddtab(const double *t, int i) { return dd(t[2 * i], t[2 * i + 1]); }
CRM_DEV Pair<double> dd_scale(Pair<double> a, int k) {
  double s = pow2d(k);
  return {a.hi * s, a.lo * s};
}

template <int H> CRM_DEV Pair<double> hyp_dd_y(float x) {
  const double *c = CRM_EXP2_TAYLOR_DD;
  if (H == HYP_EXPM1) {
    ExpRedDD R = exp_reduce_dd(x);
    Pair<double> p = ddtab(c, 12);
    for (int i = 11; i >= 1; i--) p = dd_add(dd_mul(p, R.g), ddtab(c, i));
    p = dd_mul(p, R.g);
    Pair<double> T = ddtab(CRM_EXP2_T16_DD, R.j);
    Pair<double> y = dd_add(dd_add_d(T, -pow2d(-R.k)), dd_mul(T, p));
    return dd_scale(y, R.k);
  }
  ExpRedDD R = exp_reduce_dd(fabsf(x));
  Pair<double> g2 = dd_sqr(R.g);
  Pair<double> O = ddtab(c, 13), Ev = ddtab(c, 14);
  for (int i = 11; i >= 1; i -= 2) O = dd_add(dd_mul(O, g2), ddtab(c, i));
  O = dd_mul(O, R.g);
  for (int i = 12; i >= 2; i -= 2) Ev = dd_add(dd_mul(Ev, g2), ddtab(c, i));
  Ev = dd_mul(Ev, g2);
  int jb = (16 - R.j) & 15;
  int kb = -R.k - (R.j != 0 ? 1 : 0);
  Pair<double> A = dd_scale(ddtab(CRM_EXP2_T16_DD, R.j), R.k - 1);
  Pair<double> B = dd_scale(ddtab(CRM_EXP2_T16_DD, jb), kb - 1);
  Pair<double> D = dd_add(A, dd_neg(B)), S = dd_add(A, B);
  Pair<double> sh = dd_add(dd_add(D, dd_mul(D, Ev)), dd_mul(S, O));
  Pair<double> ch = dd_add(dd_add(S, dd_mul(S, Ev)), dd_mul(D, O));
  Pair<double> y = H == HYP_SINH ? sh : (H == HYP_COSH ? ch : dd_div(sh, ch));
  if (H != HYP_COSH && x < 0.0f) y = dd_neg(y);
  return y;
}

// ------------------------------------------------------------------ FP64-free middle tier
// sinhf and coshf from the fixed-point exp2 core (exp2q_core: e^a = Y 2^(k - 124), Y in
// [2^124, 2^125), error 2^54 units, plus 2^29 from the truncated argument a log2 e 2^96):
// sinh a = (e^a - e^-a)/2, cosh a = (e^a + e^-a)/2 (a = |x|, k1 >= 0 > k2), e^-a aligned
// to e^a's scale.  The error bound is absolute in units of that scale (2^56), so sinh's
// cancellation near 0 is accounted for by the rounding test itself (|x| >= 2^-25 keeps
// the result above 2^99 units).
template <int H> CRM_DEV float hyp_int(float x, bool &hard, int *sg = nullptr) {
  const uint32_t ax = fbits(x) & 0x7FFFFFFFu;
  const U128 Xa = expq_arg<0>(ax);  // |x| log2 e 2^96; |x| >= 2^-25 here
  const ulonglong2 *T = (const ulonglong2 *)CRM_EXP2I_T;
  const U128 ERR = {1ull << 56, 0ull};
  int k1, k2;
  const U128 Y1 = exp2q_core(Xa, T, k1), Y2 = exp2q_core(neg128(Xa), T, k2);
  const int d = k1 - k2;  // >= 1
  U128 Y2s = {0ull, 0ull};
  if (d < 64) {
    Y2s = {(Y2.lo >> d) | (Y2.hi << (64 - d)), Y2.hi >> d};
  } else if (d < 128) {
    Y2s = {Y2.hi >> (d - 64), 0ull};
  }
  const U128 V = H == HYP_COSH ? add128(Y1, Y2s) : sub128(Y1, Y2s);  // 2 f(a) 2^(124 - k1)
  const float y = q_round_f(V, ERR, hard, k1 + 1, sg);
  if (H == HYP_SINH && x < 0.0f && sg) *sg = -*sg;
  return (H == HYP_SINH && x < 0.0f) ? -y : y;
}

// expm1f and tanhf in signed Q126, FP64-free, without the cancellation of e^x - 1 near 0:
//   expm1: |x| < 2^-25 gives x (x^2/2 is below half an ulp on either side); |x| < 2^-4:
//     x sum_{k<=12} x^k/(k+1)! by Horner (remainder below 2^-88 of the result, products
//     truncated: 16 units; bound 2^-84 of it plus 16 units); otherwise from the exp2 core, e^x = Y 2^(k-124) (Y within 2^54
//     units): (Y - 2^(124-k)) 2^2 with es = k for k >= 0, Y 2^(k+2) - 2^126 for k < 0, both
//     at least e^(1/16) - 1 > 2^-4 of their scale: error 2^57 units, 2^-65 relative;
//   tanh = expm1(2x)/(expm1(2x) + 2): |x| < 2^-13 gives x (x^3/3 is below half an ulp);
//     2|x| < 2^-4: m/(m + 1), m = expm1(2|x|)/2 by the series, one q_div (m's relative error
//     at most doubles); otherwise with
//     e^(2|x|) = Y 2^(k-124): (Y - 2^(124-k))/(Y + 2^(124-k)), whose absolute error is at
//     most 2^-70 (Y/D)(1 + N/D) <= 2^-69 (2^57 units; bound 2^58) though N may cancel to 2^-4.
// The special inputs and the saturated ranges are handled before (hyp_special).
CRM_DEV U128 expm1_series_q126(U128 X) {  // x sum x^k/(k+1)!, |x| < 2^-4
  U128 E = q_ld(CRM_HYPI_E + 24);
#pragma unroll
  for (int k = 11; k >= 0; k--) E = add128(q_ld(CRM_HYPI_E + 2 * k), q_mul(X, E));
  return q_mul(X, E);
}

CRM_DEV U128 rel_err_84(U128 v) {  // |v| 2^-84 + 16 units
  const U128 A = q_neg(v) ? neg128(v) : v;
  return {(A.hi >> 20) + 16ull, 0ull};
}

template <int H> CRM_DEV float hyp_int2(float x, bool &hard, int *sg = nullptr) {
  hard = false;
  const float ax = fabsf(x);
  const U128 ONE = {0ull, 1ull << 62};
  const ulonglong2 *T = (const ulonglong2 *)CRM_EXP2I_T;
  if (H == HYP_EXPM1) {
    put_sg(sg, 1);  // expm1 x > x
    if (ax < 0x1p-25f) return x;
    if (ax < 0x1p-4f) {
      const U128 X = x < 0.0f ? neg128(q_of_f(ax)) : q_of_f(ax);
      const U128 v = expm1_series_q126(X);
      return q_round_f(v, rel_err_84(v), hard, 0, sg);
    }
    U128 Xa = expq_arg<0>(fbits(ax));
    if (x < 0.0f) Xa = neg128(Xa);
    int k;
    const U128 Y = exp2q_core(Xa, T, k);
    const U128 E57 = {1ull << 57, 0ull};
    if (k >= 0) {
      const U128 W = k <= 124 ? sub128(Y, q_shr(U128{0ull, 1ull << 60}, k)) : Y;  // 2^124 >> k
      return q_round_f(q_shl(W, 2), E57, hard, k, sg);
    }
    const U128 Ys = k == -1 ? q_shl(Y, 1) : q_shr(Y, -k - 2);
    return q_round_f(sub128(Ys, ONE), E57, hard, 0, sg);
  }
  // tanh
  put_sg(sg, -sgnf(x));  // tanh x - x has the sign of -x
  if (ax < 0x1p-13f) return x;
  const float a2 = 2.0f * ax;
  U128 t;
  U128 err;
  int es;
  if (a2 < 0x1p-4f) {
    const U128 m = q_shr(expm1_series_q126(q_of_f(a2)), 1);
    const U128 w = q_div(m, add128(m, ONE), es);  // es = 0: m + 1 in [1, 2)
    t = q_shl(w, es);
    err = rel_err_84(t);
  } else {
    int k;
    const U128 Y = exp2q_core(expq_arg<0>(fbits(a2)), T, k);  // k in [0, 26]
    const U128 sk = q_shr(U128{0ull, 1ull << 60}, k);
    const U128 w = q_div(sub128(Y, sk), add128(Y, sk), es);
    t = q_shl(w, es);
    err = {1ull << 58, 0ull};
  }
  const float y = q_round_f(t, err, hard, 0, sg);
  if (sg && x < 0.0f) *sg = -*sg;
  return x < 0.0f ? -y : y;
}

template <int H> CRM_DEV float hyp_slow(float x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = false;
  float sp;
  if (hyp_special<H>(x, sp)) {
    if (!sg) return sp;
    bool step = false;  // the first saturation steps are evaluated, not assumed
    *sg = hyp_special_sg<H>(x, step);
    if (!step) return sp;
  }
  if (sg && (H == HYP_SINH || H == HYP_COSH) && fabsf(x) < 0x1p-25f) {
    *sg = hyp_special_sg<H>(x, hard);  // x or 1, with the sign of the remainder
    return H == HYP_SINH ? x : 1.0f;
  }
  float r;
  if (H == HYP_EXPM1 || H == HYP_TANH) {
    r = hyp_int2<H>(x, hard, sg);
  } else if (fabsf(x) >= 0x1p-25f) {
    r = hyp_int<H>(x, hard, sg);
  } else {
    // sinh, cosh of |x| < 2^-25 reach here only under the forced test hook
    r = hyp_plain<H>(x, CRM_EXP2_T16_D, hard);
    unresolved = 2;  // an FP64 tier ran
  }
  if (!hard && !force) return r;
  // the shortcuts of the first tier (expm1 x > x below 2^-25, tanh x - x of the sign of -x
  // below 2^-13) state the sign exactly
  if (sg && !hard &&
      ((H == HYP_EXPM1 && fabsf(x) < 0x1p-25f) || (H == HYP_TANH && fabsf(x) < 0x1p-13f)))
    return r;
  Pair<double> y = hyp_dd_y<H>(x);
  r = round_dd_to_f(y.hi, y.lo, HYP_DD_EPS * fabs(y.hi), hard, sg);
  unresolved = hard ? 3 : 2;  // the double-double tier ran
  return r;
}

}  // namespace crm
