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
    r = nan ? qnan_of(x) : (x == 0.0f ? x : (x > 0.0f ? CRM_INF_F : -1.0f));
    return nan || x == 0.0f || x > CRM_EXPF_X_OVF || x < CRM_EXPM1F_X_MONE;
  }
  if (H == HYP_SINH) {
    r = nan ? qnan_of(x) : (x == 0.0f ? x : copysignf(CRM_INF_F, x));
    return nan || x == 0.0f || ax > CRM_SINHF_X_OVF;
  }
  if (H == HYP_COSH) {
    r = nan ? qnan_of(x) : CRM_INF_F;
    return nan || ax > CRM_SINHF_X_OVF;
  }
  r = nan ? qnan_of(x) : (x == 0.0f ? x : copysignf(1.0f, x));
  return nan || x == 0.0f || ax > CRM_TANHF_X_ONE;
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

template <int H> CRM_DEV float hyp_slow(float x, bool &unresolved) {
  bool hard;
  float r = hyp_plain<H>(x, CRM_EXP2_T16_D, hard);
  unresolved = false;
  if (!hard) return r;
  Pair<double> y = hyp_dd_y<H>(x);
  r = round_dd_to_f(y.hi, y.lo, HYP_DD_EPS * fabs(y.hi), hard);
  unresolved = hard;
  return r;
}

}  // namespace crm
