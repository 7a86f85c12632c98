// fam_trig.cuh -- sinf, cosf, sincosf, tanf.
//
// Reduction: |x| 64/pi = 128 m + 32 q + j + f,  q = quadrant, j in [0,32), |f| <= 1/2 (the
// FP64 and slow tiers), and |x| 256/pi = 512 m + 128 q + j + f with j in [0,128) (the
// double-float tier, whose polynomials are shorter for the smaller t).
// The paper reduces large trigonometric arguments on a separate branch (Sec. II.A).  Here
// the double-float tier takes a Cody-Waite reduction in float pairs when every active
// lane of the warp has |x| < 2^12 (a warp-uniform vote), and otherwise an integer
// Payne-Hanek step on the 24-bit significand, which serves every magnitude: with
// x = M 2^e, the bits of 2/pi that can change |x| 64/pi modulo 128 form a window selected
// by e, and M times a 96-bit (fast tiers) or 160-bit (slow tier) window of 2/pi gives
// q, j and f (the same product read two bits further gives them for 256/pi).  The FP64
// and slow tiers always use the integer step.
// Then t = f pi/64 (|t| <= pi/128; double-float: f pi/256) and, with S_j = sin(j pi/64),
// C_j = cos(j pi/64),
//     sin(j pi/64 + t) = S_j cos t + C_j sin t,   cos(j pi/64 + t) = C_j cos t - S_j sin t,
// rotated by the quadrant.  Small |x| uses t = x, j = q = 0 directly.
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"
#include "fam_f64.cuh"

namespace crm {

enum { TRIG_SIN = 0, TRIG_COS = 1, TRIG_TAN = 2, TRIG_SINCOS = 3 };

// Multiply the 24-bit significand of |x| (2^-6 <= |x| < 2^128) by NW words of 2/pi
// starting at the bit that makes the product |x| 64/pi modulo 128.  r[0] is the least
// significant word of the (32 NW + 32)-bit product; the value is r 2^(7 - 32 NW).
template <int NW>
CRM_DEV void trig_window_mul(float ax, const uint32_t *P, uint32_t *r) {
  uint32_t b = fbits(ax);
  uint32_t M = (b & 0x007FFFFFu) | 0x00800000u;
  int e = (int)(b >> 23) - 150;
  int p = 64 + (e - 1) - 1;  // position of bit b_(e-1) after two zero words
  int k = p >> 5, o = p & 31;
  uint32_t w[NW];
#pragma unroll
  for (int i = 0; i < NW; i++) w[i] = __funnelshift_l(P[k + i + 1], P[k + i], o);
  uint64_t carry = 0;
#pragma unroll
  for (int i = NW - 1; i >= 0; i--) {  // w[NW-1] is the least significant word
    uint64_t pr = (uint64_t)M * w[i] + carry;
    r[NW - 1 - i] = (uint32_t)pr;
    carry = pr >> 32;
  }
  r[NW] = (uint32_t)carry;
}

// The same product for NW = 3 with the four words P[k .. k+3] from one 16-byte entry
// PW[k] of a window table (PW[k] = (P[k], P[k+1], P[k+2], P[k+3])): one shared-memory
// load per element.  k = (e + 62) >> 5 lies in [0, 5] for 2^-8 <= |x| < 2^128.
CRM_DEV void trig_window_mul3(float ax, const uint4 *PW, uint32_t *r) {
  uint32_t b = fbits(ax);
  uint32_t M = (b & 0x007FFFFFu) | 0x00800000u;
  int p = (int)(b >> 23) - 150 + 62;
  const uint4 Q = PW[p >> 5];
  const int o = p & 31;
  const uint32_t w0 = __funnelshift_l(Q.y, Q.x, o), w1 = __funnelshift_l(Q.z, Q.y, o),
                 w2 = __funnelshift_l(Q.w, Q.z, o);
  uint64_t pr = (uint64_t)M * w2;
  r[0] = (uint32_t)pr;
  pr = (uint64_t)M * w1 + (pr >> 32);
  r[1] = (uint32_t)pr;
  pr = (uint64_t)M * w0 + (pr >> 32);
  r[2] = (uint32_t)pr;
  r[3] = (uint32_t)(pr >> 32);
}

// Fast-tier reduction: N7 = (32 q + j) mod 128 and the fraction f as a signed 64-bit
// fixed-point number (f = fi 2^-64); error < 2^-64 (fraction) + 2^-66 (window).
CRM_DEV void trig_reduce64(float ax, const uint32_t *P, int &N7, int64_t &fi) {
  uint32_t r[4];
  trig_window_mul<3>(ax, P, r);
  uint64_t F = ((uint64_t)(r[2] & 0x01FFFFFFu) << 39) | ((uint64_t)r[1] << 7) | (r[0] >> 25);
  N7 = (int)(((r[2] >> 25) + (uint32_t)(F >> 63)) & 127u);
  fi = (int64_t)F;
}

// ------------------------------------------------------------------ plain (FP64) tier
// t = fi 2^-64 pi/64 in binary64: relative error 2^-52 plus the reduction's absolute
// error 2^-63.6 in f, which matters only when the result is as small as t (j = 0); lanes
// with j = 0 and |f| < 2^-14 go to the slow path, so the reduction adds at most 2^-49.6
// relative.  sin t and cos t by Taylor polynomials to degree 7 and 6
// (remainders below 2^-58), the table in binary64, one FMA per rotation term.  The
// combination may lose up to 2^5.4 (|result| >= sin(pi/128) when j != 0):
// eps = 2^-46 (D = 129); tan adds a division (D = 257).
struct TrigD {
  double A, B;  // sin and cos of (j pi/64 + t), before the quadrant rotation
  int q;
  bool tiny;    // j == 0 and |f| < 2^-14: the reduction's error is too large, go slow
};

CRM_DEV TrigD trig_plain_core(float x, const uint32_t *P, const double *SC) {
  float ax = fabsf(x);
  bool small = ax < 0x1p-6f;
  int N7;
  int64_t fi;
  trig_reduce64(small ? 1.0f : ax, P, N7, fi);
  double t = (double)fi * (CRM_PIO64_D_HI * 0x1p-64);
  t = small ? (double)ax : t;
  N7 = small ? 0 : N7;
  bool tiny = !small && (N7 & 31) == 0 && (fi > -(1ll << 50) && fi < (1ll << 50));
  int j = N7 & 31;
  double t2 = t * t;
  const double *s = CRM_SIN_TAYLOR_D, *c = CRM_COS_TAYLOR_D;
  double st = fma_(t2, fma_(t2, fma_(t2, s[3], s[2]), s[1]), s[0]) * t;
  double ct = fma_(t2, fma_(t2, fma_(t2, c[3], c[2]), c[1]), c[0]);
  double S = SC[2 * j], C = SC[2 * j + 1];
  TrigD R;
  R.A = fma_(S, ct, C * st);
  R.B = fma_(C, ct, -(S * st));
  R.q = N7 >> 5;
  R.tiny = tiny;
  return R;
}

// Rotate by the quadrant and apply the symmetry in x.  out[0]: sin or tan, out[1]: cos.
template <class Tv> CRM_DEV void trig_rotate(int kind, float x, int q, Tv A, Tv B, Tv &sn, Tv &cs) {
  Tv s0 = (q & 1) ? B : A, c0 = (q & 1) ? A : B;
  bool sneg = (q & 2) != 0, cneg = ((q + 1) & 2) != 0;
  sn = sneg ? -s0 : s0;
  cs = cneg ? -c0 : c0;
  if (x < 0.0f) sn = -sn;
}

CRM_DEV bool trig_special(float x, float &r) {
  bool nan = x != x, inf = fabsf(x) == CRM_INF_F;
  r = nan ? qnan_of(x) : CRM_QNAN_F;
  return nan || inf;
}

template <int KIND>
CRM_DEV void trig_plain(float x, const uint32_t *P, const double *SC, float *y, bool &hard) {
  float rsp;
  bool sp = trig_special(x, rsp);
  TrigD R = trig_plain_core(sp ? 1.0f : x, P, SC);
  double sn, cs;
  trig_rotate<double>(KIND, x, R.q, R.A, R.B, sn, cs);
  bool zero = x == 0.0f;  // sin/tan(+-0) = +-0
  if (KIND == TRIG_TAN) {
    double t = sn / cs;
    hard = !sp && !zero && (R.tiny || hard_d_to_f(t, 257));
    y[0] = sp ? rsp : (zero ? x : __double2float_rn(t));
    return;
  }
  bool hs = hard_d_to_f(sn, 129), hc = hard_d_to_f(cs, 129);
  if (KIND == TRIG_SIN) {
    hard = !sp && !zero && (R.tiny || hs);
    y[0] = sp ? rsp : (zero ? x : __double2float_rn(sn));
  } else if (KIND == TRIG_COS) {
    hard = !sp && (R.tiny || hc);
    y[0] = sp ? rsp : __double2float_rn(cs);
  } else {
    hard = !sp && (R.tiny || (hs && !zero) || hc);
    y[0] = sp ? rsp : (zero ? x : __double2float_rn(sn));
    y[1] = sp ? rsp : __double2float_rn(cs);
  }
}

// ------------------------------------------------------------------ double-float tier
// Finer steps than the other tiers: |x| 256/pi = 512 m + 128 q + j + f, a 128-entry table of
// (sin, cos)(j pi/256) and t = f pi/256, |t| <= pi/512 (Payne-Hanek) or (1/2 + 2^-6) pi/256
// (Cody-Waite), so that short polynomials suffice.  The same integer reduction as the
// other tiers, read two bits further; the 64-bit fraction becomes a float pair without
// conversion instructions: with F' = F + 2^63 (so f + 1/2 = F' 2^-64 >= 0), three chunks
// of 23, 23 and 18 bits become exact floats by the 2^23 magic-number trick and
// f = (c0 2^-23 - 1/2) + c1 2^-46 + c2 2^-64.  Then t = f pi/256 as a pair, and
//   cos t = 1 - t^2/2 + t^4/24 (remainder t^6/720 < 2^-53),
//   sin t = t - t^3/6 + t^5/120 (remainder t^7/5040 < 2^-56 |t|),
// with t^2 and 1 - t^2/2 carried as pairs (exact FMA splits), t^3/6 as one float from
// t_hi t^2 + 3 t_lo t^2 (it is at most 2^-17.2 |t|), the rest in float.
// Error budget (relative to the result): f to 2^-63 absolute plus 2^-48 relative (lanes
// with j = 0 and |f| < 2^-24, where the result is as small as t, go to the slow path: 2^-40
// there); pi/256 pair 2^-48; cos t 2^-48; sin t 2^-39.5 |t| (the float t^3/6, 2^-22.3 of
// itself); table pairs 2^-48; the rotation's pair products and sum 2^-47; the rotation
// terms S cos t + C sin t lose at most 2^7.4 (a result as small as sin(0.48 pi/256) from
// terms up to 1), and the sin t error enters weighted by C, so it stays 2^-39.4 of the
// result: total < 2^-38.5, inside the 2^-37 that the rounding test allows.  sin and cos
// leave the last sum unnormalised (|lo| < 2^-15 |hi|: the pair products' low words, 2^-22
// of terms at most 2^7.4 times the result) for round_df; tan normalises both before its
// division.
struct TrigF {
  Pair<float> A, B;  // sin and cos of (j pi/256 + t)
  int q;
  bool tiny;
};

// Cody-Waite reduction for |x| < 2^12 (the paper's reduction for moderate arguments,
// Sec. II.A): k = rint(|x| RN(256/pi)) by the shifter, N = k mod 512 from its bits, and
// t = |x| - k pi/256 with pi/256 = C1 + C2 + C3 (three floats, + < 2^-83):
//   t1 = |x| - k C1 is exact (one FMA: C1 is a multiple of 2^-30, |x| too when |x| >= 2^-7,
//        and |t1| < 2^-7, so t1 has at most 23 significant bits; for |x| < 2^-7, k is 0 or
//        1 and t1 is a multiple of 2^-31 below 2^-7.3),
//   k C2 = ph + pl exactly (FMA split), (sh, sl) = TwoSum(t1, -ph) exactly,
//   t = sh + RN(RN(sl - pl) - k C3), normalised by Fast2Sum.
// |x| RN(256/pi) is within |x| 2^-18.2 < 2^-6 of |x| 256/pi, so |t| <= (1/2 + 2^-6) pi/256.
// With k < 2^18.35: |k C2| < 2^-13, |pl| <= 2^-38, |k C3| < 2^-37.7, so the low word's
// two roundings and the split's remainder cost < 2^-59.5 absolute plus 2^-47 |t|.  The
// result is at least sin(0.48 pi/256) > 2^-7.4 unless j = 0, so this is < 2^-52 relative
// there; with j = 0 (k a nonzero multiple of 128, x near a multiple of pi/2) the result is
// as small as t, and lanes with |t| < 2^-19 (error above 2^-40 of t) are flagged for the
// slow path.
CRM_DEV void trig_reduce_cw(float ax, Pair<float> &t, int &N, bool &tiny) {
  const float ks = fma_(ax, CRM_256OPI_F, CRM_SHIFTER_F);
  const float k = ks - CRM_SHIFTER_F;
  N = (int)(fbits(ks) & 511u);  // 1.5 2^23 + k, k < 2^22: the low bits are k
  const float t1 = fma_(-k, CRM_PIO256_CW1, ax);
  const float ph = k * CRM_PIO256_CW2;
  const float pl = fma_(k, CRM_PIO256_CW2, -ph);
  const Pair<float> s = two_sum(t1, -ph);
  t = fast_two_sum(s.hi, fma_(-k, CRM_PIO256_CW3, s.lo - pl));
  tiny = (N & 127) == 0 && k != 0.0f && fabsf(s.hi) < 0x1p-19f;
}

// Whether a lane may take the Cody-Waite reduction: |x| < 2^12 (NaN and infinities, rare,
// send their vector to the general reduction).
CRM_DEV bool trig_cw_ok(float x) { return fabsf(x) < 0x1p12f; }

// The reduction shared by the double-float evaluators: t = f pi/256 as an unnormalised
// pair, N = (128 q + j) mod 512, and tiny (j = 0 and t too small for the reduction's
// accuracy: slow path).  PATH 1: Cody-Waite (about 20 operations; the caller has checked
// trig_cw_ok for every lane of the warp); PATH 2: the integer Payne-Hanek reduction below
// (about 50), which serves every |x|; PATH 0: Cody-Waite when every active lane of the
// warp has |x| < 2^12 (a vote per element), else Payne-Hanek.  Both reductions are correct
// for any lane that takes them, so the choice decides speed only.  The main kernels vote
// once per vector of elements and pass PATH 1 or 2 (a branch per element would keep the
// compiler from interleaving the elements of a vector).
template <int PATH = 0>
CRM_DEV void trig_reduce_df(float x, const uint4 *PW, Pair<float> &t, int &N, bool &tiny) {
  float ax = fabsf(x);
  if (PATH == 1 || (PATH == 0 && __all_sync(__activemask(), ax < 0x1p12f))) {
    trig_reduce_cw(ax, t, N, tiny);
    return;
  }
  bool small = ax < 0x1p-8f;  // |x| < pi/512: t = |x|, j = 0
  uint32_t r[4];
  trig_window_mul3(small ? 1.0f : ax, PW, r);
  // The product is |x| 64/pi mod 128 = r 2^-89, so |x| 256/pi mod 512 = r 2^-87: F = the 64
  // bits below the top 9 of r[2], F = (Fh, Fl); N = those 9 bits rounded by F's leading
  // bit, modulo 512 (the 32-bit sum wraps exactly there)
  const uint32_t Fh = __funnelshift_l(r[1], r[2], 9), Fl = __funnelshift_l(r[0], r[1], 9);
  N = (int)((r[2] + 0x00400000u) >> 23);
  uint32_t Ph = Fh ^ 0x80000000u;
  uint32_t c0 = Ph >> 9;
  uint32_t c1 = __funnelshift_r(Fl, Ph, 18) & 0x007FFFFFu;
  uint32_t c2 = Fl & 0x3FFFFu;
  float f0 = bitsf(0x4B000000u | c0) - 0x1p23f;
  float f1 = bitsf(0x4B000000u | c1) - 0x1p23f;
  float f2 = bitsf(0x4B000000u | c2) - 0x1p23f;
  // f = (c0 2^-23 - 1/2) + c1 2^-46 + c2 2^-64, three exact floats; the first two are
  // joined exactly (Fast2Sum: the first is 0 or a nonzero multiple of 2^-23, the second
  // below 2^-23), so that (fh, fl) carries f to 2^-24 |fl| + 2^-64 even when the first
  // chunk is zero or cancels (|f| small: the case that decides the rounding of results
  // near multiples of pi/2).
  Pair<float> fs = fast_two_sum(fma_(f0, 0x1p-23f, -0.5f), f1 * 0x1p-46f);
  float fh = fs.hi;
  float fl = fma_(f2, 0x1p-64f, fs.lo);
  // t = f pi/256 as an unnormalised pair (|tl| < 2^-22 |th|: dropping tl^2 from t^2
  // costs 2^-44.8 of t^2, below 2^-58 of cos t, sin t and tan t)
  t.hi = fh * CRM_PIO256_F_HI;
  t.lo = fma_(fh, CRM_PIO256_F_HI, -t.hi);
  t.lo = fma_(fh, CRM_PIO256_F_LO, t.lo);
  t.lo = fma_(fl, CRM_PIO256_F_HI, t.lo);
  tiny = !small && (N & 127) == 0 && fabsf(fh + fl) < 0x1p-24f;
  t.hi = small ? ax : t.hi;
  t.lo = small ? 0.0f : t.lo;
  N = small ? 0 : N;
}

// KIND = TRIG_SIN or TRIG_COS: only the rotation term the quadrant needs is formed, in R.A
// (sin: B when q is odd, else A; cos: A when q is odd, else B); otherwise both.
template <int KIND, int PATH = 0> CRM_DEV TrigF trig_df_core(float x, const uint4 *PW, const float4 *SC) {
  Pair<float> t;
  int N;
  TrigF R;
  trig_reduce_df<PATH>(x, PW, t, N, R.tiny);
  // t^2 as a pair
  float u = t.hi * t.hi;
  float ul = fma_(t.hi, t.hi, -u);
  ul = fma_(2.0f * t.hi, t.lo, ul);
  // cos t = 1 - t^2/2 + t^4/24
  float ch = fma_(u, -0.5f, 1.0f);
  float cl = fma_(u, -0.5f, 1.0f - ch);
  cl = fma_(ul, -0.5f, cl);
  cl = fma_(u * u, 0x1.555556p-5f, cl);
  // sin t = t - t^3/6 + t^5/120, t^3 = t_hi t^2 + 3 t_lo t^2 to 2^-23 of itself
  const float w = fma_(t.hi, u, (3.0f * t.lo) * u);
  const float s3 = w * CRM_INV6_F_HI;
  float sh = t.hi - s3;
  float sl = (t.hi - sh) - s3;  // Fast2Sum: |t| > |t^3/6|
  sl = sl + t.lo;
  sl = fma_(w * u, 0x1.111112p-7f, sl);
  // rotation by j pi/256
  int j = N & 127;
  float4 T = SC[j];  // (sin hi, lo, cos hi, lo)
  Pair<float> S = {T.x, T.y}, C = {T.z, T.w}, ct = {ch, cl}, st = {sh, sl};
  R.q = (N >> 7) & 3;
  if (KIND == TRIG_SIN || KIND == TRIG_COS) {
    // B = C cos t + (-S) sin t, A = S cos t + C sin t: one product pair with chosen factors
    const bool useB = (KIND == TRIG_SIN) == ((R.q & 1) != 0);
    const Pair<float> Pf = useB ? C : S, Qf = useB ? -S : C;
    R.A = df_add_ordered_raw(df_mul_raw(Pf, ct), df_mul_raw(Qf, st));
    R.B = R.A;
    return R;
  }
  // In both sums the first term dominates: |S_j cos t| >= sin(pi/256) cos(pi/512) > 0.0122
  // > 0.0064 > |C_j sin t| when j >= 1 (S_0 = 0 makes the sum exact), and |C_j cos t| >
  // 0.0122 > |S_j sin t| for j <= 127: Fast2Sum applies.
  Pair<float> a1 = df_mul_raw(S, ct), a2 = df_mul_raw(C, st);
  Pair<float> b1 = df_mul_raw(C, ct), b2 = df_mul_raw(S, st);
  R.A = df_add_ordered_raw(a1, a2);
  R.B = df_add_ordered_raw(b1, -b2);
  return R;
}

// tan by the addition formula on the same reduction: with T = tan(j pi/256) (a 128-entry
// float-pair table) and tau = tan t,
//   tan(j pi/256 + t) = N / D,  N = T + tau,  D = 1 - T tau,
// and tan x = +-N/D for even q, -+D/N for odd q (tan(a + pi/2) = -1/tan a).
// tau = t + t^3/3 + (2/15) t^5 with t^3/3 as one float, 2^-22.3 of itself (2^-38.5 of t),
// the t^7 term below 2^-47.9 of t.  N: T >= tan(pi/256) > 0.0122 > 0.0064 > |tau| for j >= 1 (T = 0 for j = 0), so
// Fast2Sum applies and N cancels by at most a factor 2.1; D: |T tau| <= tan(127 pi/256)
// tan((1/2 + 2^-6) pi/256) < 0.52, so D lies in [0.48, 1.52] and 1 - T tau is a Fast2Sum.
// Both are normalised for the pair division.  Error budget, relative to the result: tau
// 2^-38.5 |t| (with j = 0 the result is about t; with j >= 1 the 2^-45.8 absolute error of
// tau is 2^-38.4 of N >= 0.0059), T 2^-48, D 2^-44, the division 2^-43, the reduction as for
// sin and cos (2^-40 for j = 0 at the slow-path threshold): total < 2^-38, inside the
// rounding test's 2^-37.
CRM_DEV Pair<float> tan_df_nd(Pair<float> t, int j, const float2 *TT, Pair<float> &D) {
  // t^3 = t_hi t^2 + 3 t_lo t^2 to 2^-23 of itself, t^3/3 as one float (at most 2^-16.2 |t|)
  const float u = t.hi * t.hi;
  const float w = fma_(t.hi, u, (3.0f * t.lo) * u);
  const float s3 = w * CRM_INV3_F_HI;
  const float th = t.hi + s3;
  float tl = s3 - (th - t.hi);  // Fast2Sum: |t| > |t^3/3|
  tl = tl + t.lo;
  tl = fma_(w * u, CRM_TAN_C5_F, tl);
  const float2 T = TT[j];
  Pair<float> N = df_add_ordered({T.x, T.y}, {th, tl});
  const Pair<float> P = df_mul_raw({T.x, T.y}, {th, tl});
  D = fast_two_sum(1.0f, -P.hi);
  D.lo = D.lo - P.lo;
  D = fast_two_sum(D.hi, D.lo);
  return N;
}

// Sign of a rounded result as a bit mask: sin(j pi/256 + t) rotated by q quadrants is
// negative for q = 2, 3, cos for q = 1, 2; sin and tan are odd in x.
CRM_DEV uint32_t trig_sin_sign(int q, float x) { return (((uint32_t)q << 30) ^ fbits(x)) & 0x80000000u; }
CRM_DEV uint32_t trig_cos_sign(int q) { return ((uint32_t)(q + 1) << 30) & 0x80000000u; }

// The pairs are rounded before the quadrant rotation: round-to-nearest and round_df's
// test are symmetric under negation, so rounding A and B and then swapping and negating
// the floats gives the same bits as rotating the pairs first.
// With sg (two entries for sincosf): the sign of f(x) - y for each result, turned with the
// result's sign; the special results are exact (NaN, +-0).
template <int KIND, int PATH = 0>
CRM_DEV void trig_df(float x, const uint4 *PW, const float4 *SC, const float2 *TT, float *y, bool &hard,
                     int *sg = nullptr) {
  if (sg && fabsf(x) < 0x1p-12f) {  // sin x, tan x within x^3/3 of x, cos x within x^2/2 of 1
    hard = false;
    const int ss = KIND == TRIG_TAN ? sgnf(x) : -sgnf(x), cs = x == 0.0f ? 0 : -1;
    y[0] = KIND == TRIG_COS ? 1.0f : x;
    sg[0] = KIND == TRIG_COS ? cs : ss;
    if (KIND == TRIG_SINCOS) {
      y[1] = 1.0f;
      sg[1] = cs;
    }
    return;
  }
  const bool sp = !(fabsf(x) < CRM_INF_F);  // NaN or infinite
  if (KIND == TRIG_TAN) {
    Pair<float> t, D;
    int Nq;
    bool tiny;
    trig_reduce_df<PATH>(sp ? 1.0f : x, PW, t, Nq, tiny);
    const Pair<float> N = tan_df_nd(t, Nq & 127, TT, D);
    const bool odd = (Nq & 128) != 0;
    const Pair<float> q = df_div_raw(odd ? D : N, odd ? N : D);
    bool h;
    const float yt = round_df(q.hi, q.lo, h, sg);
    if (__builtin_expect(sp, 0)) {
      hard = false;
      put_sg(sg, 0);
      y[0] = x != x ? qnan_of(x) : CRM_QNAN_F;
      return;
    }
    // negative in odd quadrants (-cot), and odd in x
    const uint32_t sgb = (((uint32_t)Nq << 24) ^ fbits(x)) & 0x80000000u;
    const bool zero = x == 0.0f;  // tan(+-0) = +-0
    hard = !zero && (tiny || h);
    if (sg) *sg = zero ? 0 : (sgb ? -*sg : *sg);
    y[0] = zero ? x : bitsf(fbits(yt) ^ sgb);
    return;
  }
  TrigF R = trig_df_core<KIND, PATH>(sp ? 1.0f : x, PW, SC);
  if (__builtin_expect(sp, 0)) {
    hard = false;
    const float r = x != x ? qnan_of(x) : CRM_QNAN_F;
    y[0] = r;
    if (KIND == TRIG_SINCOS) y[1] = r;
    if (sg) {
      sg[0] = 0;
      if (KIND == TRIG_SINCOS) sg[1] = 0;
    }
    return;
  }
  const bool zero = x == 0.0f;  // sin/tan(+-0) = +-0
  const bool odd = (R.q & 1) != 0;
  bool ha, hb;
  int sa = 0, sb = 0;
  // sin and cos alone: R.A is already the term the quadrant needs
  const float ya = round_df(R.A.hi, R.A.lo, ha, sg ? &sa : nullptr);
  if (KIND == TRIG_SIN) {
    hard = !zero && (R.tiny || ha);
    const uint32_t s1 = trig_sin_sign(R.q, x);
    if (sg) sg[0] = zero ? 0 : (s1 ? -sa : sa);
    y[0] = zero ? x : bitsf(fbits(ya) ^ s1);
  } else if (KIND == TRIG_COS) {
    hard = R.tiny || ha;
    const uint32_t c1 = trig_cos_sign(R.q);
    if (sg) sg[0] = c1 ? -sa : sa;
    y[0] = bitsf(fbits(ya) ^ c1);
  } else {
    const float yb = round_df(R.B.hi, R.B.lo, hb, sg ? &sb : nullptr);
    hard = R.tiny || ha || hb;  // sin takes one of A, B and cos the other
    const float s0 = odd ? yb : ya, c0 = odd ? ya : yb;
    const uint32_t s1 = trig_sin_sign(R.q, x), c1 = trig_cos_sign(R.q);
    if (sg) {
      const int ss = odd ? sb : sa, cs = odd ? sa : sb;
      sg[0] = zero ? 0 : (s1 ? -ss : ss);
      sg[1] = c1 ? -cs : cs;
    }
    y[0] = zero ? x : bitsf(fbits(s0) ^ s1);
    y[1] = bitsf(fbits(c0) ^ c1);
  }
}

// ------------------------------------------------------------------ double-double tier
// 160-bit window: the fraction to 128 bits (error < 2^-127.6), t = f pi/64 in
// double-double, sin/cos t by Taylor polynomials to degree 15 / 14 (remainders < 2^-118),
// the double-double table, double-double rotation.  Relative error < 2^-96 with the same
// 2^5.4 combination bound, plus 2^-127.6/|f| from the reduction when j = 0 (below 2^-87
// for |f| >= 2^-40; a closer approach of x to a multiple of pi/64 would be reported as
// unresolved, never silently mis-rounded).
constexpr double TRIG_DD_EPS = 0x1p-84;

CRM_DEV void trig_dd_core(float x, Pair<double> &A, Pair<double> &B, int &q) {
  float ax = fabsf(x);
  Pair<double> t;
  int N7 = 0;
  if (ax < 0x1p-6f) {
    t = {(double)ax, 0.0};
  } else {
    uint32_t r[6];
    trig_window_mul<5>(ax, CRM_TWO_OVER_PI_W, r);
    uint64_t Fh = ((uint64_t)(r[4] & 0x01FFFFFFu) << 39) | ((uint64_t)r[3] << 7) | (r[2] >> 25);
    uint64_t Fl = ((uint64_t)(r[2] & 0x01FFFFFFu) << 39) | ((uint64_t)r[1] << 7) | (r[0] >> 25);
    N7 = (int)(((r[4] >> 25) + (uint32_t)(Fh >> 63)) & 127u);
    long long fh = (long long)Fh;  // two's complement: f - 1 when f >= 1/2
    long long ft = fh & ~0x7FFll;    // 53 significant bits: exact in binary64
    double h = __ll2double_rn(ft);
    long long rem = fh - ft;
    Pair<double> f = fast_two_sum(h, (double)rem + __ull2double_rn(Fl) * 0x1p-64);
    f = {f.hi * 0x1p-64, f.lo * 0x1p-64};
    t = dd_mul(f, dd(CRM_PIO64_D_HI, CRM_PIO64_D_LO));
  }
  int j = N7 & 31;
  q = N7 >> 5;
  Pair<double> t2 = dd_sqr(t);
  const double *s = CRM_SIN_TAYLOR_DD, *c = CRM_COS_TAYLOR_DD;
  Pair<double> st = dd(s[14], s[15]), ct = dd(c[14], c[15]);
  for (int k = 6; k >= 0; k--) {
    st = dd_add(dd_mul(st, t2), dd(s[2 * k], s[2 * k + 1]));
    ct = dd_add(dd_mul(ct, t2), dd(c[2 * k], c[2 * k + 1]));
  }
  st = dd_mul(st, t);
  const double *T = CRM_SINCOS_T32_DD + 4 * j;
  Pair<double> S = dd(T[0], T[1]), C = dd(T[2], T[3]);
  A = dd_add(dd_mul(S, ct), dd_mul(C, st));
  B = dd_add(dd_mul(C, ct), dd_neg(dd_mul(S, st)));
}

// ------------------------------------------------------------------ FP64-free middle tier
// sin and cos in signed Q126 fixed point (128-bit two's complement) on the integer pipes,
// for the lanes the double-float test sends to the slow path (on GB300 one warp issues an
// FP64 instruction only every few dozen cycles, see logf_int).  The 160-bit window of 2/pi
// gives f to 2^-127.6 and t = f pi/64; sin t = t + t u (s1 + ... + u^5 s6) and
// cos t - 1 = u (c1 + ... + u^6 c7), u = t^2 (remainders t^15/15! < 2^-120 and
// t^16/16! < 2^-130); then A = S + S (cos t - 1) + C sin t, B = C + C (cos t - 1) - S sin t
// with (S, C) = (sin, cos)(j pi/64) in Q126.  Every product truncates by less than a unit
// of 2^-126 and every constant is rounded to half a unit: with the sin remainder (64
// units) the error stays below 2^7 units of 2^-126, far inside half an ulp except for
// results within ~2^-119 of a midpoint (|sin|, |cos| >= 2^-35 for a binary32 x: those lanes
// continue to double-double); tan divides the two in fixed point (q_div).
template <int KIND> CRM_DEV void trig_int(float x, float *y, bool &hard, int *sg = nullptr) {
  const float ax = fabsf(x);
  hard = false;
  if (ax < 0x1p-12f) {  // RN(sin x) = x and RN(cos x) = 1: x^3/6 and x^2/2 are below half an ulp
    // sin x - x has the sign of -x, tan x - x that of x, cos x - 1 is negative (x != 0)
    const int ssx = KIND == TRIG_TAN ? sgnf(x) : -sgnf(x), scx = x == 0.0f ? 0 : -1;
    if (KIND == TRIG_COS) {
      y[0] = 1.0f;
      put_sg(sg, scx);
    } else {
      y[0] = x;
      put_sg(sg, ssx);
      if (KIND == TRIG_SINCOS) {
        y[1] = 1.0f;
        if (sg) sg[1] = scx;
      }
    }
    return;
  }
  U128 T;
  int N7 = 0;
  if (ax < 0x1p-6f) {  // t = |x|: the significand at 2^(E - 150), in Q126 M 2^(E - 24)
    const uint32_t b = fbits(ax);
    const uint64_t M = (b & 0x007FFFFFu) | 0x00800000u;
    T = {0ull, M << ((int)(b >> 23) - 88)};  // E - 24 - 64 in [27, 32]
  } else {
    uint32_t r[6];
    trig_window_mul<5>(ax, CRM_TWO_OVER_PI_W, r);
    const uint64_t Fh = ((uint64_t)(r[4] & 0x01FFFFFFu) << 39) | ((uint64_t)r[3] << 7) | (r[2] >> 25);
    const uint64_t Fl = ((uint64_t)(r[2] & 0x01FFFFFFu) << 39) | ((uint64_t)r[1] << 7) | (r[0] >> 25);
    N7 = (int)(((r[4] >> 25) + (uint32_t)(Fh >> 63)) & 127u);
    // F = f 2^128 (two's complement); F (pi/64 in Q126) 2^-126 = t 2^128, then to Q126
    const U128 t128 = q_mul({Fl, Fh}, q_ld(CRM_TRIGI_PIO64));
    T = {(t128.lo >> 2) | (t128.hi << 62), (uint64_t)((int64_t)t128.hi >> 2)};
  }
  const int j = N7 & 31, q = N7 >> 5;
  const U128 u = q_mul(T, T);
  U128 ps = q_ld(CRM_TRIGI_S + 10);
#pragma unroll
  for (int k = 4; k >= 0; k--) ps = add128(q_ld(CRM_TRIGI_S + 2 * k), q_mul(u, ps));
  const U128 st = add128(T, q_mul(T, q_mul(u, ps)));
  U128 pc = q_ld(CRM_TRIGI_C + 12);
#pragma unroll
  for (int k = 5; k >= 0; k--) pc = add128(q_ld(CRM_TRIGI_C + 2 * k), q_mul(u, pc));
  const U128 cm = q_mul(u, pc);
  const U128 S = q_ld(CRM_TRIGI_SC + 4 * j), C = q_ld(CRM_TRIGI_SC + 4 * j + 2);
  const bool odd = (q & 1) != 0;
  const U128 ERR = {128ull, 0ull};
  if (KIND == TRIG_TAN) {
    // tan = A / B, or -B / A for odd q.  With |A|, |B| >= 2^-36 (else the lane goes to
    // double-double) their 2^-119 absolute errors are below 2^-83 of them, and the
    // quotient's relative error (with q_div's 2^-118) below 2^-80: the bound is taken as
    // 2^-80 of |w| plus 2^10 units
    const U128 A = add128(add128(S, q_mul(S, cm)), q_mul(C, st));
    const U128 B = sub128(add128(C, q_mul(C, cm)), q_mul(S, st));
    const U128 N = odd ? B : A, D = odd ? A : B;
    const U128 aN = q_neg(N) ? neg128(N) : N, aD = q_neg(D) ? neg128(D) : D;
    if ((aN.hi >> 26) == 0 || (aD.hi >> 26) == 0) {  // |N| or |D| below 2^-36
      hard = true;
      y[0] = 0.0f;
      return;
    }
    int es;
    const U128 w = q_div(N, D, es);
    const U128 aw = q_neg(w) ? neg128(w) : w;
    const float yt = q_round_f(w, U128{(aw.hi >> 16) + 1024ull, 0ull}, hard, es, sg);
    const uint32_t tb = (((uint32_t)q << 31)) ^ (fbits(x) & 0x80000000u);
    if (sg && tb) *sg = -*sg;
    y[0] = bitsf(fbits(yt) ^ tb);
    return;
  }
  bool ha = false, hb = false;
  float ya = 0.0f, yb = 0.0f;
  int sa = 0, sb = 0;
  // sin of the reduced angle is A when q is even, B when odd; cos the other one
  const bool needA = KIND == TRIG_SINCOS || (KIND == TRIG_SIN) != odd;
  const bool needB = KIND == TRIG_SINCOS || (KIND == TRIG_SIN) == odd;
  if (needA) ya = q_round_f(add128(add128(S, q_mul(S, cm)), q_mul(C, st)), ERR, ha, 0, sg ? &sa : nullptr);
  if (needB) yb = q_round_f(sub128(add128(C, q_mul(C, cm)), q_mul(S, st)), ERR, hb, 0, sg ? &sb : nullptr);
  hard = ha || hb;
  const float s0 = odd ? yb : ya, c0 = odd ? ya : yb;
  const int ss = odd ? sb : sa, cs = odd ? sa : sb;
  if (KIND == TRIG_COS) {
    const uint32_t c1 = trig_cos_sign(q);
    if (sg) sg[0] = c1 ? -cs : cs;
    y[0] = bitsf(fbits(c0) ^ c1);
  } else {
    const uint32_t s1 = trig_sin_sign(q, x);
    if (sg) sg[0] = s1 ? -ss : ss;
    y[0] = bitsf(fbits(s0) ^ s1);
    if (KIND == TRIG_SINCOS) {
      const uint32_t c1 = trig_cos_sign(q);
      if (sg) sg[1] = c1 ? -cs : cs;
      y[1] = bitsf(fbits(c0) ^ c1);
    }
  }
}

// Slow path: the FP64-free tier, then double-double.
template <int KIND> CRM_DEV void trig_slow(float x, float *y, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = false;
  float sp;
  if (trig_special(x, sp)) {
    y[0] = sp;
    if (KIND == TRIG_SINCOS) y[1] = sp;
    if (sg) {
      sg[0] = 0;
      if (KIND == TRIG_SINCOS) sg[1] = 0;
    }
    return;
  }
  trig_int<KIND>(x, y, hard, sg);
  if ((!hard && !force) || trig_special(x, sp)) return;
  if (sg && fabsf(x) < 0x1p-12f) return;  // the tiny range's results and signs are exact statements
  Pair<double> A, B, sn, cs;
  int q;
  trig_dd_core(x, A, B, q);
  trig_rotate<Pair<double>>(KIND, x, q, A, B, sn, cs);
  bool h0 = false, h1 = false;
  int s0 = 0, s1 = 0;
  int *p0 = sg ? &s0 : nullptr, *p1 = sg ? &s1 : nullptr;
  if (KIND == TRIG_TAN) {
    Pair<double> t = dd_div(sn, cs);
    y[0] = round_dd_to_f(t.hi, t.lo, TRIG_DD_EPS * fabs(t.hi), h0, p0);
  } else {
    if (KIND != TRIG_COS) y[0] = round_dd_to_f(sn.hi, sn.lo, TRIG_DD_EPS * fabs(sn.hi), h0, p0);
    float c = round_dd_to_f(cs.hi, cs.lo, TRIG_DD_EPS * fabs(cs.hi), h1, p1);
    if (KIND == TRIG_COS) {
      y[0] = c;
      s0 = s1;
    }
    if (KIND == TRIG_SINCOS) y[1] = c;
  }
  if (sg) {
    sg[0] = s0;
    if (KIND == TRIG_SINCOS) sg[1] = s1;
  }
  if (x == 0.0f && KIND != TRIG_COS) y[0] = x;
  unresolved = (h0 || h1) ? 3 : 2;  // the double-double tier ran
}

}  // namespace crm
