// fam_f64.cuh -- the binary64 pair of Sec. II.B: exp2 and log.
//
// Main path (double-double in FP64), following the paper's design: a highly accurate but
// not always correctly rounded evaluation plus a rounding test; lanes that fail it are
// sent to a slower exact path (Sec. II.B).
//   exp2: x = k + (256 i1 + 16 i2 + i3)/4096 + R, |R| <= 2^-13, and
//         2^x = 2^k T1[i1] T2[i2] T3[i3] 2^R with three 16-entry double-double tables
//         (the paper's 0.75 KB of tables) and a degree-7 polynomial for 2^R - 1;
//   log:  x = 2^e m (m in [3/4, 3/2)), a short reciprocal rcp_j ~ 1/m from a 193-entry
//         table, r = m rcp_j - 1 exactly as a double-double (TwoProd), and
//         log x = e ln2 + (-log rcp_j) + log1p(r) with log1p by an odd/even-split
//         polynomial of degree 11.
// Slow path: 192-bit unsigned fixed-point integer arithmetic (no FP64 at all), with the
// rounding decided exactly from the computed interval; it cannot be wrong, only
// unresolved (never observed: that would need a result within 2^-180 of a midpoint).
#pragma once
#include "crm_common.cuh"
#include "crm_tables.h"

namespace crm {

// ------------------------------------------------------------------ rounding test (binary64)
// y = s + t (|t| <= ulp(s)/2) approximates v with |v - y| <= eps |s|; RN64(v) = s unless
// a midpoint next to s lies within |t| + eps |s|, which the hardware's rounding measures:
// with u = t + copysign(E |s|, t), the lane is hard iff RN(s + u) != s (the quarter-ulp
// gap below a power of two included).  E = 2^-98 covers eps <= 2^-100 plus the rounding
// of the sum.
CRM_DEV bool hard_dd(double s, double t) {
  double e = fabs(s) * 0x1p-98;
  double u = t + copysign(e, t);
  return (s + u) != s;
}

// ------------------------------------------------------------------ exp2, main path
// Error: tables 2^-106 each, two double-double products 2^-104 each, the polynomial
// (c1..c3 in double-double, c4..c7 in double: |R|^4 c4 <= 2^-58.3 so the double tail adds
// 2^-111) 2^-104, the final product and sum 2^-104: below 2^-101.5 relative.
constexpr double EXP2D_EPS_OK = 0x1p-100;

CRM_DEV bool exp2d_special(double x, double &r) {
  bool nan = x != x;
  r = nan ? qnan_of(x) : (x >= 1024.0 ? CRM_INF_D : 0.0);
  return nan || x >= 1024.0 || x <= -1075.0;
}

CRM_DEV Pair<double> exp2d_core(double x, int &k, const double *T) {
  const double sh = 0x1.8p52;
  double xs = x * 4096.0;  // exact
  double nd = (xs + sh) - sh;  // rint(4096 x)
  long long N = (long long)nd;
  double R = fma_(nd, -0x1p-12, x);  // exact (Sterbenz)
  int i = (int)(N & 4095);
  k = (int)(N >> 12);
  const double *T1 = T, *T2 = T + 32, *T3 = T + 64;  // the three tables, contiguous
  int i1 = i >> 8, i2 = (i >> 4) & 15, i3 = i & 15;
  Pair<double> t = dd_mul(dd(T1[2 * i1], T1[2 * i1 + 1]), dd(T2[2 * i2], T2[2 * i2 + 1]));
  t = dd_mul(t, dd(T3[2 * i3], T3[2 * i3 + 1]));
  const double *c = CRM_EXP2D_C;  // (ln2)^k/k!, k = 1..8, pairs
  double tail = fma_(R, fma_(R, fma_(R, c[12], c[10]), c[8]), c[6]) * R;  // R (c4 + R c5 + ...)
  Pair<double> q = dd_add_d(dd(c[4], c[5]), tail);
  q = dd_add(dd(c[2], c[3]), dd_mul_d(q, R));
  q = dd_add(dd(c[0], c[1]), dd_mul_d(q, R));
  Pair<double> p = dd_mul_d(q, R);  // 2^R - 1
  return dd_add(t, dd_mul(t, p));
}

CRM_DEV double exp2d_main(double x, const double *T, bool &hard, int *sg = nullptr) {
  double r;
  bool sp = exp2d_special(x, r);
  int k;
  Pair<double> y = exp2d_core(sp ? 0.0 : x, k, T);
  // Subnormal results (x < -1022): the result is the integer nearest to
  // u = y 2^(k + 1074) (u < 2^53, the scaling exact) times 2^-1074.  With q = rint(u_hi)
  // and d = (u_hi - q) + u_lo in [-1, 1], the nearest integer is q, q + 1 (d > 1/2) or
  // q - 1 (d < -1/2); y's error (2^-100 relative, below 2^-47 in u) can move u across a
  // half-integer only when ||d| - 1/2| <= 2^-46: those lanes take the exact path.
  const bool sub = x < -1022.0;
  const double sc = pow2d(sub ? k + 1074 : 0);
  const double uh = y.hi * sc, ul = y.lo * sc;
  const double q = rint(uh);
  const double d = (uh - q) + ul;
  const double qi = q + (d > 0.5 ? 1.0 : (d < -0.5 ? -1.0 : 0.0));
  const bool hsub = fabs(fabs(d) - 0.5) <= 0x1p-46;
  hard = !sp && (sub ? hsub : hard_dd(y.hi, y.lo));
  if (sg) {  // the sign of 2^x - result, from the low word (or u - qi); 0 for exact specials
    const double dq = d - (qi - q);
    const bool inf = fabs(x) == CRM_INF_D;
    *sg = sp ? ((x != x || inf) ? 0 : (x > 0.0 ? -1 : 1)) : (sub ? (dq > 0.0 ? 1 : -1) : (y.lo > 0.0 ? 1 : -1));
    hard = !sp && (sub ? !(fabs(dq) > 0x1p-46) : !(fabs(y.lo) > fabs(y.hi) * 0x1p-98));
  }
  double out = sub ? qi * 0x1p-1074 : scale_d(y.hi, k);
  return sp ? r : out;
}

// ------------------------------------------------------------------ exp2, FP64-free main path
// 128-bit fixed point on the integer pipes (GB300's FP64 rate is a small fraction of its
// integer rate).  |x| 2^96 is formed exactly from x's significand (truncated below 2^-96
// for |x| < 2^-16), negated for x < 0, so that k = floor(x') and the 96 fraction bits give
// f = x' - k in [0, 1).  f = i/1024 + r, r < 2^-10; T = 2^(i/1024) from a 1024-entry
// table (Q124, 16 KB of shared memory); 2^r - 1 = 2^-10 P with
// P = rho (a1 + rho 2^-10 (a2 + ...)), rho = r 2^10, a_n = (ln 2)^n/n!, n <= 6, by
// Horner with truncating products: Q64 for a1..a4, Q32 for a5, a6 (their weight is
// 2^-40 or less).  Error in 2^f: P to 2^-62.2 (2^r - 1 to 2^-72.2), r's truncation to 64
// bits 2^-74.5, the omitted degree-7 term 2^-86: |Y - 2^f| < 2^-70.9, i.e. below 2^54
// units of Y (Q124).  The rounding (normal results at bit 72 of Y, subnormal ones further
// up) is decided unless the discarded part is within 2^54 units of half an ulp: those
// lanes take the slow path.
struct U128 {
  uint64_t lo, hi;
};
CRM_DEV U128 mul64w(uint64_t a, uint64_t b) { return {a * b, __umul64hi(a, b)}; }
CRM_DEV U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
CRM_DEV U128 add128_64(U128 a, uint64_t b) {
  U128 r;
  r.lo = a.lo + b;
  r.hi = a.hi + (r.lo < b ? 1ull : 0ull);
  return r;
}
CRM_DEV bool le128(U128 a, U128 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
CRM_DEV U128 shr128(U128 a, int s) {  // 0 < s < 64
  return {(a.lo >> s) | (a.hi << (64 - s)), a.hi >> s};
}

// exp2d_special on the bit pattern (integer compares: the FP64 pipe stays idle)
CRM_DEV bool exp2d_special_bits(uint64_t b, double &r) {
  const uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
  const bool neg = (b >> 63) != 0;
  const bool nan = ab > 0x7FF0000000000000ull;
  const bool ovf = !neg && ab >= 0x4090000000000000ull;  // x >= 1024 (and +inf)
  const bool unf = neg && ab >= 0x4090CC0000000000ull;   // x <= -1075 (and -inf)
  r = nan ? bitsd(b | 0x0008000000000000ull) : (ovf ? CRM_INF_D : 0.0);
  return nan || ovf || unf;
}

// 2^x' for the fixed-point argument X = x' 2^96 (two's complement, |x'| < 2^31): k =
// floor(x') and Y = 2^(x' - k) in Q124 (Y in [2^124, 2^125)), error < 2^54 units.
CRM_DEV U128 exp2q_core(U128 X, const ulonglong2 *T, int &k) {
  k = (int)((int64_t)X.hi >> 32);
  const uint32_t Fh = (uint32_t)X.hi;
  const int i = (int)(Fh >> 22);
  const uint64_t rho = ((uint64_t)(Fh & 0x3FFFFFu) << 42) | (X.lo >> 22);
  // P = rho (a1 + rho 2^-10 (a2 + ...)): a6, a5 in Q32, the rest in Q64
  const uint32_t rho32 = (uint32_t)(rho >> 32);
  uint32_t h32 = CRM_EXP2I_A6_32;
  h32 = CRM_EXP2I_A5_32 + (__umulhi(rho32, h32) >> 10);
  const uint64_t rh5 = (uint64_t)rho32 * h32 + (((uint64_t)(uint32_t)rho * h32) >> 32);  // rho h5 2^-32
  uint64_t h = CRM_EXP2I_A4 + (rh5 >> 10);
  h = CRM_EXP2I_A3 + (__umul64hi(rho, h) >> 10);
  h = CRM_EXP2I_A2 + (__umul64hi(rho, h) >> 10);
  h = CRM_EXP2I_A1 + (__umul64hi(rho, h) >> 10);
  const uint64_t P = __umul64hi(rho, h);
  // Y = T + T 2^-10 P 2^-64 (Q124)
  const ulonglong2 t = T[i];  // (low, high)
  U128 tp = shr128(mul64w(t.y, P), 10);
  tp = add128_64(tp, __umul64hi(t.x, P) >> 10);
  return add128({t.x, t.y}, tp);  // in [2^124, 2^125)
}

CRM_DEV double exp2d_int(double x, const ulonglong2 *T, bool &hard, int *sg = nullptr) {
  double rs;
  const uint64_t b = dbits(x);
  const bool sp = exp2d_special_bits(b, rs);
  const int E = (int)((b >> 52) & 0x7FF);
  const bool tiny = E < 1023 - 60;  // |x| < 2^-60: 2^x rounds to 1
  const uint64_t M = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  int s = E - 979;  // |x| 2^96 = M 2^s, s in [-16, 54] on the main path
  s = (sp || tiny) ? 0 : s;
  U128 X;
  X.lo = s >= 0 ? (M << s) : (M >> -s);
  X.hi = s > 0 ? (M >> (64 - s)) : 0ull;
  if (b >> 63) {  // two's complement: k = floor(x'), the fraction bits give x' - k
    X.lo = ~X.lo + 1ull;
    X.hi = ~X.hi + (X.lo == 0 ? 1ull : 0ull);
  }
  int k;
  const U128 Y = exp2q_core(X, T, k);
  const uint64_t ERR = 1ull << 54;
  uint64_t bits;
  bool near;
  bool up, ndir;  // ndir: the discarded part is within ERR of 0 or of a full unit
  if (__builtin_expect(k >= -1022, 1)) {  // normal result: round at bit 72
    const uint64_t dh = (Y.hi & 0xFFull) - 0x80ull;  // high word of (discarded part - half ulp)
    up = (int64_t)dh > 0 || (dh == 0 && Y.lo != 0);
    near = (dh == 0 && Y.lo <= ERR) || (dh == ~0ull && Y.lo >= 0ull - ERR);
    bits = ((uint64_t)(int64_t)(k + 1022) << 52) + (Y.hi >> 8) + (up ? 1ull : 0ull);
    const uint64_t rh = Y.hi & 0xFFull;
    ndir = (rh == 0 && Y.lo <= ERR) || (rh == 0xFFull && Y.lo >= 0ull - ERR);
  } else {  // subnormal result: round at bit 72 + (-1022 - k) <= 125
    const int sh64 = 8 + (-1022 - k);
    const uint64_t remh = Y.hi & ((1ull << sh64) - 1ull);
    const uint64_t dh = remh - (1ull << (sh64 - 1));
    up = (int64_t)dh > 0 || (dh == 0 && Y.lo != 0);
    near = (dh == 0 && Y.lo <= ERR) || (dh == ~0ull && Y.lo >= 0ull - ERR);
    bits = (Y.hi >> sh64) + (up ? 1ull : 0ull);
    ndir = (remh == 0 && Y.lo <= ERR) || (remh == (1ull << sh64) - 1ull && Y.lo >= 0ull - ERR);
  }
  hard = !sp && !tiny && near;
  if (sg) {  // the sign of 2^x - result
    const uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
    *sg = sp ? ((ab >= 0x7FF0000000000000ull) ? 0 : ((b >> 63) ? 1 : -1)) : (tiny ? (ab == 0 ? 0 : ((b >> 63) ? -1 : 1)) : (up ? -1 : 1));
    hard = !sp && !tiny && ndir;
  }
  return sp ? rs : (tiny ? 1.0 : bitsd(bits));
}

// ------------------------------------------------------------------ log, main path
// r = m rcp - 1 exactly (TwoProd; m rcp - 1 is Sterbenz-exact in its leading word),
// |r| <= 2^-8.6; log1p(r) = sum (-1)^(k+1) r^k / k to degree 11 (remainder r^12/12 <=
// 2^-106.8), c1..c5 in double-double Horner, the r^6.. tail in double (2^-113).
// e ln2 with a double-double ln2; -log(rcp) from the table.  Error < 2^-102 relative
// (|log x| >= 2^-9.6 unless e = 0 and rcp = 1, where all terms scale with r).
CRM_DEV bool logd_special(double x, double &r) {
  bool nan = x != x;
  r = nan ? qnan_of(x) : (x == 0.0 ? -CRM_INF_D : (x < 0.0 ? CRM_QNAN_D : CRM_INF_D));
  return nan || x <= 0.0 || x == CRM_INF_D;
}

CRM_DEV Pair<double> logd_core(double x) {
  bool sub = x < 0x1p-1022;
  double xs = sub ? x * 0x1p54 : x;
  uint64_t b = dbits(xs);
  uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
  bool big = mant >= (1ull << 51);
  int e = (int)(b >> 52) - 1023 + (big ? 1 : 0) - (sub ? 54 : 0);
  double m = bitsd(mant | (big ? 0x3FE0000000000000ull : 0x3FF0000000000000ull));
  // j = round(256 m) in [192, 384]
  int j = big ? 128 + (int)((mant + (1ull << 44)) >> 45) : 256 + (int)((mant + (1ull << 43)) >> 44);
  double rc = CRM_LOGD_RCP[j - 192];
  Pair<double> p = two_prod(m, rc);
  Pair<double> r = fast_two_sum(p.hi - 1.0, p.lo);
  const double *c = CRM_LOGD_C;  // (-1)^(k+1)/k, k = 1..12, pairs
  double rh = r.hi;
  double tail = c[20];
  for (int q = 9; q >= 5; q--) tail = fma_(rh, tail, c[2 * q]);  // c6..c11 (index k-1)
  tail = tail * rh;                                                // r (c6 + r c7 + ...)
  Pair<double> s = dd_add_d(dd(c[8], c[9]), tail);                 // c5 + ...
  for (int q = 3; q >= 0; q--) s = dd_add(dd(c[2 * q], c[2 * q + 1]), dd_mul(s, r));
  Pair<double> l1p = dd_mul(s, r);
  Pair<double> L = dd(CRM_LOGD_L[2 * (j - 192)], CRM_LOGD_L[2 * (j - 192) + 1]);
  Pair<double> eK = dd_mul_d(dd(CRM_LN2_DD_HI, CRM_LN2_DD_LO), (double)e);
  return dd_add(dd_add(eK, L), l1p);
}

CRM_DEV double logd_main(double x, bool &hard, int *sg = nullptr) {
  double r;
  bool sp = logd_special(x, r);
  Pair<double> y = logd_core(sp ? 2.0 : x);
  hard = !sp && hard_dd(y.hi, y.lo);
  if (sg) {  // the sign of log x - result from the low word; specials are exact
    *sg = sp ? 0 : (y.lo > 0.0 ? 1 : -1);
    hard = !sp && !(fabs(y.lo) > fabs(y.hi) * 0x1p-98);
  }
  return sp ? r : y.hi;
}

// ------------------------------------------------------------------ log, FP64-free main path
// 128-bit fixed point on the integer pipes.  x = 2^e m, m in [3/4, 3/2) (subnormal x
// normalised by its leading zeros), j = round(256 m), R_j = round(2^17/j) (10 bits) and
// r = m R_j 2^-9 - 1, exact as a 64-bit integer (m has 53 bits, R_j 10), |r| < 2^-8.
//   log x = e ln 2 + L_j + log1p(r),  L_j = -log(R_j 2^-9)  (table, Q116),
//   log1p(r) = r (1 + S'),  S' = -r/2 + r^2 U(r),  U = 1/3 - r/4 + r^2/5 - ... (n <= 7),
// U by Horner with signed truncating products, Q63 for the first four coefficients and Q31
// for the rest (error 2^-61, the omitted term 2^-67.5), r^2 U and r/2 in Q127, so that
// log1p(r) is good to 2^-77 of itself however small r is.  Z = log x in Q116; errors in units of 2^-116: e ln2 |e|/2, L_j 1/2,
// products and shifts 4, log1p |r| 2^38: the bound used is 16 + |e| + |r| 2^40.  The
// rounding to binary64 is decided unless the discarded part of |Z| is within that bound
// of half an ulp: those lanes take the slow path.
CRM_DEV U128 neg128(U128 a) {
  U128 r;
  r.lo = ~a.lo + 1ull;
  r.hi = ~a.hi + (r.lo == 0 ? 1ull : 0ull);
  return r;
}
CRM_DEV U128 sub128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}

// logd_special on the bit pattern (integer compares)
CRM_DEV bool logd_special_bits(uint64_t b, double &r) {
  const uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
  const bool nan = ab > 0x7FF0000000000000ull;
  const bool zero = ab == 0;
  const bool neg = (b >> 63) != 0;
  const bool inf = b == 0x7FF0000000000000ull;
  r = nan ? bitsd(b | 0x0008000000000000ull) : (zero ? -CRM_INF_D : (neg ? CRM_QNAN_D : CRM_INF_D));
  return nan || zero || neg || inf;
}

// Z = log x in Q116 (two's complement) for the bit pattern b of a positive finite double
// (normal or subnormal), with its error bound in units of 2^-116 in err.
CRM_DEV U128 logz_q116(uint64_t b, const ulonglong2 *LT, const unsigned short *RT, uint64_t &err) {
  int E = (int)(b >> 52);
  uint64_t M = b & 0x000FFFFFFFFFFFFFull;
  if (E == 0) {  // subnormal: shift the leading bit to position 52
    const int lz = __clzll(M) - 11;
    M <<= lz;
    E = 1 - lz;
  } else {
    M |= 1ull << 52;
  }
  const bool big = M >= (3ull << 51);  // m >= 3/2: use m/2
  const int e = E - 1023 + (big ? 1 : 0);
  const uint64_t Mq = big ? M : (M << 1);              // m 2^53
  const int j = (int)((Mq + (1ull << 44)) >> 45);      // 192 .. 384
  const uint64_t R = RT[j - 192];
  const int64_t r64 = (int64_t)(Mq * R - (1ull << 62)) * 4;  // r 2^64, exact
  const uint64_t ar = r64 < 0 ? 0ull - (uint64_t)r64 : (uint64_t)r64;
  // U(r) in Q63; its tail C4 + r (C5 + r (C6 + r C7)) enters with weight r^4 <= 2^-32 and
  // is formed in Q31 (error 2^-29.4, i.e. 2^-61.4 in U)
  const int32_t r32 = (int32_t)(r64 >> 32);
  int32_t v = CRM_LOGI_C7_32;
  v = CRM_LOGI_C6_32 + __mulhi(r32, v);
  v = CRM_LOGI_C5_32 + __mulhi(r32, v);
  v = CRM_LOGI_C4_32 + __mulhi(r32, v);
  int64_t u = CRM_LOGI_C3 + __mul64hi(r64, (int64_t)v << 32);
  u = CRM_LOGI_C2 + __mul64hi(r64, u);
  u = CRM_LOGI_C1 + __mul64hi(r64, u);
  u = CRM_LOGI_C0 + __mul64hi(r64, u);
  // S' = r^2 U - r/2 in Q127
  const U128 r2 = mul64w(ar, ar);  // Q128
  const U128 r2u = add128_64(mul64w(r2.hi, (uint64_t)u), __umul64hi(r2.lo, (uint64_t)u));
  const U128 rhalf = {(uint64_t)r64 << 62, (uint64_t)(r64 >> 2)};  // r/2 in Q127
  const U128 Sp = sub128(r2u, rhalf);
  const bool sneg = (int64_t)Sp.hi < 0;
  const U128 aS = sneg ? neg128(Sp) : Sp;
  // r S' in Q116, with the sign of r S'
  U128 rS = shr128(add128_64(mul64w(ar, aS.hi), __umul64hi(ar, aS.lo)), 11);
  if ((r64 < 0) != sneg) rS = neg128(rS);
  const U128 rQ = {(uint64_t)r64 << 52, (uint64_t)(r64 >> 12)};  // r in Q116
  // e ln 2 in Q116
  const uint64_t ae = (uint64_t)(e < 0 ? -e : e);
  const U128 p0 = mul64w(CRM_LOGI_LN2_LO, ae);
  U128 eL = {p0.lo, CRM_LOGI_LN2_HI * ae + p0.hi};
  if (e < 0) eL = neg128(eL);
  const ulonglong2 Lj = LT[j - 192];
  err = 16ull + ae + (ar >> 24);
  return add128(add128(eL, {Lj.x, Lj.y}), add128(rQ, rS));
}

CRM_DEV double logd_int(double x, const ulonglong2 *LT, const unsigned short *RT, bool &hard, int *sg = nullptr) {
  double rs;
  const bool sp = logd_special_bits(dbits(x), rs);
  const uint64_t b = sp ? 0x4000000000000000ull : dbits(x);  // 2.0 on the special lanes
  uint64_t err;
  const U128 Z = logz_q116(b, LT, RT, err);
  // round |Z| (Q116) to 53 bits
  const bool zneg = (int64_t)Z.hi < 0;
  const U128 A = zneg ? neg128(Z) : Z;
  const bool zero = (A.hi | A.lo) == 0;  // x == 1
  const int lz = A.hi ? __clzll(A.hi) : 64 + __clzll(A.lo | 1ull);
  const int sh = 75 - lz;  // (127 - lz) - 52, 11 .. 74 for x != 1
  uint64_t mant;
  U128 rem, half;
  if (sh < 64) {
    mant = (A.lo >> sh) | (A.hi << (64 - sh));
    rem = {A.lo & ((1ull << sh) - 1ull), 0ull};
    half = {1ull << (sh - 1), 0ull};
  } else {
    mant = A.hi >> (sh - 64);
    rem = {A.lo, A.hi & ((1ull << (sh - 64)) - 1ull)};
    half = sh == 64 ? U128{1ull << 63, 0ull} : U128{0ull, 1ull << (sh - 65)};
  }
  const U128 dlt = sub128(rem, half);
  const bool near = (dlt.hi == 0 && dlt.lo <= err) || (dlt.hi == ~0ull && dlt.lo >= 0ull - err);
  const bool up = (int64_t)dlt.hi > 0 || (dlt.hi == 0 && dlt.lo != 0);
  const uint64_t bits = ((uint64_t)(sh + 958) << 52) + mant + (up ? 1ull : 0ull);
  hard = !sp && !zero && near;
  if (sg) {  // the sign of log x - result: decided unless rem is within err of 0 or a unit
    const U128 E = {err, 0ull};
    const U128 unit = add128(half, half);
    hard = !sp && !zero && (le128(rem, E) || le128(sub128(unit, rem), E));
    *sg = (sp || zero) ? 0 : ((up != zneg) ? -1 : 1);
  }
  return sp ? rs : (zero ? 0.0 : bitsd(bits | (zneg ? 0x8000000000000000ull : 0ull)));
}

// ------------------------------------------------------------------ e^x, 10^x, FP64-free
// b^x = 2^(x log2 b) on the same fixed-point exp2 core: |x| log2(b) 2^96 is formed from x's
// 53-bit significand times log2 e (Q125) or log2 10 (Q124), truncated (the constant's and
// the product's truncations stay below 2 units of 2^-96, i.e. 2^29 units of Y: the rounding
// bound is taken as 2^55 units); then the rounding of exp2d_int.  KIND 0: e^x, 2: 10^x.
template <int KIND> CRM_DEV U128 expbd_arg(uint64_t ab) {  // 2^-60 <= |x| < 2^10
  const int E = (int)(ab >> 52);
  const uint64_t M = (ab & 0x000FFFFFFFFFFFFFull) | (1ull << 52);  // |x| = M 2^(E - 1075)
  const uint64_t ch = KIND == 0 ? CRM_EXPI_LOG2E_Q125_HI : CRM_EXPI_LOG2_10_Q124_HI;
  const uint64_t cl = KIND == 0 ? CRM_EXPI_LOG2E_Q125_LO : CRM_EXPI_LOG2_10_Q124_LO;
  const int F = KIND == 0 ? 125 : 124;
  const U128 ml = mul64w(M, cl), mh = mul64w(M, ch);  // M C as 192 bits p2:p1:p0
  const uint64_t p0 = ml.lo, p1 = ml.hi + mh.lo;
  const uint64_t p2 = mh.hi + (p1 < ml.hi ? 1ull : 0ull);
  const int sft = F - 96 - (E - 1075);  // X = M C >> sft, sft in [60, 141]
  U128 X;
  if (sft < 64) {
    X.lo = (p0 >> sft) | (p1 << (64 - sft));
    X.hi = (p1 >> sft) | (p2 << (64 - sft));
  } else if (sft < 128) {
    const int s2 = sft - 64;
    X.lo = s2 ? ((p1 >> s2) | (p2 << (64 - s2))) : p1;
    X.hi = p2 >> s2;
  } else {
    X.lo = p2 >> (sft - 128);
    X.hi = 0ull;
  }
  return X;
}

template <int KIND>
CRM_DEV double expbd_int(double x, const ulonglong2 *T, bool &hard, int *sg = nullptr) {
  const uint64_t b = dbits(x), ab = b & 0x7FFFFFFFFFFFFFFFull;
  const bool neg = (b >> 63) != 0;
  hard = false;
  if (ab >= 0x4090000000000000ull) {  // NaN, +-inf, |x| >= 1024: b^x overflows or underflows
    put_sg(sg, ab >= 0x7FF0000000000000ull ? 0 : (neg ? 1 : -1));
    return ab > 0x7FF0000000000000ull ? bitsd(b | 0x0008000000000000ull) : (neg ? 0.0 : CRM_INF_D);
  }
  if ((int)(ab >> 52) < 1023 - 60) {  // |x| < 2^-60: b^x - 1 is below 2^-57, rounds to 1
    put_sg(sg, ab == 0 ? 0 : (neg ? -1 : 1));
    return 1.0;
  }
  U128 X = expbd_arg<KIND>(ab);
  if (neg) X = neg128(X);
  int k;
  const U128 Y = exp2q_core(X, T, k);
  if (k >= 1024) {
    put_sg(sg, -1);
    return CRM_INF_D;
  }
  if (k < -1075) {
    put_sg(sg, 1);
    return 0.0;
  }
  const uint64_t ERR = 1ull << 55;
  uint64_t bits;
  bool up, near, ndir;
  if (k >= -1022) {  // normal result: round at bit 72
    const uint64_t dh = (Y.hi & 0xFFull) - 0x80ull;
    up = (int64_t)dh > 0 || (dh == 0 && Y.lo != 0);
    near = (dh == 0 && Y.lo <= ERR) || (dh == ~0ull && Y.lo >= 0ull - ERR);
    bits = ((uint64_t)(int64_t)(k + 1022) << 52) + (Y.hi >> 8) + (up ? 1ull : 0ull);
    const uint64_t rh = Y.hi & 0xFFull;
    ndir = (rh == 0 && Y.lo <= ERR) || (rh == 0xFFull && Y.lo >= 0ull - ERR);
  } else {  // subnormal result: round at bit 72 + (-1022 - k) <= 125
    const int sh64 = 8 + (-1022 - k);
    const uint64_t remh = Y.hi & ((1ull << sh64) - 1ull);
    const uint64_t dh = remh - (1ull << (sh64 - 1));
    up = (int64_t)dh > 0 || (dh == 0 && Y.lo != 0);
    near = (dh == 0 && Y.lo <= ERR) || (dh == ~0ull && Y.lo >= 0ull - ERR);
    bits = (Y.hi >> sh64) + (up ? 1ull : 0ull);
    ndir = (remh == 0 && Y.lo <= ERR) || (remh == (1ull << sh64) - 1ull && Y.lo >= 0ull - ERR);
  }
  hard = near;
  if (sg) {
    hard = ndir;
    *sg = up ? -1 : 1;
  }
  return bitsd(bits);
}

// ------------------------------------------------------------------ log2, log10, FP64-free
// The log core (Z = ln x in Q116, error err units) times 1/ln 2 or 1/ln 10 in Q126 (the
// product truncated: W = Z C 2^-126, error err C + 2 units, taken as err + err/2 + 3), then
// |W| rounded to 53 bits with the rounding test of logd_int.  KIND 1: log2, 2: log10.
CRM_DEV U128 mul_q126_const(U128 A, uint64_t ch, uint64_t cl) {  // A C 2^-126 for A, C >= 0
  const U128 hh = mul64w(A.hi, ch), hl = mul64w(A.hi, cl), lh = mul64w(A.lo, ch);
  const uint64_t ll_hi = __umul64hi(A.lo, cl);
  U128 mid = add128(hl, lh);
  const uint64_t c1 = (mid.hi < hl.hi || (mid.hi == hl.hi && mid.lo < hl.lo)) ? 1ull : 0ull;
  mid = add128_64(mid, ll_hi);
  const uint64_t c2 = (mid.hi == 0 && mid.lo < ll_hi) ? 1ull : 0ull;
  const uint64_t w2 = hh.lo + mid.hi;
  const uint64_t w3 = hh.hi + c1 + c2 + (w2 < hh.lo ? 1ull : 0ull);
  const uint64_t w1 = mid.lo;
  return {(w2 << 2) | (w1 >> 62), (w3 << 2) | (w2 >> 62)};
}

template <int KIND>
CRM_DEV double logbd_int(double x, const ulonglong2 *LT, const unsigned short *RT, bool &hard, int *sg = nullptr) {
  double rs;
  const bool sp = logd_special_bits(dbits(x), rs);
  const uint64_t b = sp ? 0x4000000000000000ull : dbits(x);
  uint64_t err;
  const U128 Z = logz_q116(b, LT, RT, err);
  const bool zneg = (int64_t)Z.hi < 0;
  const U128 A = mul_q126_const(zneg ? neg128(Z) : Z, KIND == 1 ? CRM_LOGI_INV_LN2_Q126_HI : CRM_LOGI_INV_LN10_Q126_HI,
                                KIND == 1 ? CRM_LOGI_INV_LN2_Q126_LO : CRM_LOGI_INV_LN10_Q126_LO);
  err = err + (err >> 1) + 3ull;
  const bool zero = (A.hi | A.lo) == 0;  // x == 1
  const int lz = A.hi ? __clzll(A.hi) : 64 + __clzll(A.lo | 1ull);
  const int sh = 75 - lz;  // (127 - lz) - 52
  uint64_t mant;
  U128 rem, half;
  if (sh < 64) {
    mant = (A.lo >> sh) | (A.hi << (64 - sh));
    rem = {A.lo & ((1ull << sh) - 1ull), 0ull};
    half = {1ull << (sh - 1), 0ull};
  } else {
    mant = A.hi >> (sh - 64);
    rem = {A.lo, A.hi & ((1ull << (sh - 64)) - 1ull)};
    half = sh == 64 ? U128{1ull << 63, 0ull} : U128{0ull, 1ull << (sh - 65)};
  }
  const U128 dlt = sub128(rem, half);
  const bool near = (dlt.hi == 0 && dlt.lo <= err) || (dlt.hi == ~0ull && dlt.lo >= 0ull - err);
  const bool up = (int64_t)dlt.hi > 0 || (dlt.hi == 0 && dlt.lo != 0);
  const uint64_t bits = ((uint64_t)(sh + 958) << 52) + mant + (up ? 1ull : 0ull);
  // |W| >= 2^-60 unless x == 1 (|ln x| >= 2^-53 for x != 1), so sh >= 11: the shifts are valid
  hard = !sp && !zero && (near || sh < 11);
  if (sg) {
    const U128 E = {err, 0ull};
    hard = !sp && !zero && (sh < 11 || le128(rem, E) || le128(sub128(add128(half, half), rem), E));
    *sg = (sp || zero) ? 0 : ((up != zneg) ? -1 : 1);
  }
  return sp ? rs : (zero ? 0.0 : bitsd(bits | (zneg ? 0x8000000000000000ull : 0ull)));
}

// ------------------------------------------------------------------ signed Q126 helpers
// Signed fixed point with 126 fraction bits in 128-bit two's complement, for the
// FP64-free middle tiers of the binary32 functions.
CRM_DEV U128 q_ld(const unsigned long long *p) { return {p[0], p[1]}; }
CRM_DEV bool q_neg(U128 a) { return (int64_t)a.hi < 0; }
// (a b) 2^-126, the magnitude truncated (error below one unit); |a|, |b| <= 2^127
CRM_DEV U128 q_mul(U128 a, U128 b) {
  const bool n = q_neg(a) != q_neg(b);
  const U128 A = q_neg(a) ? neg128(a) : a, B = q_neg(b) ? neg128(b) : b;
  const U128 hh = mul64w(A.hi, B.hi), hl = mul64w(A.hi, B.lo), lh = mul64w(A.lo, B.hi);
  const uint64_t llh = __umul64hi(A.lo, B.lo);
  U128 mid = add128(hl, lh);
  uint64_t c = (mid.hi < hl.hi || (mid.hi == hl.hi && mid.lo < hl.lo)) ? 1ull : 0ull;
  mid = add128_64(mid, llh);
  c += (mid.hi == 0 && mid.lo < llh) ? 1ull : 0ull;
  const uint64_t w1 = mid.lo, w2 = hh.lo + mid.hi;
  const uint64_t w3 = hh.hi + c + (w2 < hh.lo ? 1ull : 0ull);
  const U128 r = {(w2 << 2) | (w1 >> 62), (w3 << 2) | (w2 >> 62)};
  return n ? neg128(r) : r;
}
// RN to binary32 of v 2^(es - 126) (|v| < 2^127, es >= 0, |value| >= 2^-126) when no
// midpoint lies within err units of v (err a 128-bit count)
// With sg: also the sign of the value minus the result (decided unless the discarded
// part is within err of 0 or of a full unit: then hard).
CRM_DEV float q_round_f(U128 v, U128 err, bool &hard, int es = 0, int *sg = nullptr) {
  const bool n = q_neg(v);
  const U128 A = n ? neg128(v) : v;
  const int p = A.hi ? 127 - __clzll(A.hi) : 63 - __clzll(A.lo | 1ull);  // leading bit
  const int sh = p - 23;  // discarded bits; the value is below 2^-102 when sh < 1
  if (sh < 1) {
    hard = true;
    return 0.0f;
  }
  uint64_t mant;
  U128 rem, half;
  if (sh >= 64) {
    mant = A.hi >> (sh - 64);
    rem = {A.lo, A.hi & ((1ull << (sh - 64)) - 1ull)};
    half = sh == 64 ? U128{1ull << 63, 0ull} : U128{0ull, 1ull << (sh - 65)};
  } else {
    mant = (A.lo >> sh) | (A.hi << (64 - sh));
    rem = {A.lo & ((1ull << sh) - 1ull), 0ull};
    half = {1ull << (sh - 1), 0ull};
  }
  const U128 dlt = sub128(rem, half);
  hard = le128(q_neg(dlt) ? neg128(dlt) : dlt, err);
  const uint32_t up = ((int64_t)dlt.hi > 0 || (dlt.hi == 0 && dlt.lo != 0)) ? 1u : 0u;
  if (sg) {
    hard = le128(rem, err) || le128(sub128(add128(half, half), rem), err);
    *sg = (up != 0) != n ? -1 : 1;  // |v| below |result| when rounded up; negated for v < 0
  }
  // mant 2^(sh - 126), mant in [2^23, 2^24): exponent field sh + 24, the leading bit adds 1
  if (sh + 23 + es >= 255) {  // |value| >= 2^128: infinity, beyond the finite value
    if (sg) {
      hard = false;
      *sg = n ? 1 : -1;
    }
    return n ? -CRM_INF_F : CRM_INF_F;
  }
  const uint32_t bits = ((uint32_t)(sh + 23 + es) << 23) + (uint32_t)mant + up;
  return bitsf(bits | (n ? 0x80000000u : 0u));
}

// v / d for signed Q126 values with 2^-60 <= |d| < 2: returns w and es with
// v/d = w 2^(es - 126), |w| <= |v|.  d is normalised to [1, 2) (dn = |d| 2^es, es in
// [0, 60]), 1/dn (in (1/2, 1], so Q126 holds it) by three Newton steps from a binary32
// seed (24, 48, 96 bits, then the truncation limit: relative error below 2^-118), and
// w = v (1/dn).
CRM_DEV U128 q_div(U128 v, U128 d, int &es) {
  const bool dneg = q_neg(d);
  U128 D = dneg ? neg128(d) : d;
  const int p = D.hi ? 127 - __clzll(D.hi) : 63 - __clzll(D.lo | 1ull);
  es = 126 - p;  // D 2^es in [2^126, 2^127): value in [1, 2)
  if (es > 0) D = {D.lo << es, (D.hi << es) | (D.lo >> (64 - es))};
  // seed: the leading 24 bits of D as a float, reciprocal
  const float df = (float)(D.hi >> 39) * 0x1p-23f;  // value in [1, 2)
  const float rf = 1.0f / df;                        // (1/2, 1]
  U128 R = {0ull, (uint64_t)(rf * 0x1p38f) << 24};  // rf in Q126: rf 2^126 = rf 2^62 2^64
  const U128 TWO = {0ull, 1ull << 63};               // 2 in Q126
#pragma unroll
  for (int it = 0; it < 3; it++) R = q_mul(R, sub128(TWO, q_mul(D, R)));
  const U128 w = q_mul(v, R);
  return dneg ? neg128(w) : w;
}

CRM_DEV U128 q_shr(U128 a, int s) {  // 0 <= s, a >= 0
  if (s == 0) return a;
  if (s < 64) return {(a.lo >> s) | (a.hi << (64 - s)), a.hi >> s};
  return {s < 128 ? a.hi >> (s - 64) : 0ull, 0ull};
}
CRM_DEV U128 q_shl(U128 a, int s) {  // 0 <= s < 128, no overflow
  if (s == 0) return a;
  if (s < 64) return {a.lo << s, (a.hi << s) | (a.lo >> (64 - s))};
  return {0ull, a.lo << (s - 64)};
}
// The Q126 value of a binary32 x with 2^-62 <= |x| < 2 (exact), |x|: M 2^(E - 24).
CRM_DEV U128 q_of_f(float x) {
  const uint32_t b = fbits(fabsf(x));
  const U128 M = {(uint64_t)((b & 0x007FFFFFu) | 0x00800000u), 0ull};
  const int s = (int)(b >> 23) - 24;
  return s >= 0 ? q_shl(M, s) : q_shr(M, -s);
}

// ------------------------------------------------------------------ exact slow path
struct U192 {
  uint64_t w[3];  // little endian
};
CRM_DEV U192 u_zero() { return {{0, 0, 0}}; }
CRM_DEV U192 u_add(U192 a, U192 b) {
  U192 r;
  uint64_t c = 0;
  for (int i = 0; i < 3; i++) {
    uint64_t s = a.w[i] + b.w[i];
    uint64_t c1 = s < a.w[i];
    uint64_t s2 = s + c;
    uint64_t c2 = s2 < s;
    r.w[i] = s2;
    c = c1 | c2;
  }
  return r;
}
CRM_DEV U192 u_sub(U192 a, U192 b) {  // a >= b
  U192 r;
  uint64_t br = 0;
  for (int i = 0; i < 3; i++) {
    uint64_t d = a.w[i] - b.w[i];
    uint64_t b1 = a.w[i] < b.w[i];
    uint64_t d2 = d - br;
    uint64_t b2 = d < br;
    r.w[i] = d2;
    br = b1 | b2;
  }
  return r;
}
CRM_DEV int u_cmp(U192 a, U192 b) {
  for (int i = 2; i >= 0; i--)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
CRM_DEV bool u_is_zero(U192 a) { return (a.w[0] | a.w[1] | a.w[2]) == 0; }
// floor(a b / 2^fb), 128 <= fb < 192, result assumed to fit in 192 bits
CRM_DEV U192 u_mulfx(U192 a, U192 b, int fb) {
  uint64_t p[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 3; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < 3; j++) {
      uint64_t lo = a.w[i] * b.w[j], hi = __umul64hi(a.w[i], b.w[j]);
      uint64_t s = p[i + j] + lo;
      hi += s < lo;
      uint64_t s2 = s + carry;
      hi += s2 < s;
      p[i + j] = s2;
      carry = hi;
    }
    p[i + 3] += carry;
  }
  int wsh = fb >> 6, bsh = fb & 63;
  U192 r;
  for (int i = 0; i < 3; i++) {
    uint64_t lo = p[i + wsh];
    uint64_t hi = (i + wsh + 1 < 6) ? p[i + wsh + 1] : 0;
    r.w[i] = bsh ? (lo >> bsh) | (hi << (64 - bsh)) : lo;
  }
  return r;
}
CRM_DEV U192 u_divsmall(U192 a, uint64_t d) {  // floor(a / d), d < 2^32
  U192 r;
  uint64_t rem = 0;
  for (int i = 2; i >= 0; i--) {
    uint64_t hi = (rem << 32) | (a.w[i] >> 32);
    uint64_t qh = hi / d;
    rem = hi - qh * d;
    uint64_t lo = (rem << 32) | (a.w[i] & 0xFFFFFFFFull);
    uint64_t ql = lo / d;
    rem = lo - ql * d;
    r.w[i] = (qh << 32) | ql;
  }
  return r;
}
CRM_DEV U192 u_mul_small(U192 a, uint64_t m) {  // a m, m < 2^32, no overflow
  U192 r;
  uint64_t carry = 0;
  for (int i = 0; i < 3; i++) {
    uint64_t lo = a.w[i] * m, hi = __umul64hi(a.w[i], m);
    uint64_t s = lo + carry;
    hi += s < lo;
    r.w[i] = s;
    carry = hi;
  }
  return r;
}
CRM_DEV U192 u_shr(U192 a, int k) {  // k < 192
  U192 r = u_zero();
  int ws = k >> 6, bs = k & 63;
  for (int i = 0; i + ws < 3; i++) {
    uint64_t lo = a.w[i + ws], hi = (i + ws + 1 < 3) ? a.w[i + ws + 1] : 0;
    r.w[i] = bs ? (lo >> bs) | (hi << (64 - bs)) : lo;
  }
  return r;
}
CRM_DEV U192 u_shl(U192 a, int k) {  // k < 192, no overflow
  U192 r = u_zero();
  int ws = k >> 6, bs = k & 63;
  for (int i = 2; i - ws >= 0; i--) {
    uint64_t hi = a.w[i - ws], lo = (i - ws - 1 >= 0) ? a.w[i - ws - 1] : 0;
    r.w[i] = bs ? (hi << bs) | (lo >> (64 - bs)) : hi;
  }
  return r;
}
CRM_DEV int u_bitlen(U192 a) {
  for (int i = 2; i >= 0; i--)
    if (a.w[i]) return 64 * i + 64 - __clzll((long long)a.w[i]);
  return 0;
}
CRM_DEV bool u_bit(U192 a, int i) { return i >= 0 && i < 192 && ((a.w[i >> 6] >> (i & 63)) & 1); }
CRM_DEV U192 u_low(U192 a, int k) {  // a mod 2^k
  U192 r = a;
  for (int i = 0; i < 3; i++) {
    int lo = 64 * i;
    if (k <= lo) r.w[i] = 0;
    else if (k < lo + 64) r.w[i] &= (1ull << (k - lo)) - 1;
  }
  return r;
}
CRM_DEV U192 u_pow2(int k) {
  U192 r = u_zero();
  r.w[k >> 6] = 1ull << (k & 63);
  return r;
}

// Round the interval [M - dlo, M + dhi] (value M 2^-fb, M > 0) to binary64 nearest.
// Returns false (unresolved) if a midpoint lies inside.  `neg` sets the sign.
// With sg (directed rounding): out = the truncation of M (q ulps) and *sg = +-1 (the sign
// of the value minus out), when the whole interval lies strictly between q and q + 1 ulps;
// false otherwise (an exact result is decided by the caller).
CRM_DEV bool u_round64(U192 M, int fb, uint64_t dlo, uint64_t dhi, bool neg, double &out, int *sg = nullptr) {
  int b = u_bitlen(M);  // value in [2^(b-1-fb), 2^(b-fb))
  int ex = b - 1 - fb;
  int drop;
  if (ex >= -1022)
    drop = b - 53;
  else
    drop = b - 53 + (-1022 - ex);
  if (drop <= 0 || drop > 191) return false;  // not reached by exp2 / log
  U192 q = u_shr(M, drop);
  U192 rem = u_low(M, drop);
  U192 half = u_pow2(drop - 1);
  U192 lo = u_sub(rem, U192{{dlo, 0, 0}});  // rem >= dlo assumed (checked below)
  bool lo_ok = u_cmp(rem, U192{{dlo, 0, 0}}) >= 0;
  U192 hi = u_add(rem, U192{{dhi, 0, 0}});
  bool up;
  if (sg) {
    if (!lo_ok || u_is_zero(lo) || u_cmp(hi, u_add(half, half)) >= 0) return false;
    up = false;
    *sg = neg ? -1 : 1;
  } else if (lo_ok && u_cmp(lo, half) > 0)
    up = true;
  else if (u_cmp(hi, half) < 0)
    up = false;
  else
    return false;
  uint64_t qv = q.w[0];
  uint64_t bits;
  if (ex >= -1022)
    bits = ((uint64_t)(ex + 1023) << 52) + (qv - (1ull << 52));
  else
    bits = qv;
  bits += up ? 1 : 0;
  if (bits >= 0x7FF0000000000000ull) bits = 0x7FF0000000000000ull;
  out = bitsd(bits | (neg ? 0x8000000000000000ull : 0));
  return true;
}

// exp2(x), x in (-1075, 1024), exactly: R = x - floor(4096 x)/4096 in [0, 2^-12),
// u = R ln2 (Q0.191), e^u by Taylor (Q2.190), times the three table values (Q2.190).
// Every step truncates (floors), so the computed y satisfies y <= 2^x 2^-k < y + 2^10
// units of 2^-190 (16 Taylor terms, 4 products, R and ln2 truncation).
// R = x - N/4096 is exact in binary64 unless -2^-13 < x < 0 (then N = -1 and R = 2^-12 - |x|
// spans more than 53 bits): there R is formed in fixed point, rounded down like every other
// step, as 2^179 - ceil(|x| 2^191).
CRM_DEV bool exp2d_exact(double x, double &out, int *sg = nullptr) {
  double nd = floor(x * 4096.0);
  long long N = (long long)nd;
  double R = fma_(nd, -0x1p-12, x);  // exact, in [0, 2^-12), unless -2^-13 < x < 0
  int k = (int)(N >> 12);
  int i = (int)(N & 4095);
  U192 Rf = u_zero();
  if (x < 0.0 && x > -0x1p-13) {
    const uint64_t xb = dbits(x) & 0x7FFFFFFFFFFFFFFFull;
    const int be = (int)(xb >> 52);
    const uint64_t xm = (xb & 0x000FFFFFFFFFFFFFull) | (be ? (1ull << 52) : 0ull);
    const int sh = (be ? be - 1075 : -1074) + 191;  // |x| 2^191 = xm 2^sh, sh <= 125
    U192 c;
    if (sh >= 0) {
      c = u_shl(U192{{xm, 0, 0}}, sh);
    } else {
      const int d = -sh;
      const uint64_t q = d < 64 ? (xm >> d) : 0ull;
      const bool lost = d < 64 ? (xm & ((1ull << d) - 1ull)) != 0 : true;
      c = U192{{q + (lost ? 1ull : 0ull), 0, 0}};
    }
    Rf = u_sub(u_pow2(179), c);
  } else if (R > 0.0) {
    uint64_t rb = dbits(R);
    int re = (int)(rb >> 52) - 1075;
    uint64_t rm = (rb & 0x000FFFFFFFFFFFFFull) | ((rb >> 52) ? (1ull << 52) : 0);
    if ((rb >> 52) == 0) re = -1074;
    int sh = re + 191;  // R 2^191 = rm 2^sh
    U192 t = {{rm, 0, 0}};
    Rf = sh >= 0 ? u_shl(t, sh) : (sh > -64 ? u_shr(t, -sh) : u_zero());
  }
  U192 ln2 = {{CRM_LN2_FX[0], CRM_LN2_FX[1], CRM_LN2_FX[2]}};
  U192 u = u_shr(u_mulfx(Rf, ln2, 191), 1);  // Q2.190
  U192 one = u_pow2(190);
  U192 sum = u_add(one, u), term = u;
  for (uint64_t n = 2; n < 40 && !u_is_zero(term); n++) {
    term = u_divsmall(u_mulfx(term, u, 190), n);
    sum = u_add(sum, term);
  }
  const unsigned long long *T = CRM_EXP2_FX_T;
  int idx[3] = {i >> 8, (i >> 4) & 15, i & 15};
  for (int a = 0; a < 3; a++) {
    const unsigned long long *e = T + 48 * a + 3 * idx[a];
    sum = u_mulfx(sum, U192{{e[0], e[1], e[2]}}, 190);
  }
  // value = sum 2^(k - 190): round with the interval [sum, sum + 2^10]
  return u_round64(sum, 190 - k, 0, 1024, false, out, sg);
}

// log(x), x > 0 finite, exactly: x = 2^e m, m in [1,2), c = 1 + j/128 <= m,
// r = (m - c)/c in [0, 1/128) (Q0.191), log1p(r) = P - Q with P and Q the positive and
// negative Taylor terms, S = log(c) + log1p(r); |log x| = |e ln2 + S| in Q11.181.
// |ln x| in Q11.181 (M, with the sign of ln x in neg) for x = 2^e (1 + f 2^-52), within
// |e| + 16 units (below); false for x = 1.
CRM_DEV bool logd_abs_q181(int e, uint64_t f, U192 &M, bool &neg, uint64_t &ae) {
  int j = (int)(f >> 45);
  uint64_t dlow = f & ((1ull << 45) - 1);  // (m - c) 2^52
  // r = (m - c) 128 / (128 + j) in Q0.191: (m - c) 2^191 = dlow 2^139
  U192 r = u_divsmall(u_shl(U192{{dlow, 0, 0}}, 139 + 7), 128 + j);
  U192 P = u_zero(), Q = u_zero(), pw = r;
  for (uint64_t n = 1; n < 40 && !u_is_zero(pw); n++) {
    U192 t = u_divsmall(pw, n);
    if (n & 1) P = u_add(P, t); else Q = u_add(Q, t);
    pw = u_mulfx(pw, r, 191);
  }
  U192 L = {{CRM_LOG_FX_T[3 * j], CRM_LOG_FX_T[3 * j + 1], CRM_LOG_FX_T[3 * j + 2]}};
  U192 S = u_sub(u_add(L, P), Q);  // in [0, ln2), Q0.191, error within +-64 units
  U192 ln2 = {{CRM_LN2_FX[0], CRM_LN2_FX[1], CRM_LN2_FX[2]}};
  U192 S10 = u_shr(S, 10);  // Q11.181
  ae = (uint64_t)(e < 0 ? -e : e);
  U192 E = u_mul_small(u_shr(ln2, 10), ae);  // |e| ln2 < 2^10.5 fits Q11.181
  neg = false;
  if (e >= 0) {
    M = u_add(E, S10);
  } else {
    M = u_sub(E, S10);
    neg = true;
  }
  return !u_is_zero(M);
}

CRM_DEV bool logd_exact(double x, double &out, int *sg = nullptr) {
  uint64_t b = dbits(x);
  int be = (int)(b >> 52);
  uint64_t f = b & 0x000FFFFFFFFFFFFFull;
  int e;
  if (be == 0) {  // subnormal: move the leading 1 (at bit 52 - lz) to bit 52
    int lz = __clzll((long long)f) - 11;
    f = (f << lz) & 0x000FFFFFFFFFFFFFull;
    e = -1022 - lz;
  } else {
    e = be - 1023;
  }
  U192 M;
  bool neg;
  uint64_t ae;
  if (!logd_abs_q181(e, f, M, neg, ae)) return false;
  // errors (units of 2^-181): S within 64 units of 2^-191 (< 1), the shift of S 1, the
  // truncated ln2 times |e|: |e| + 1.  The interval is M -+ (|e| + 16).
  return u_round64(M, 181, ae + 16, ae + 16, neg, out, sg);
}

CRM_DEV double exp2d_slow(double x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  double r = exp2d_main(x, CRM_EXP2D_T, hard, sg);
  unresolved = 2;  // the double-double tier (FP64) ran
  double sp;
  if ((!hard && !force) || exp2d_special(x, sp)) return r;
  double out;
  if (x == rint(x)) {  // exact powers of two
    put_sg(sg, 0);
    return ldexp(1.0, (int)x);
  }
  bool ok = exp2d_exact(x, out, sg);
  unresolved = ok ? 2 : 3;
  return ok ? out : r;
}

CRM_DEV double logd_slow(double x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  double r = logd_main(x, hard, sg);
  unresolved = 2;  // the double-double tier (FP64) ran
  double sp;
  if ((!hard && !force) || logd_special(x, sp)) return r;
  if (x == 1.0) {
    put_sg(sg, 0);
    return 0.0;
  }
  double out;
  bool ok = logd_exact(x, out, sg);
  unresolved = ok ? 2 : 3;
  return ok ? out : r;
}


// ------------------------------------------------------------------ exact tiers of e^x, 10^x, log2, log10
// b^x: t = x log2 b in Q180 from x's significand times log2 b (Q190 / Q189, truncated),
// t = N/4096 + R (R in [0, 2^-12)), then exp2d_exact's pipeline on R.  The truncations move
// t by at most 2^-169 (|x| < 2^10), i.e. 2^-169.5 of the result or 2^21.5 units of 2^-190:
// the interval [sum - 2^23, sum + 2^23 + 2^10].
template <int KIND> CRM_DEV bool expbd_exact(double x, double &out, int *sg = nullptr) {
  const uint64_t b = dbits(x), ab = b & 0x7FFFFFFFFFFFFFFFull;
  const int E = (int)(ab >> 52);
  const uint64_t M = (ab & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  const U192 C = KIND == 0 ? U192{{CRM_LOG2E_FX[0], CRM_LOG2E_FX[1], CRM_LOG2E_FX[2]}}
                           : U192{{CRM_LOG2_10_FX[0], CRM_LOG2_10_FX[1], CRM_LOG2_10_FX[2]}};
  const int fc = KIND == 0 ? 190 : 189;
  // |t| 2^180 = M C 2^(E - 1075 - fc + 180) = (M C) >> (fc + 895 - E), the shift in [52, 122]
  const U192 tf = u_mulfx(U192{{M, 0, 0}}, C, fc + 895 - E);
  // N = floor(4096 t), R = t - N/4096 in Q191
  const U192 q = u_shr(tf, 168);
  const U192 rem = u_low(tf, 168);
  long long N = (long long)q.w[0];
  U192 Rf;
  if (!(b >> 63)) {
    Rf = u_shl(rem, 11);
  } else if (u_is_zero(rem)) {
    N = -N;
    Rf = u_zero();
  } else {
    N = -N - 1;
    Rf = u_shl(u_sub(u_pow2(168), rem), 11);
  }
  const int k = (int)(N >> 12);
  const int i = (int)(N & 4095);
  U192 ln2 = {{CRM_LN2_FX[0], CRM_LN2_FX[1], CRM_LN2_FX[2]}};
  U192 u = u_shr(u_mulfx(Rf, ln2, 191), 1);  // Q2.190
  U192 sum = u_add(u_pow2(190), u), term = u;
  for (uint64_t n = 2; n < 40 && !u_is_zero(term); n++) {
    term = u_divsmall(u_mulfx(term, u, 190), n);
    sum = u_add(sum, term);
  }
  const unsigned long long *T = CRM_EXP2_FX_T;
  int idx[3] = {i >> 8, (i >> 4) & 15, i & 15};
  for (int a = 0; a < 3; a++) {
    const unsigned long long *e = T + 48 * a + 3 * idx[a];
    sum = u_mulfx(sum, U192{{e[0], e[1], e[2]}}, 190);
  }
  return u_round64(sum, 190 - k, 1ull << 23, (1ull << 23) + 1024, false, out, sg);
}

template <int KIND> CRM_DEV double expbd_slow(double x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = 0;
  double r = expbd_int<KIND>(x, (const ulonglong2 *)CRM_EXP2I_T, hard, sg);
  if (!hard && !force) return r;
  const uint64_t ab = dbits(x) & 0x7FFFFFFFFFFFFFFFull;
  // special inputs, |x| < 2^-60, and results decided as overflow (+inf) or below half the
  // smallest subnormal (+0) by the range of k are exact statements of the first tier
  if (ab >= 0x4090000000000000ull || (int)(ab >> 52) < 1023 - 60 || (!hard && (isinf(r) || r == 0.0))) return r;
  if (KIND == 2 && x == rint(x) && x >= 1.0 && x <= 27.0) {
    // 10^k = 5^k 2^k (5^k < 2^63) rounded directly: exact for k <= 22, a midpoint for
    // k = 23 (5^23 is an odd 54-bit integer), which no error bound can decide
    const int kk = (int)x;
    uint64_t p5 = 1;
    for (int j = 0; j < kk; j++) p5 *= 5ull;
    const int bl = 64 - __clzll((long long)p5);
    uint64_t q = p5;
    int sh = 0, s5 = 0;
    if (bl > 53) {
      sh = bl - 53;
      const uint64_t rem = p5 & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
      q = p5 >> sh;
      const bool up = rem > half || (rem == half && (q & 1ull));
      q += up ? 1ull : 0ull;
      s5 = rem == 0 ? 0 : (up ? -1 : 1);
    }
    put_sg(sg, s5);
    return ldexp((double)q, sh + kk);
  }
  double out;
  const bool ok = expbd_exact<KIND>(x, out, sg);
  unresolved = ok ? 0 : 1;
  return ok ? out : r;
}

// log2, log10: |ln x| in Q181 from logd_exact's pipeline, times 1/ln b in Q190 (truncated),
// error (|e| + 16) C + 2 units, taken as 2 (|e| + 16) + 4.
template <int KIND> CRM_DEV bool logbd_exact(double x, double &out, int *sg = nullptr) {
  uint64_t b = dbits(x);
  int be = (int)(b >> 52);
  uint64_t f = b & 0x000FFFFFFFFFFFFFull;
  int e;
  if (be == 0) {
    const int lz = __clzll(f) - 11;
    f = (f << lz) & 0x000FFFFFFFFFFFFFull;
    e = -1022 - lz;
  } else {
    e = be - 1023;
  }
  U192 M;
  bool neg;
  uint64_t ae;
  if (!logd_abs_q181(e, f, M, neg, ae)) return false;
  const U192 C = KIND == 1 ? U192{{CRM_INV_LN2_FX[0], CRM_INV_LN2_FX[1], CRM_INV_LN2_FX[2]}}
                           : U192{{CRM_INV_LN10_FX[0], CRM_INV_LN10_FX[1], CRM_INV_LN10_FX[2]}};
  const U192 W = u_mulfx(M, C, 190);
  const uint64_t er = 2 * (ae + 16) + 4;
  return u_round64(W, 181, er, er, neg, out, sg);
}

template <int KIND> CRM_DEV double logbd_slow(double x, int &unresolved, bool force, int *sg = nullptr) {
  bool hard;
  unresolved = 0;
  double r = logbd_int<KIND>(x, (const ulonglong2 *)CRM_LOGI_L, CRM_LOGI_R, hard, sg);
  if (!hard && !force) return r;
  double sp;
  if (logd_special(x, sp)) return r;
  if (x == 1.0) {
    put_sg(sg, 0);
    return 0.0;
  }
  if (sg) {  // exact results: log2 of a power of two, log10 of 10^k (k <= 22)
    const uint64_t b = dbits(x), f = b & 0x000FFFFFFFFFFFFFull;
    const int be = (int)(b >> 52);
    if (KIND == 1 && ((be != 0 && f == 0) || (be == 0 && (f & (f - 1)) == 0))) {
      *sg = 0;
      return be != 0 ? (double)(be - 1023) : (double)(63 - __clzll(f) - 1074);
    }
    if (KIND == 2) {
      double p = 1.0;
      for (int j = 1; j <= 22; j++) {
        p *= 10.0;
        if (x == p) {
          *sg = 0;
          return (double)j;
        }
      }
    }
  }
  double out;
  const bool ok = logbd_exact<KIND>(x, out, sg);
  unresolved = ok ? 0 : 1;
  return ok ? out : r;
}

}  // namespace crm
