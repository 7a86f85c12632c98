/*
 * crm_oracle.c -- correctly rounded reference evaluator (TEST INFRASTRUCTURE ONLY).
 *
 * What it computes: out = RN_fmt(f(x)), the correctly rounded (to nearest, ties to
 * even) value of f at the floating-point input x, in binary32 or binary64, with
 * gradual underflow and overflow to infinity (the correct-rounding goal of Sec. I and
 * Sec. II; GPU runs use round-to-nearest-even only, Sec. III.C).  The _rm entry points
 * round in a directed mode instead (toward -inf, +inf or zero, IEEE 754 Sec. 4.3): the
 * same loop with the mode in the final rounding, exact results listed before it.
 *
 * How: Ziv's strategy (Sec. I).  Every quantity is an interval [lo, hi] of fixed-point
 * numbers N / 2^F held as two's-complement multi-limb integers (F = 64*(n-1) fraction
 * bits, one 64-bit integer limb).  Every operation rounds lo down and hi up, every
 * truncated series is widened by a bound on its remainder, so the final interval
 * provably contains f(x).  If both ends round to the same format value the answer is
 * decided (rounding to nearest is monotone, so no midpoint lies in between);
 * otherwise the precision is raised.  Exact midpoints and exact zeros would never be
 * decided that way; they are produced as exact (degenerate) intervals or as special
 * values before the loop.  Reaching the last precision is reported as an error.
 *
 * Special-value conventions (the paper does not fix them; this is the reading used
 * throughout the project): a NaN input is returned quieted with sign and payload kept;
 * an invalid operation returns the default quiet NaN (+, 0x7FC00000 / 0x7FF8...);
 * odd functions keep the sign of zero; log-family(+-0) = -inf; rsqrt(+-0) = +-inf.
 *
 * This file shares no code with the GPU library.  The C library's floating-point
 * math is used only to pick reduction integers (any choice is correct; a good one is
 * merely faster), never to produce a value.
 */
#include "crm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef uint64_t limb;
typedef unsigned __int128 u128;

#define MAXL 48 /* limbs per fixed-point number */
#define FB(n) (64 * ((n) - 1)) /* fraction bits at n limbs */

static void die(const char *what) {
  fprintf(stderr, "crm_oracle: internal error: %s\n", what);
  abort();
}

/* Set when an operation cannot give a valid enclosure at this precision (division by
   an interval containing zero, square root of an interval reaching below zero).  The
   Ziv loop then retries at a higher precision. */
static __thread int g_fail;
static __thread int g_last_level;

/* ===================== magnitude (unsigned) helpers ===================== */

static int mag_bitlen(const limb *a, int n) {
  for (int i = n - 1; i >= 0; i--)
    if (a[i]) return 64 * i + 64 - __builtin_clzll(a[i]);
  return 0;
}
static int mag_is_zero(const limb *a, int n) {
  for (int i = 0; i < n; i++)
    if (a[i]) return 0;
  return 1;
}
static int mag_cmp(const limb *a, const limb *b, int n) {
  for (int i = n - 1; i >= 0; i--)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}
static void mag_inc(limb *a, int n) {
  for (int i = 0; i < n; i++)
    if (++a[i]) return;
}
static void mag_add(limb *r, const limb *a, const limb *b, int n) {
  u128 c = 0;
  for (int i = 0; i < n; i++) {
    c += (u128)a[i] + b[i];
    r[i] = (limb)c;
    c >>= 64;
  }
}
static void mag_sub(limb *r, const limb *a, const limb *b, int n) { /* a >= b */
  limb br = 0;
  for (int i = 0; i < n; i++) {
    u128 t = (u128)a[i] - b[i] - br;
    r[i] = (limb)t;
    br = (limb)(t >> 64) ? 1 : 0;
  }
}
/* bit i of a (0 if beyond) */
static int mag_bit(const limb *a, int n, int64_t i) {
  if (i < 0 || i >= 64 * (int64_t)n) return 0;
  return (int)((a[i >> 6] >> (i & 63)) & 1);
}
/* 1 if any bit strictly below position i is set */
static int mag_any_below(const limb *a, int n, int64_t i) {
  if (i <= 0) return 0;
  if (i >= 64 * (int64_t)n) return !mag_is_zero(a, n);
  int64_t w = i >> 6;
  for (int64_t j = 0; j < w; j++)
    if (a[j]) return 1;
  int b = (int)(i & 63);
  return b ? (a[w] & ((1ull << b) - 1)) != 0 : 0;
}
/* r = a << k within n limbs; dies if bits are lost */
static void mag_shl(limb *r, const limb *a, int n, int64_t k) {
  if (mag_is_zero(a, n)) {
    memset(r, 0, 8 * (size_t)n);
    return;
  }
  if (mag_bitlen(a, n) + k > 64 * (int64_t)n) die("shift overflow");
  limb t[MAXL * 2];
  int64_t w = k >> 6;
  int b = (int)(k & 63);
  for (int i = n - 1; i >= 0; i--) {
    int64_t s = i - w;
    limb v = 0;
    if (s >= 0) {
      v = a[s] << b;
      if (b && s - 1 >= 0) v |= a[s - 1] >> (64 - b);
    }
    t[i] = v;
  }
  memcpy(r, t, 8 * (size_t)n);
}
/* r = a >> k; returns 1 if nonzero bits were dropped */
static int mag_shr(limb *r, const limb *a, int n, int64_t k) {
  int inexact = mag_any_below(a, n, k);
  limb t[MAXL * 2];
  int64_t w = k >> 6;
  int b = (int)(k & 63);
  for (int i = 0; i < n; i++) {
    int64_t s = i + w;
    limb v = 0;
    if (s < n) {
      v = a[s] >> b;
      if (b && s + 1 < n) v |= a[s + 1] << (64 - b);
    }
    t[i] = v;
  }
  memcpy(r, t, 8 * (size_t)n);
  return inexact;
}
static void mag_mul(limb *p, const limb *a, int na, const limb *b, int nb) {
  memset(p, 0, 8 * (size_t)(na + nb));
  for (int i = 0; i < na; i++) {
    if (!a[i]) continue;
    u128 c = 0;
    for (int j = 0; j < nb; j++) {
      c += (u128)a[i] * b[j] + p[i + j];
      p[i + j] = (limb)c;
      c >>= 64;
    }
    p[i + nb] = (limb)c;
  }
}

/* Long division of 32-bit digit strings (Knuth, TAOCP vol. 2, 4.3.1, Algorithm D).
   q = floor(u / v) with m - nv + 1 digits; returns 1 if the remainder is nonzero. */
static int divmod_d32(uint32_t *q, const uint32_t *u, int m, const uint32_t *v, int nv) {
  if (nv == 1) {
    uint64_t rem = 0;
    for (int i = m - 1; i >= 0; i--) {
      uint64_t cur = (rem << 32) | u[i];
      q[i] = (uint32_t)(cur / v[0]);
      rem = cur % v[0];
    }
    return rem != 0;
  }
  uint32_t un[4 * MAXL + 4], vn[4 * MAXL + 4];
  int s = __builtin_clz(v[nv - 1]);
  for (int i = nv - 1; i > 0; i--)
    vn[i] = (v[i] << s) | (s ? (uint32_t)((uint64_t)v[i - 1] >> (32 - s)) : 0u);
  vn[0] = v[0] << s;
  un[m] = s ? (uint32_t)((uint64_t)u[m - 1] >> (32 - s)) : 0u;
  for (int i = m - 1; i > 0; i--)
    un[i] = (u[i] << s) | (s ? (uint32_t)((uint64_t)u[i - 1] >> (32 - s)) : 0u);
  un[0] = u[0] << s;
  for (int j = m - nv; j >= 0; j--) {
    uint64_t num = ((uint64_t)un[j + nv] << 32) | un[j + nv - 1];
    uint64_t qhat = num / vn[nv - 1];
    uint64_t rhat = num - qhat * vn[nv - 1];
    while (qhat >= (1ull << 32) || qhat * vn[nv - 2] > ((rhat << 32) | un[j + nv - 2])) {
      qhat--;
      rhat += vn[nv - 1];
      if (rhat >= (1ull << 32)) break;
    }
    int64_t borrow = 0, t;
    for (int i = 0; i < nv; i++) {
      uint64_t p = qhat * vn[i];
      t = (int64_t)un[i + j] - borrow - (int64_t)(p & 0xFFFFFFFFull);
      un[i + j] = (uint32_t)t;
      borrow = (int64_t)(p >> 32) - (t >> 32);
    }
    t = (int64_t)un[j + nv] - borrow;
    un[j + nv] = (uint32_t)t;
    q[j] = (uint32_t)qhat;
    if (t < 0) {
      q[j]--;
      uint64_t c = 0;
      for (int i = 0; i < nv; i++) {
        c += (uint64_t)un[i + j] + vn[i];
        un[i + j] = (uint32_t)c;
        c >>= 32;
      }
      un[j + nv] = (uint32_t)((uint64_t)un[j + nv] + c);
    }
  }
  for (int i = 0; i < nv; i++)
    if (un[i]) return 1;
  return 0;
}

/* q = floor(a / b) for magnitudes a (na limbs) and b (nb limbs, nonzero); q gets na
   limbs; returns 1 if inexact. */
static int mag_div(limb *q, const limb *a, int na, const limb *b, int nb) {
  uint32_t u[4 * MAXL + 4], v[4 * MAXL + 4], qq[4 * MAXL + 4];
  int m = 2 * na, nv = 2 * nb;
  for (int i = 0; i < na; i++) {
    u[2 * i] = (uint32_t)a[i];
    u[2 * i + 1] = (uint32_t)(a[i] >> 32);
  }
  for (int i = 0; i < nb; i++) {
    v[2 * i] = (uint32_t)b[i];
    v[2 * i + 1] = (uint32_t)(b[i] >> 32);
  }
  while (nv > 0 && v[nv - 1] == 0) nv--;
  if (nv == 0) die("division by zero");
  while (m > 0 && u[m - 1] == 0) m--;
  memset(q, 0, 8 * (size_t)na);
  if (m < nv) return m > 0;
  int inexact = divmod_d32(qq, u, m, v, nv);
  for (int i = 0; i <= m - nv; i++) q[i >> 1] |= (limb)qq[i] << (32 * (i & 1));
  return inexact;
}

/* floor(sqrt(N)) by Newton's iteration on integers (Heron's rule with floors): from any
   start x >= floor(sqrt(N)) the sequence x' = floor((x + floor(N / x)) / 2) decreases
   strictly until it reaches floor(sqrt(N)), where the next step no longer decreases.
   Returns 1 if inexact (N is not a perfect square). */
static int mag_isqrt(limb *res, const limb *N, int nl) {
  limb x[2 * MAXL + 2], q[2 * MAXL + 2], y[2 * MAXL + 2], sq[4 * MAXL + 4];
  int b = mag_bitlen(N, nl);
  memset(res, 0, 8 * (size_t)nl);
  if (b == 0) return 0;
  memset(x, 0, 8 * (size_t)(nl + 1));
  int h = (b + 1) / 2; /* 2^h >= sqrt(N) since N < 2^b <= 2^(2h) */
  x[h >> 6] = 1ull << (h & 63);
  for (;;) {
    mag_div(q, N, nl, x, nl);
    q[nl] = 0;
    mag_add(y, x, q, nl + 1);
    mag_shr(y, y, nl + 1, 1);
    if (mag_cmp(y, x, nl + 1) >= 0) break;
    memcpy(x, y, 8 * (size_t)(nl + 1));
  }
  memcpy(res, x, 8 * (size_t)nl);
  mag_mul(sq, x, nl, x, nl);
  for (int i = nl; i < 2 * nl; i++)
    if (sq[i]) die("isqrt: square too large");
  return mag_cmp(sq, N, nl) != 0;
}

/* ===================== signed fixed point (value = N / 2^F) ===================== */

static int fx_isneg(const limb *a, int n) { return (int64_t)a[n - 1] < 0; }
static int fx_sgn(const limb *a, int n) {
  if (fx_isneg(a, n)) return -1;
  return mag_is_zero(a, n) ? 0 : 1;
}
static void fx_neg(limb *r, const limb *a, int n) {
  u128 c = 1;
  for (int i = 0; i < n; i++) {
    c += (limb)~a[i];
    r[i] = (limb)c;
    c >>= 64;
  }
}
static int fx_abs(limb *r, const limb *a, int n) { /* returns 1 if a < 0 */
  if (fx_isneg(a, n)) {
    fx_neg(r, a, n);
    return 1;
  }
  if (r != a) memcpy(r, a, 8 * (size_t)n);
  return 0;
}
static int fx_cmp(const limb *a, const limb *b, int n) {
  int64_t ta = (int64_t)a[n - 1], tb = (int64_t)b[n - 1];
  if (ta != tb) return ta < tb ? -1 : 1;
  for (int i = n - 2; i >= 0; i--)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}
static void fx_add(limb *r, const limb *a, const limb *b, int n) { mag_add(r, a, b, n); }
static void fx_sub(limb *r, const limb *a, const limb *b, int n) {
  limb br = 0;
  for (int i = 0; i < n; i++) {
    u128 t = (u128)a[i] - b[i] - br;
    r[i] = (limb)t;
    br = (limb)(t >> 64) ? 1 : 0;
  }
}
static void fx_set_i64(limb *r, int64_t v, int n) {
  memset(r, 0, 8 * (size_t)n);
  r[n - 1] = (limb)v;
}
/* Given the magnitude q of a result, its sign and whether it was truncated, store the
   signed result rounded toward -inf (dir < 0) or +inf (dir > 0). */
static void fx_finish(limb *r, limb *q, int n, int neg, int inexact, int dir) {
  int away = neg ? (dir < 0) : (dir > 0);
  if (away && inexact) mag_inc(q, n);
  if (q[n - 1] >> 63) die("fixed-point overflow");
  if (neg)
    fx_neg(r, q, n);
  else
    memcpy(r, q, 8 * (size_t)n);
}
/* r = a * b, rounded in direction dir */
static void fx_mul(limb *r, const limb *a, const limb *b, int n, int dir) {
  limb ma[MAXL], mb[MAXL], p[2 * MAXL], q[MAXL];
  int neg = fx_abs(ma, a, n) ^ fx_abs(mb, b, n);
  mag_mul(p, ma, n, mb, n);
  int inexact = 0;
  for (int i = 0; i < n - 1; i++)
    if (p[i]) inexact = 1;
  if (p[2 * n - 1]) die("mul overflow");
  memcpy(q, p + n - 1, 8 * (size_t)n);
  fx_finish(r, q, n, neg, inexact, dir);
}
/* r = a / b, rounded in direction dir (b != 0) */
static void fx_div(limb *r, const limb *a, const limb *b, int n, int dir) {
  limb ma[MAXL], mb[MAXL], num[2 * MAXL], q[2 * MAXL];
  int neg = fx_abs(ma, a, n) ^ fx_abs(mb, b, n);
  memset(num, 0, 8 * (size_t)(2 * n - 1));
  memcpy(num + n - 1, ma, 8 * (size_t)n);
  int inexact = mag_div(q, num, 2 * n - 1, mb, n);
  for (int i = n; i < 2 * n - 1; i++)
    if (q[i]) die("div overflow");
  fx_finish(r, q, n, neg, inexact, dir);
}
/* r = a * m (exact) */
static void fx_mul_u(limb *r, const limb *a, uint64_t m, int n) {
  limb ma[MAXL], q[MAXL];
  int neg = fx_abs(ma, a, n);
  u128 c = 0;
  for (int i = 0; i < n; i++) {
    c += (u128)ma[i] * m;
    q[i] = (limb)c;
    c >>= 64;
  }
  if (c) die("mul_u overflow");
  fx_finish(r, q, n, neg, 0, 0);
}
/* r = a / d rounded in direction dir */
static void fx_div_u(limb *r, const limb *a, uint64_t d, int n, int dir) {
  limb ma[MAXL], q[MAXL];
  int neg = fx_abs(ma, a, n);
  u128 rem = 0;
  for (int i = n - 1; i >= 0; i--) {
    u128 cur = (rem << 64) | ma[i];
    q[i] = (limb)(cur / d);
    rem = cur % d;
  }
  fx_finish(r, q, n, neg, rem != 0, dir);
}
/* r = a * 2^-k rounded in direction dir (k >= 0) */
static void fx_shr(limb *r, const limb *a, int64_t k, int n, int dir) {
  limb ma[MAXL], q[MAXL];
  int neg = fx_abs(ma, a, n);
  int inexact = mag_shr(q, ma, n, k);
  fx_finish(r, q, n, neg, inexact, dir);
}
static void fx_shl(limb *r, const limb *a, int64_t k, int n) {
  limb ma[MAXL], q[MAXL];
  int neg = fx_abs(ma, a, n);
  mag_shl(q, ma, n, k);
  fx_finish(r, q, n, neg, 0, 0);
}
/* r = sqrt(a) rounded in direction dir (a >= 0) */
static void fx_sqrt(limb *r, const limb *a, int n, int dir) {
  limb N[2 * MAXL], s[2 * MAXL];
  memset(N, 0, 8 * (size_t)(2 * n - 1));
  memcpy(N + n - 1, a, 8 * (size_t)n);
  int inexact = mag_isqrt(s, N, 2 * n - 1);
  for (int i = n; i < 2 * n - 1; i++)
    if (s[i]) die("sqrt overflow");
  fx_finish(r, s, n, 0, inexact, dir);
}
/* r = M * 2^e rounded in direction dir (value >= 0) */
static void fx_set_scaled(limb *r, uint64_t M, int64_t e, int n, int dir) {
  limb q[MAXL];
  memset(q, 0, 8 * (size_t)n);
  q[0] = M;
  int64_t k = e + FB(n);
  int inexact = 0;
  if (k >= 0)
    mag_shl(q, q, n, k);
  else
    inexact = mag_shr(q, q, n, -k);
  fx_finish(r, q, n, 0, inexact, dir);
}

/* ===================== intervals ===================== */

typedef struct {
  limb lo[MAXL], hi[MAXL];
} iv_t;

static void iv_set_i(iv_t *r, int64_t v, int n) {
  fx_set_i64(r->lo, v, n);
  fx_set_i64(r->hi, v, n);
}
/* [+-M*2^e] */
static void iv_set_scaled(iv_t *r, int neg, uint64_t M, int64_t e, int n) {
  limb lo[MAXL], hi[MAXL];
  fx_set_scaled(lo, M, e, n, -1);
  fx_set_scaled(hi, M, e, n, +1);
  if (neg) {
    fx_neg(r->lo, hi, n);
    fx_neg(r->hi, lo, n);
  } else {
    memcpy(r->lo, lo, 8 * (size_t)n);
    memcpy(r->hi, hi, 8 * (size_t)n);
  }
}
static void iv_add(iv_t *r, const iv_t *a, const iv_t *b, int n) {
  fx_add(r->lo, a->lo, b->lo, n);
  fx_add(r->hi, a->hi, b->hi, n);
}
static void iv_sub(iv_t *r, const iv_t *a, const iv_t *b, int n) {
  limb lo[MAXL];
  fx_sub(lo, a->lo, b->hi, n);
  fx_sub(r->hi, a->hi, b->lo, n);
  memcpy(r->lo, lo, 8 * (size_t)n);
}
static void iv_neg(iv_t *r, const iv_t *a, int n) {
  limb lo[MAXL];
  fx_neg(lo, a->hi, n);
  fx_neg(r->hi, a->lo, n);
  memcpy(r->lo, lo, 8 * (size_t)n);
}
static void iv_mul(iv_t *r, const iv_t *a, const iv_t *b, int n) {
  limb lo[MAXL], hi[MAXL];
  int alo = fx_sgn(a->lo, n), ahi = fx_sgn(a->hi, n);
  int blo = fx_sgn(b->lo, n), bhi = fx_sgn(b->hi, n);
  if (alo >= 0 && blo >= 0) {
    fx_mul(lo, a->lo, b->lo, n, -1);
    fx_mul(hi, a->hi, b->hi, n, +1);
  } else if (ahi <= 0 && bhi <= 0) {
    fx_mul(lo, a->hi, b->hi, n, -1);
    fx_mul(hi, a->lo, b->lo, n, +1);
  } else if (alo >= 0 && bhi <= 0) {
    fx_mul(lo, a->hi, b->lo, n, -1);
    fx_mul(hi, a->lo, b->hi, n, +1);
  } else if (ahi <= 0 && blo >= 0) {
    fx_mul(lo, a->lo, b->hi, n, -1);
    fx_mul(hi, a->hi, b->lo, n, +1);
  } else { /* general: min and max over the four corner products */
    const limb *as[2] = {a->lo, a->hi}, *bs[2] = {b->lo, b->hi};
    limb t[MAXL];
    for (int i = 0; i < 4; i++) {
      fx_mul(t, as[i >> 1], bs[i & 1], n, -1);
      if (i == 0 || fx_cmp(t, lo, n) < 0) memcpy(lo, t, 8 * (size_t)n);
      fx_mul(t, as[i >> 1], bs[i & 1], n, +1);
      if (i == 0 || fx_cmp(t, hi, n) > 0) memcpy(hi, t, 8 * (size_t)n);
    }
  }
  memcpy(r->lo, lo, 8 * (size_t)n);
  memcpy(r->hi, hi, 8 * (size_t)n);
}
static void iv_sqr(iv_t *r, const iv_t *a, int n) {
  limb lo[MAXL], hi[MAXL], t[MAXL];
  int slo = fx_sgn(a->lo, n), shi = fx_sgn(a->hi, n);
  if (slo >= 0) {
    fx_mul(lo, a->lo, a->lo, n, -1);
    fx_mul(hi, a->hi, a->hi, n, +1);
  } else if (shi <= 0) {
    fx_mul(lo, a->hi, a->hi, n, -1);
    fx_mul(hi, a->lo, a->lo, n, +1);
  } else {
    memset(lo, 0, 8 * (size_t)n);
    fx_mul(hi, a->lo, a->lo, n, +1);
    fx_mul(t, a->hi, a->hi, n, +1);
    if (fx_cmp(t, hi, n) > 0) memcpy(hi, t, 8 * (size_t)n);
  }
  memcpy(r->lo, lo, 8 * (size_t)n);
  memcpy(r->hi, hi, 8 * (size_t)n);
}
/* 1 / b; fails if b contains 0 */
static void iv_recip(iv_t *r, const iv_t *b, int n) {
  int slo = fx_sgn(b->lo, n), shi = fx_sgn(b->hi, n);
  if (!((slo > 0) || (shi < 0))) {
    g_fail = 1;
    iv_set_i(r, 1, n);
    return;
  }
  limb one[MAXL], lo[MAXL], hi[MAXL];
  fx_set_i64(one, 1, n);
  fx_div(lo, one, b->hi, n, -1);
  fx_div(hi, one, b->lo, n, +1);
  memcpy(r->lo, lo, 8 * (size_t)n);
  memcpy(r->hi, hi, 8 * (size_t)n);
}
static void iv_div(iv_t *r, const iv_t *a, const iv_t *b, int n) {
  iv_t rb;
  iv_recip(&rb, b, n);
  iv_mul(r, a, &rb, n);
}
static void iv_sqrt(iv_t *r, const iv_t *a, int n) {
  if (fx_isneg(a->hi, n)) {
    g_fail = 1;
    iv_set_i(r, 0, n);
    return;
  }
  limb lo[MAXL], hi[MAXL];
  if (fx_isneg(a->lo, n))
    memset(lo, 0, 8 * (size_t)n);
  else
    fx_sqrt(lo, a->lo, n, -1);
  fx_sqrt(hi, a->hi, n, +1);
  memcpy(r->lo, lo, 8 * (size_t)n);
  memcpy(r->hi, hi, 8 * (size_t)n);
}
static void iv_mul_u(iv_t *r, const iv_t *a, uint64_t m, int n) {
  fx_mul_u(r->lo, a->lo, m, n);
  fx_mul_u(r->hi, a->hi, m, n);
}
static void iv_mul_i(iv_t *r, const iv_t *a, int64_t k, int n) {
  if (k >= 0) {
    iv_mul_u(r, a, (uint64_t)k, n);
  } else {
    iv_t t;
    iv_mul_u(&t, a, (uint64_t)(-k), n);
    iv_neg(r, &t, n);
  }
}
static void iv_div_u(iv_t *r, const iv_t *a, uint64_t d, int n) {
  fx_div_u(r->lo, a->lo, d, n, -1);
  fx_div_u(r->hi, a->hi, d, n, +1);
}
static void iv_shr(iv_t *r, const iv_t *a, int64_t k, int n) {
  fx_shr(r->lo, a->lo, k, n, -1);
  fx_shr(r->hi, a->hi, k, n, +1);
}
static void iv_shl(iv_t *r, const iv_t *a, int64_t k, int n) {
  fx_shl(r->lo, a->lo, k, n);
  fx_shl(r->hi, a->hi, k, n);
}
/* max(|lo|, |hi|) */
static void iv_absmax(limb *m, const iv_t *a, int n) {
  limb t[MAXL];
  fx_abs(m, a->lo, n);
  fx_abs(t, a->hi, n);
  if (mag_cmp(t, m, n) > 0) memcpy(m, t, 8 * (size_t)n);
}
/* [lo - w, hi + w] for w >= 0 */
static void iv_widen(iv_t *r, const limb *w, int n) {
  fx_sub(r->lo, r->lo, w, n);
  fx_add(r->hi, r->hi, w, n);
}
/* 1 if |term| <= 2 units in the last place (the series is then truncated) */
static int small_enough(const limb *m, int n) {
  if (m[n - 1]) return 0;
  for (int i = 1; i < n - 1; i++)
    if (m[i]) return 0;
  return m[0] <= 2;
}
/* Widen a truncated series by twice the magnitude of its first omitted term.  All series
   below are used only where the tail after that term is at most the term itself
   (alternating with decreasing terms, or ratio of successive terms <= 1/2). */
static void iv_widen_tail(iv_t *sum, const iv_t *first_omitted, int n) {
  limb m[MAXL];
  iv_absmax(m, first_omitted, n);
  fx_mul_u(m, m, 2, n);
  iv_widen(sum, m, n);
}

/* ===================== constants ===================== */

/* atanh(1/m) = sum_k 1 / ((2k+1) m^(2k+1)), positive terms, ratio <= 1/m^2 */
static void iv_atanh_inv(iv_t *r, uint64_t m, int n) {
  iv_t p, s, t;
  iv_set_i(&p, 1, n);
  iv_div_u(&p, &p, m, n);
  iv_set_i(&s, 0, n);
  for (uint64_t k = 0;; k++) {
    iv_div_u(&t, &p, 2 * k + 1, n);
    limb mg[MAXL];
    iv_absmax(mg, &t, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&s, &t, n);
      break;
    }
    iv_add(&s, &s, &t, n);
    iv_div_u(&p, &p, m, n);
    iv_div_u(&p, &p, m, n);
  }
  *r = s;
}
/* atan(1/m) = sum_k (-1)^k / ((2k+1) m^(2k+1)), alternating, decreasing */
static void iv_atan_inv(iv_t *r, uint64_t m, int n) {
  iv_t p, s, t;
  iv_set_i(&p, 1, n);
  iv_div_u(&p, &p, m, n);
  iv_set_i(&s, 0, n);
  for (uint64_t k = 0;; k++) {
    iv_div_u(&t, &p, 2 * k + 1, n);
    limb mg[MAXL];
    iv_absmax(mg, &t, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&s, &t, n);
      break;
    }
    if (k & 1)
      iv_sub(&s, &s, &t, n);
    else
      iv_add(&s, &s, &t, n);
    iv_div_u(&p, &p, m, n);
    iv_div_u(&p, &p, m, n);
  }
  *r = s;
}

typedef struct {
  iv_t ln2, ln10, pi, pio2, twoopi;
} consts_t;

static consts_t *g_consts[MAXL + 1];
static pthread_mutex_t g_consts_mu = PTHREAD_MUTEX_INITIALIZER;

static void compute_consts(consts_t *c, int n) {
  iv_t t, u;
  /* ln 2 = 2 atanh(1/3) */
  iv_atanh_inv(&t, 3, n);
  iv_mul_u(&c->ln2, &t, 2, n);
  /* ln 10 = 3 ln 2 + ln(5/4),  ln(5/4) = 2 atanh(1/9) */
  iv_atanh_inv(&t, 9, n);
  iv_mul_u(&t, &t, 2, n);
  iv_mul_u(&u, &c->ln2, 3, n);
  iv_add(&c->ln10, &u, &t, n);
  /* pi = 16 atan(1/5) - 4 atan(1/239)  (Machin) */
  iv_atan_inv(&t, 5, n);
  iv_mul_u(&t, &t, 16, n);
  iv_atan_inv(&u, 239, n);
  iv_mul_u(&u, &u, 4, n);
  iv_sub(&c->pi, &t, &u, n);
  iv_shr(&c->pio2, &c->pi, 1, n);
  /* 2/pi */
  iv_recip(&t, &c->pi, n);
  iv_mul_u(&c->twoopi, &t, 2, n);
}

static const consts_t *get_consts(int n) {
  if (n < 2 || n > MAXL) die("bad precision");
  consts_t *c = __atomic_load_n(&g_consts[n], __ATOMIC_ACQUIRE);
  if (c) return c;
  pthread_mutex_lock(&g_consts_mu);
  c = g_consts[n];
  if (!c) {
    c = (consts_t *)malloc(sizeof(consts_t));
    if (!c) die("out of memory");
    compute_consts(c, n);
    __atomic_store_n(&g_consts[n], c, __ATOMIC_RELEASE);
  }
  pthread_mutex_unlock(&g_consts_mu);
  return c;
}

/* ===================== series kernels ===================== */

/* e^r for |r| <= 1/2: e^r = (e^(r/2^8))^(2^8), Taylor series for the inner value */
static void iv_exp_small(iv_t *res, const iv_t *r, int n) {
  const int s = 8;
  iv_t y, sum, term;
  iv_shr(&y, r, s, n);
  iv_set_i(&sum, 1, n);
  iv_set_i(&term, 1, n);
  for (uint64_t k = 1;; k++) {
    iv_mul(&term, &term, &y, n);
    iv_div_u(&term, &term, k, n);
    limb mg[MAXL];
    iv_absmax(mg, &term, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&sum, &term, n);
      break;
    }
    iv_add(&sum, &sum, &term, n);
  }
  for (int i = 0; i < s; i++) iv_sqr(&sum, &sum, n);
  *res = sum;
}

/* E1(x) = (e^x - 1)/x = sum_j x^j/(j+1)!  for |x| <= 2^-10 */
static void iv_expm1_over_x(iv_t *res, const iv_t *x, int n) {
  iv_t sum, term;
  iv_set_i(&sum, 1, n);
  iv_set_i(&term, 1, n);
  for (uint64_t j = 1;; j++) {
    iv_mul(&term, &term, x, n);
    iv_div_u(&term, &term, j + 1, n);
    limb mg[MAXL];
    iv_absmax(mg, &term, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&sum, &term, n);
      break;
    }
    iv_add(&sum, &sum, &term, n);
  }
  *res = sum;
}

/* atanh(u) = sum u^(2k+1)/(2k+1)  for |u| <= 1/5 */
static void iv_atanh_series(iv_t *res, const iv_t *u, int n) {
  iv_t u2, p, sum, t;
  iv_sqr(&u2, u, n);
  p = *u;
  iv_set_i(&sum, 0, n);
  for (uint64_t k = 0;; k++) {
    iv_div_u(&t, &p, 2 * k + 1, n);
    limb mg[MAXL];
    iv_absmax(mg, &t, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&sum, &t, n);
      break;
    }
    iv_add(&sum, &sum, &t, n);
    iv_mul(&p, &p, &u2, n);
  }
  *res = sum;
}

/* sin and cos of r for |r| <= 1: series at r/16, then four doublings */
static void iv_sincos_small(iv_t *s_out, iv_t *c_out, const iv_t *r, int n) {
  iv_t y, y2, s, c, term, t;
  limb mg[MAXL];
  iv_shr(&y, r, 4, n);
  iv_sqr(&y2, &y, n);
  /* sin y = sum (-1)^k y^(2k+1)/(2k+1)! */
  term = y;
  s = y;
  for (uint64_t k = 1;; k++) {
    iv_mul(&term, &term, &y2, n);
    iv_div_u(&term, &term, (2 * k) * (2 * k + 1), n);
    iv_absmax(mg, &term, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&s, &term, n);
      break;
    }
    if (k & 1)
      iv_sub(&s, &s, &term, n);
    else
      iv_add(&s, &s, &term, n);
  }
  /* cos y = sum (-1)^k y^(2k)/(2k)! */
  iv_set_i(&term, 1, n);
  iv_set_i(&c, 1, n);
  for (uint64_t k = 1;; k++) {
    iv_mul(&term, &term, &y2, n);
    iv_div_u(&term, &term, (2 * k - 1) * (2 * k), n);
    iv_absmax(mg, &term, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&c, &term, n);
      break;
    }
    if (k & 1)
      iv_sub(&c, &c, &term, n);
    else
      iv_add(&c, &c, &term, n);
  }
  /* sin 2a = 2 sin a cos a ; cos 2a = cos^2 a - sin^2 a */
  for (int i = 0; i < 4; i++) {
    iv_t s2, c2;
    iv_mul(&t, &s, &c, n);
    iv_mul_u(&s2, &t, 2, n);
    iv_sqr(&c2, &c, n);
    iv_sqr(&t, &s, n);
    iv_sub(&c, &c2, &t, n);
    s = s2;
  }
  *s_out = s;
  *c_out = c;
}

/* atan(w) = sum (-1)^k w^(2k+1)/(2k+1) for |w| <= 1/8 */
static void iv_atan_series(iv_t *res, const iv_t *w, int n) {
  iv_t w2, p, sum, t;
  iv_sqr(&w2, w, n);
  p = *w;
  iv_set_i(&sum, 0, n);
  for (uint64_t k = 0;; k++) {
    iv_div_u(&t, &p, 2 * k + 1, n);
    limb mg[MAXL];
    iv_absmax(mg, &t, n);
    if (small_enough(mg, n)) {
      iv_widen_tail(&sum, &t, n);
      break;
    }
    if (k & 1)
      iv_sub(&sum, &sum, &t, n);
    else
      iv_add(&sum, &sum, &t, n);
    iv_mul(&p, &p, &w2, n);
  }
  *res = sum;
}

/* atan(z) for any real interval z.  |z| <= 1: atan z = 2 atan(z / (1 + sqrt(1 + z^2)))
   applied three times, then the series.  |z| > 1: atan z = sign(z) pi/2 - atan(1/z). */
static void iv_atan(iv_t *res, const iv_t *z, int n) {
  limb one[MAXL], mone[MAXL];
  fx_set_i64(one, 1, n);
  fx_set_i64(mone, -1, n);
  int pos = fx_cmp(z->lo, one, n) > 0, negb = fx_cmp(z->hi, mone, n) < 0;
  if (pos || negb) {
    iv_t rz, a;
    iv_recip(&rz, z, n);
    iv_atan(&a, &rz, n);
    const consts_t *C = get_consts(n);
    if (pos)
      iv_sub(res, &C->pio2, &a, n);
    else {
      iv_t npio2;
      iv_neg(&npio2, &C->pio2, n);
      iv_sub(res, &npio2, &a, n);
    }
    return;
  }
  iv_t w = *z, t, one_iv;
  iv_set_i(&one_iv, 1, n);
  for (int i = 0; i < 3; i++) {
    iv_sqr(&t, &w, n);
    iv_add(&t, &t, &one_iv, n);
    iv_sqrt(&t, &t, n);
    iv_add(&t, &t, &one_iv, n);
    iv_div(&w, &w, &t, n);
  }
  iv_atan_series(&t, &w, n);
  iv_shl(res, &t, 3, n);
}

/* ===================== decoding, rounding ===================== */

enum { CL_ZERO, CL_FINITE, CL_INF, CL_NAN };
typedef struct {
  int cls, neg;
  uint64_t M; /* significand as an integer */
  int64_t e;  /* |x| = M * 2^e */
} dec_t;

static dec_t dec32(uint32_t b) {
  dec_t d;
  d.neg = (int)(b >> 31);
  uint32_t be = (b >> 23) & 0xFF, f = b & 0x7FFFFF;
  d.M = 0;
  d.e = 0;
  if (be == 0xFF) {
    d.cls = f ? CL_NAN : CL_INF;
  } else if (be == 0) {
    d.cls = f ? CL_FINITE : CL_ZERO;
    d.M = f;
    d.e = -149;
  } else {
    d.cls = CL_FINITE;
    d.M = f | 0x800000u;
    d.e = (int64_t)be - 150;
  }
  return d;
}
static dec_t dec64(uint64_t b) {
  dec_t d;
  d.neg = (int)(b >> 63);
  uint64_t be = (b >> 52) & 0x7FF, f = b & 0xFFFFFFFFFFFFFull;
  d.M = 0;
  d.e = 0;
  if (be == 0x7FF) {
    d.cls = f ? CL_NAN : CL_INF;
  } else if (be == 0) {
    d.cls = f ? CL_FINITE : CL_ZERO;
    d.M = f;
    d.e = -1074;
  } else {
    d.cls = CL_FINITE;
    d.M = f | (1ull << 52);
    d.e = (int64_t)be - 1075;
  }
  return d;
}
/* approximate |x| as a double, only for choosing reduction integers and branches */
static double approx(const dec_t *x) { return ldexp((double)x->M, (int)x->e); }
/* is |x| an integer? */
static int is_integer(const dec_t *x) {
  if (x->e >= 0) return 1;
  if (x->e <= -64) return x->M == 0;
  return (x->M & ((1ull << (-x->e)) - 1)) == 0;
}

typedef struct {
  int p, emin, emax, bias, w; /* precision, exponent range, bias, width */
} fmt_t;
static const fmt_t FMT32 = {24, -126, 127, 127, 32};
static const fmt_t FMT64 = {53, -1022, 1023, 1023, 64};
static const fmt_t FMT16 = {11, -14, 15, 15, 16};      /* IEEE binary16 */
static const fmt_t FMTB16 = {8, -126, 127, 127, 16};   /* bfloat16: binary32's range, 8 bits */

/* Decode a bit pattern of the 16-bit formats (the same rules as dec32 / dec64). */
static dec_t dec_fmt(uint64_t b, const fmt_t *f) {
  dec_t d;
  const int ew = f->w - f->p;  /* exponent field width */
  d.neg = (int)((b >> (f->w - 1)) & 1);
  uint64_t be = (b >> (f->p - 1)) & ((1ull << ew) - 1), fr = b & ((1ull << (f->p - 1)) - 1);
  d.M = 0;
  d.e = 0;
  if (be == (1ull << ew) - 1) {
    d.cls = fr ? CL_NAN : CL_INF;
  } else if (be == 0) {
    d.cls = fr ? CL_FINITE : CL_ZERO;
    d.M = fr;
    d.e = f->emin - (f->p - 1);
  } else {
    d.cls = CL_FINITE;
    d.M = fr | (1ull << (f->p - 1));
    d.e = (int64_t)be - f->bias - (f->p - 1);
  }
  return d;
}

static uint64_t inf_bits(const fmt_t *f) { return (uint64_t)(2 * f->bias + 1) << (f->p - 1); }
static uint64_t sign_bit(const fmt_t *f) { return 1ull << (f->w - 1); }
static uint64_t one_bits(const fmt_t *f) { return (uint64_t)f->bias << (f->p - 1); }
static uint64_t qnan_bits(const fmt_t *f) { return inf_bits(f) | (1ull << (f->p - 2)); }

/* Round the exact value a * 2^(E - F) to the format: mode ORC_RN to nearest with ties to
   even, ORC_RD toward -inf, ORC_RU toward +inf, ORC_RZ toward zero (IEEE 754 Sec. 4.3).
   A directed mode moves the magnitude up ("away") when it points away from zero. */
static uint64_t round_fixed(const limb *a, int n, int64_t E, const fmt_t *f, int mode) {
  limb m[MAXL];
  int neg = fx_abs(m, a, n);
  int b = mag_bitlen(m, n);
  if (b == 0) return 0;
  uint64_t sbit = neg ? sign_bit(f) : 0;
  int away = (mode == ORC_RU && !neg) || (mode == ORC_RD && neg);
  int64_t F = FB(n);
  int64_t ex = (int64_t)b - 1 + E - F; /* value in [2^ex, 2^(ex+1)) */
  if (ex > f->emax) return sbit | ((mode == ORC_RN || away) ? inf_bits(f) : inf_bits(f) - 1);
  int64_t qe = (ex < f->emin ? f->emin : ex) - (f->p - 1); /* exponent of the last place */
  int64_t shift = E - F - qe;                              /* significand = m * 2^shift */
  uint64_t sig;
  if (shift >= 0) {
    sig = m[0] << shift; /* b + shift <= p <= 53 */
  } else {
    int64_t k = -shift;
    sig = 0;
    for (int i = 0; i < f->p + 1; i++) sig |= (uint64_t)mag_bit(m, n, k + i) << i;
    int rb = mag_bit(m, n, k - 1);
    int st = mag_any_below(m, n, k - 1);
    if (mode == ORC_RN) {
      if (rb && (st || (sig & 1))) sig++;
    } else if (away && (rb || st)) {
      sig++;
    }
  }
  uint64_t bits;
  if (ex < f->emin)
    bits = sig;
  else
    bits = ((uint64_t)(ex + f->bias) << (f->p - 1)) + sig - (1ull << (f->p - 1));
  if (bits >= inf_bits(f)) bits = inf_bits(f);
  return sbit | bits;
}

/* ===================== function evaluators ===================== */

enum {
  K_EXP, K_EXP2, K_EXP10, K_EXPM1, K_LOG, K_LOG2, K_LOG10, K_LOG1P, K_SIN, K_COS, K_TAN,
  K_ASIN, K_ACOS, K_ATAN, K_SINH, K_COSH, K_TANH, K_RSQRT
};

typedef struct {
  iv_t v;
  int64_t E; /* f(x) in v * 2^E */
} res_t;

static const double LN2_APPROX = 0.6931471805599453;

/* e^x for the exact interval xv (|x| < 1000), as e^(x - k ln2) * 2^k */
static void ev_exp_at(res_t *R, const iv_t *xv, double xd, int n) {
  const consts_t *C = get_consts(n);
  int64_t k = llround(xd / LN2_APPROX);
  iv_t t, r;
  iv_mul_i(&t, &C->ln2, k, n);
  iv_sub(&r, xv, &t, n);
  iv_exp_small(&R->v, &r, n);
  R->E = k;
}

static void ev_exp(res_t *R, const dec_t *x, int n) {
  iv_t xv;
  iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  ev_exp_at(R, &xv, x->neg ? -approx(x) : approx(x), n);
}

static void ev_exp2(res_t *R, const dec_t *x, int n) {
  double xd = x->neg ? -approx(x) : approx(x);
  if (is_integer(x)) { /* 2^k exactly */
    iv_set_i(&R->v, 1, n);
    R->E = (int64_t)xd;
    return;
  }
  const consts_t *C = get_consts(n);
  int64_t k = llround(xd);
  iv_t xv, f, r;
  iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  iv_t kv;
  iv_set_i(&kv, k, n);
  iv_sub(&f, &xv, &kv, n); /* 2^x = 2^k * e^((x-k) ln2) */
  iv_mul(&r, &f, &C->ln2, n);
  iv_exp_small(&R->v, &r, n);
  R->E = k;
}

static void ev_exp10(res_t *R, const dec_t *x, int n) {
  const consts_t *C = get_consts(n);
  double xd = x->neg ? -approx(x) : approx(x);
  int64_t k = llround(xd * 3.321928094887362);
  iv_t xv, y, t, r;
  iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  iv_mul(&y, &xv, &C->ln10, n); /* 10^x = e^(x ln10) = 2^k e^(x ln10 - k ln2) */
  iv_mul_i(&t, &C->ln2, k, n);
  iv_sub(&r, &y, &t, n);
  iv_exp_small(&R->v, &r, n);
  R->E = k;
}

/* scaled form for tiny |x|: f(x) = x * S, returned as (M * S) * 2^e with sign */
static void scaled_result(res_t *R, const dec_t *x, const iv_t *S, int n) {
  iv_mul_u(&R->v, S, x->M, n);
  if (x->neg) iv_neg(&R->v, &R->v, n);
  R->E = x->e;
}
static int is_tiny(const dec_t *x) { return approx(x) < 0.0009765625; /* 2^-10 */ }

static void ev_expm1(res_t *R, const dec_t *x, int n) {
  iv_t xv;
  iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  if (is_tiny(x)) {
    iv_t S;
    iv_expm1_over_x(&S, &xv, n);
    scaled_result(R, x, &S, n);
    return;
  }
  /* e^x - 1 = 2^k (e^r - 2^-k) */
  res_t ex;
  ev_exp_at(&ex, &xv, x->neg ? -approx(x) : approx(x), n);
  int64_t k = ex.E;
  iv_t p;
  if (k >= 0) {
    iv_set_i(&p, 1, n);
    iv_shr(&p, &p, k, n);
  } else {
    iv_set_i(&p, (int64_t)1 << (-k), n);
  }
  iv_sub(&R->v, &ex.v, &p, n);
  R->E = k;
}

/* log of the exact positive fixed-point interval-free value y (y.lo == y.hi):
   y = m 2^K with m in [3/4, 3/2); log y = K ln2 + 2 atanh((m-1)/(m+1)).
   Returns K and the atanh term separately (A = 2 atanh(u)). */
static void log_parts(const limb *y, int n, int64_t *Kout, iv_t *A) {
  int b = mag_bitlen(y, n);
  int64_t K = (int64_t)b - 1 - FB(n); /* y in [2^K, 2^(K+1)) */
  limb m[MAXL];
  if (K >= 0)
    mag_shr(m, y, n, K); /* exact by construction of callers */
  else
    mag_shl(m, y, n, -K);
  /* m in [1,2); move to [3/4, 3/2) */
  limb three_half[MAXL];
  fx_set_i64(three_half, 3, n);
  mag_shr(three_half, three_half, n, 1);
  if (mag_cmp(m, three_half, n) >= 0) {
    mag_shr(m, m, n, 1); /* exact: m has at most 54 significant bits here */
    K += 1;
  }
  iv_t mv, one, num, den, u;
  memcpy(mv.lo, m, 8 * (size_t)n);
  memcpy(mv.hi, m, 8 * (size_t)n);
  iv_set_i(&one, 1, n);
  iv_sub(&num, &mv, &one, n);
  iv_add(&den, &mv, &one, n);
  iv_div(&u, &num, &den, n);
  iv_atanh_series(A, &u, n);
  iv_mul_u(A, A, 2, n);
  *Kout = K;
}

static void ev_log_any(res_t *R, const dec_t *x, int n, int kind) {
  const consts_t *C = get_consts(n);
  /* x = M 2^e = (M / 2^(bl-1)) 2^(e+bl-1), the first factor in [1,2) and exact */
  int bl = 64 - __builtin_clzll(x->M);
  limb mm[MAXL];
  fx_set_scaled(mm, x->M, -(int64_t)(bl - 1), n, 0);
  int64_t K1;
  iv_t A, t;
  log_parts(mm, n, &K1, &A);
  int64_t K = x->e + bl - 1 + K1;
  switch (kind) {
    case K_LOG:
      iv_mul_i(&t, &C->ln2, K, n);
      iv_add(&R->v, &t, &A, n);
      break;
    case K_LOG2: {
      iv_t q, kv;
      iv_div(&q, &A, &C->ln2, n);
      iv_set_i(&kv, K, n);
      iv_add(&R->v, &kv, &q, n);
      break;
    }
    default: { /* K_LOG10 */
      iv_mul_i(&t, &C->ln2, K, n);
      iv_add(&t, &t, &A, n);
      iv_div(&R->v, &t, &C->ln10, n);
      break;
    }
  }
  R->E = 0;
}

static void ev_log1p(res_t *R, const dec_t *x, int n) {
  const consts_t *C = get_consts(n);
  iv_t xv, one;
  iv_set_i(&one, 1, n);
  double xd = x->neg ? -approx(x) : approx(x);
  if (xd < 1.0) iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  if (is_tiny(x)) {
    /* log1p(x) = 2 atanh(u), u = x/(2+x);  = x * (2/(2+x)) * sum u^(2k)/(2k+1) */
    iv_t two, den, u, u2, p, sum, t, S;
    iv_set_i(&two, 2, n);
    iv_add(&den, &two, &xv, n);
    iv_div(&u, &xv, &den, n);
    iv_sqr(&u2, &u, n);
    iv_set_i(&p, 1, n);
    iv_set_i(&sum, 0, n);
    for (uint64_t k = 0;; k++) {
      iv_div_u(&t, &p, 2 * k + 1, n);
      limb mg[MAXL];
      iv_absmax(mg, &t, n);
      if (small_enough(mg, n)) {
        iv_widen_tail(&sum, &t, n);
        break;
      }
      iv_add(&sum, &sum, &t, n);
      iv_mul(&p, &p, &u2, n);
    }
    iv_div(&S, &two, &den, n);
    iv_mul(&S, &S, &sum, n);
    scaled_result(R, x, &S, n);
    return;
  }
  if (xd >= 1.0) {
    /* log1p(x) = log(x) + 2 atanh(w), w = 1/(2x+1) = 2^-(e+1) / (M + 2^-(e+1)) */
    res_t L;
    ev_log_any(&L, x, n, K_LOG);
    iv_t h, d, w, A, mv;
    iv_set_i(&h, 1, n);
    if (x->e + 1 >= 0)
      iv_shr(&h, &h, x->e + 1, n);
    else
      iv_shl(&h, &h, -(x->e + 1), n);
    iv_set_i(&mv, (int64_t)x->M, n);
    iv_add(&d, &mv, &h, n);
    iv_div(&w, &h, &d, n);
    iv_atanh_series(&A, &w, n);
    iv_mul_u(&A, &A, 2, n);
    iv_add(&R->v, &L.v, &A, n);
    R->E = 0;
    return;
  }
  /* 2^-10 <= |x| < 1: y = 1 + x exact at this precision (x has >= -34 exponent) */
  iv_t y;
  iv_add(&y, &one, &xv, n);
  if (fx_cmp(y.lo, y.hi, n) != 0) die("log1p: 1+x not exact");
  int64_t K;
  iv_t A, t;
  log_parts(y.lo, n, &K, &A);
  iv_mul_i(&t, &C->ln2, K, n);
  iv_add(&R->v, &t, &A, n);
  R->E = 0;
}

/* Reduction for |x| >= 3/4: |x| * 2/pi = N + f with N integer, |f| <= 1/2 (+tiny);
   returns r = f * pi/2 (interval) and N mod 4. */
static void trig_reduce(iv_t *r, int *quadrant, const dec_t *x, int n) {
  const int n3 = n + 5; /* F + 320 fraction bits: covers e <= 104 plus guard bits */
  const consts_t *C3 = get_consts(n3);
  iv_t c;
  if (x->e >= 0) {
    /* c = (2^e * 2/pi) mod 4 : shift the lower end, keep 2 integer bits, add the width */
    limb lo[MAXL], w[MAXL] = {0};
    memcpy(lo, C3->twoopi.lo, 8 * (size_t)n3);
    fx_sub(w, C3->twoopi.hi, C3->twoopi.lo, n3);
    limb wide[2 * MAXL];
    /* shift in a double-width buffer so that no bits are lost before the mod */
    memset(wide, 0, sizeof(wide));
    memcpy(wide, lo, 8 * (size_t)n3);
    mag_shl(wide, wide, 2 * n3, x->e);
    memcpy(lo, wide, 8 * (size_t)n3);
    lo[n3 - 1] &= 3; /* integer part mod 4 */
    mag_shl(w, w, n3, x->e);
    memcpy(c.lo, lo, 8 * (size_t)n3);
    fx_add(c.hi, lo, w, n3);
  } else {
    iv_shr(&c, &C3->twoopi, -x->e, n3);
  }
  iv_t u;
  iv_mul_u(&u, &c, x->M, n3); /* |x| * 2/pi  mod 4 (M times the reduced constant) */
  /* N = nearest integer to the lower end */
  int64_t ip = (int64_t)u.lo[n3 - 1];
  int half = (int)(u.lo[n3 - 2] >> 63);
  int64_t N = ip + half;
  iv_t nv, f;
  iv_set_i(&nv, N, n3);
  iv_sub(&f, &u, &nv, n3);
  /* drop to n limbs */
  iv_t fn;
  fx_shr(fn.lo, f.lo, 64 * 5, n3, -1);
  fx_shr(fn.hi, f.hi, 64 * 5, n3, +1);
  /* fn now has F fraction bits in the low n limbs; sign-extend into n limbs */
  iv_t fr;
  memcpy(fr.lo, fn.lo, 8 * (size_t)n);
  memcpy(fr.hi, fn.hi, 8 * (size_t)n);
  const consts_t *C = get_consts(n);
  iv_mul(r, &fr, &C->pio2, n);
  *quadrant = (int)(N & 3);
}

/* sin, cos or tan of x (finite, nonzero) */
static void ev_trig(res_t *R, const dec_t *x, int n, int kind) {
  double ax = approx(x);
  if (ax < 0.0009765625) {
    iv_t xv, x2, term, S, C;
    limb mg[MAXL];
    iv_set_scaled(&xv, 0, x->M, x->e, n);
    iv_sqr(&x2, &xv, n);
    if (kind == K_SIN || kind == K_TAN) {
      iv_set_i(&term, 1, n);
      iv_set_i(&S, 1, n);
      for (uint64_t k = 1;; k++) {
        iv_mul(&term, &term, &x2, n);
        iv_div_u(&term, &term, (2 * k) * (2 * k + 1), n);
        iv_absmax(mg, &term, n);
        if (small_enough(mg, n)) {
          iv_widen_tail(&S, &term, n);
          break;
        }
        if (k & 1)
          iv_sub(&S, &S, &term, n);
        else
          iv_add(&S, &S, &term, n);
      }
    }
    if (kind == K_COS || kind == K_TAN) {
      iv_set_i(&term, 1, n);
      iv_set_i(&C, 1, n);
      for (uint64_t k = 1;; k++) {
        iv_mul(&term, &term, &x2, n);
        iv_div_u(&term, &term, (2 * k - 1) * (2 * k), n);
        iv_absmax(mg, &term, n);
        if (small_enough(mg, n)) {
          iv_widen_tail(&C, &term, n);
          break;
        }
        if (k & 1)
          iv_sub(&C, &C, &term, n);
        else
          iv_add(&C, &C, &term, n);
      }
    }
    if (kind == K_COS) {
      R->v = C;
      R->E = 0;
      return;
    }
    if (kind == K_TAN) iv_div(&S, &S, &C, n);
    scaled_result(R, x, &S, n);
    return;
  }
  iv_t r, s, c;
  int q = 0;
  if (ax < 0.75) {
    iv_set_scaled(&r, 0, x->M, x->e, n);
  } else {
    trig_reduce(&r, &q, x, n);
  }
  iv_sincos_small(&s, &c, &r, n);
  iv_t out;
  if (kind == K_SIN) {
    switch (q) {
      case 0: out = s; break;
      case 1: out = c; break;
      case 2: iv_neg(&out, &s, n); break;
      default: iv_neg(&out, &c, n); break;
    }
    if (x->neg) iv_neg(&out, &out, n);
  } else if (kind == K_COS) {
    switch (q) {
      case 0: out = c; break;
      case 1: iv_neg(&out, &s, n); break;
      case 2: iv_neg(&out, &c, n); break;
      default: out = s; break;
    }
  } else {
    if (q & 1) {
      iv_div(&out, &c, &s, n);
      iv_neg(&out, &out, n);
    } else {
      iv_div(&out, &s, &c, n);
    }
    if (x->neg) iv_neg(&out, &out, n);
  }
  R->v = out;
  R->E = 0;
}

static void ev_atan(res_t *R, const dec_t *x, int n) {
  if (is_tiny(x)) { /* atan x = x * sum (-1)^k x^(2k)/(2k+1) */
    iv_t xv, x2, p, S, t;
    iv_set_scaled(&xv, 0, x->M, x->e, n);
    iv_sqr(&x2, &xv, n);
    iv_set_i(&p, 1, n);
    iv_set_i(&S, 0, n);
    for (uint64_t k = 0;; k++) {
      iv_div_u(&t, &p, 2 * k + 1, n);
      limb mg[MAXL];
      iv_absmax(mg, &t, n);
      if (small_enough(mg, n)) {
        iv_widen_tail(&S, &t, n);
        break;
      }
      if (k & 1)
        iv_sub(&S, &S, &t, n);
      else
        iv_add(&S, &S, &t, n);
      iv_mul(&p, &p, &x2, n);
    }
    scaled_result(R, x, &S, n);
    return;
  }
  iv_t xv;
  if (approx(x) >= 1073741824.0) { /* |x| >= 2^30: atan x = pi/2 - atan(1/x), 1/x = 2^-e / M */
    iv_t m, rz, a;
    iv_set_i(&m, (int64_t)x->M, n);
    iv_recip(&rz, &m, n);
    iv_shr(&rz, &rz, x->e, n); /* 1/x = (1/M) 2^-e */
    iv_atan_series(&a, &rz, n);
    const consts_t *C = get_consts(n);
    iv_sub(&R->v, &C->pio2, &a, n);
  } else {
    iv_set_scaled(&xv, 0, x->M, x->e, n);
    iv_atan(&R->v, &xv, n);
  }
  if (x->neg) iv_neg(&R->v, &R->v, n);
  R->E = 0;
}

static void ev_asin(res_t *R, const dec_t *x, int n) {
  iv_t xv, x2;
  iv_set_scaled(&xv, 0, x->M, x->e, n);
  if (is_tiny(x)) {
    /* asin x = x * sum c_k x^(2k), c_0 = 1, c_(k+1) = c_k (2k+1)^2 / ((2k+2)(2k+3)) */
    iv_t term, S;
    limb mg[MAXL];
    iv_sqr(&x2, &xv, n);
    iv_set_i(&term, 1, n);
    iv_set_i(&S, 1, n);
    for (uint64_t k = 0;; k++) {
      iv_mul(&term, &term, &x2, n);
      iv_mul_u(&term, &term, (2 * k + 1) * (2 * k + 1), n);
      iv_div_u(&term, &term, (2 * k + 2) * (2 * k + 3), n);
      iv_absmax(mg, &term, n);
      if (small_enough(mg, n)) {
        iv_widen_tail(&S, &term, n);
        break;
      }
      iv_add(&S, &S, &term, n);
    }
    scaled_result(R, x, &S, n);
    return;
  }
  /* asin x = 2 atan(x / (1 + sqrt(1 - x^2))), |x| < 1 */
  iv_t one, t, w, a;
  iv_set_i(&one, 1, n);
  iv_sqr(&x2, &xv, n);
  iv_sub(&t, &one, &x2, n);
  iv_sqrt(&t, &t, n);
  iv_add(&t, &t, &one, n);
  iv_div(&w, &xv, &t, n);
  iv_atan(&a, &w, n);
  iv_mul_u(&R->v, &a, 2, n);
  if (x->neg) iv_neg(&R->v, &R->v, n);
  R->E = 0;
}

static void ev_acos(res_t *R, const dec_t *x, int n) {
  /* acos x = 2 atan(sqrt((1 - x)/(1 + x))), -1 < x <= 1 */
  iv_t xv, one, a, b, q, s, t;
  iv_set_scaled(&xv, x->neg, x->M, x->e, n);
  iv_set_i(&one, 1, n);
  iv_sub(&a, &one, &xv, n);
  iv_add(&b, &one, &xv, n);
  iv_div(&q, &a, &b, n);
  iv_sqrt(&s, &q, n);
  iv_atan(&t, &s, n);
  iv_mul_u(&R->v, &t, 2, n);
  R->E = 0;
}

static void ev_sinh_cosh(res_t *R, const dec_t *x, int n, int kind) {
  if (kind == K_SINH && is_tiny(x)) { /* sinh x = x sum x^(2k)/(2k+1)! */
    iv_t xv, x2, term, S;
    limb mg[MAXL];
    iv_set_scaled(&xv, 0, x->M, x->e, n);
    iv_sqr(&x2, &xv, n);
    iv_set_i(&term, 1, n);
    iv_set_i(&S, 1, n);
    for (uint64_t k = 1;; k++) {
      iv_mul(&term, &term, &x2, n);
      iv_div_u(&term, &term, (2 * k) * (2 * k + 1), n);
      iv_absmax(mg, &term, n);
      if (small_enough(mg, n)) {
        iv_widen_tail(&S, &term, n);
        break;
      }
      iv_add(&S, &S, &term, n);
    }
    scaled_result(R, x, &S, n);
    return;
  }
  /* |x| = k ln2 + r:  sinh|x| = 2^(k-1) (e^r - e^-r 2^-2k), cosh|x| = 2^(k-1)(e^r + e^-r 2^-2k) */
  iv_t xv;
  iv_set_scaled(&xv, 0, x->M, x->e, n);
  res_t ex;
  ev_exp_at(&ex, &xv, approx(x), n);
  int64_t k = ex.E;
  iv_t er = ex.v, emr, t;
  iv_recip(&emr, &er, n);
  if (k >= 0)
    iv_shr(&t, &emr, 2 * k, n);
  else
    iv_shl(&t, &emr, -2 * k, n);
  if (kind == K_SINH) {
    iv_sub(&R->v, &er, &t, n);
    if (x->neg) iv_neg(&R->v, &R->v, n);
  } else {
    iv_add(&R->v, &er, &t, n);
  }
  R->E = k - 1;
}

static void ev_tanh(res_t *R, const dec_t *x, int n) {
  iv_t xv, one;
  iv_set_i(&one, 1, n);
  iv_set_scaled(&xv, 0, x->M, x->e, n);
  if (is_tiny(x)) {
    /* tanh x = x E1(2x) / (1 + x E1(2x)) */
    iv_t x2v, E1, d, S;
    iv_mul_u(&x2v, &xv, 2, n);
    iv_expm1_over_x(&E1, &x2v, n);
    iv_mul(&d, &xv, &E1, n);
    iv_add(&d, &d, &one, n);
    iv_div(&S, &E1, &d, n);
    scaled_result(R, x, &S, n);
    return;
  }
  /* tanh a = 1 - 2/(e^(2a) + 1) = 1 - 2^(1-k) / (e^r + 2^-k), e^(2a) = 2^k e^r */
  iv_t x2v;
  iv_mul_u(&x2v, &xv, 2, n);
  res_t ex;
  ev_exp_at(&ex, &x2v, 2.0 * approx(x), n);
  int64_t k = ex.E;
  iv_t p, d, q, t;
  iv_set_i(&p, 1, n);
  if (k >= 0)
    iv_shr(&p, &p, k, n);
  else
    iv_shl(&p, &p, -k, n);
  iv_add(&d, &ex.v, &p, n);
  iv_recip(&q, &d, n);
  if (1 - k >= 0)
    iv_shl(&t, &q, 1 - k, n);
  else
    iv_shr(&t, &q, k - 1, n);
  iv_sub(&R->v, &one, &t, n);
  if (x->neg) iv_neg(&R->v, &R->v, n);
  R->E = 0;
}

static void ev_rsqrt(res_t *R, const dec_t *x, int n) {
  /* x = M 2^e with e made even: x^(-1/2) = 2^(-e/2) / sqrt(M) */
  uint64_t M = x->M;
  int64_t e = x->e;
  if (e & 1) {
    M <<= 1;
    e -= 1;
  }
  iv_t m, s;
  iv_set_i(&m, (int64_t)M, n);
  iv_sqrt(&s, &m, n);
  iv_recip(&R->v, &s, n);
  R->E = -e / 2;
}

/* ===================== specials and the Ziv loop ===================== */

/* Handles NaN, infinities, zeros, out-of-domain inputs and saturated ranges.
   Returns 1 and sets *out if the result is decided here. */
/* The rounding, in mode, of a value beyond the largest finite number (huge) or of a
   nonzero value below half the smallest subnormal (tiny), of the given sign. */
static uint64_t rnd_huge(int neg, const fmt_t *f, int mode) {
  int away = (mode == ORC_RU && !neg) || (mode == ORC_RD && neg);
  return (neg ? sign_bit(f) : 0) | ((mode == ORC_RN || away) ? inf_bits(f) : inf_bits(f) - 1);
}
static uint64_t rnd_tiny(int neg, const fmt_t *f, int mode) {
  int away = (mode == ORC_RU && !neg) || (mode == ORC_RD && neg);
  return (neg ? sign_bit(f) : 0) | (away ? 1 : 0);
}
/* The rounding, in mode, of a value strictly between 1 - 2^-p and 1 in magnitude (sign
   neg): 1 to nearest or away from zero, else the largest number below 1. */
static uint64_t rnd_below_one(int neg, const fmt_t *f, int mode) {
  int away = (mode == ORC_RU && !neg) || (mode == ORC_RD && neg);
  return (neg ? sign_bit(f) : 0) | ((mode == ORC_RN || away) ? one_bits(f) : one_bits(f) - 1);
}

static int special(int kind, const dec_t *x, const fmt_t *f, uint64_t xbits, uint64_t *out, int mode) {
  const uint64_t INF = inf_bits(f), SB = sign_bit(f), ONE = one_bits(f), QN = qnan_bits(f);
  if (x->cls == CL_NAN) {
    *out = xbits | (1ull << (f->p - 2));
    return 1;
  }
  const uint64_t sgn = x->neg ? SB : 0;
  double ax = approx(x);
  switch (kind) {
    case K_EXP: case K_EXP2: case K_EXP10: {
      if (x->cls == CL_ZERO) { *out = ONE; return 1; }
      if (x->cls == CL_INF) { *out = x->neg ? 0 : INF; return 1; }
      /* saturation outside the finite-result range of the format, with 8 binades to
         spare: |x| log2(b) >= max(emax + 1, p - emin) + 8 gives b^x >= 2^(emax + 9)
         (overflow) or b^x <= 2^(emin - p - 8) (below half the smallest subnormal); the
         boundary band is left to the Ziv loop */
      double lim = (double)(f->emax + 1 > f->p - f->emin ? f->emax + 1 : f->p - f->emin) + 8.0;
      double hi = kind == K_EXP2 ? lim : (kind == K_EXP ? lim * LN2_APPROX : lim * 0.30102999566398120);
      if (ax >= hi) { *out = x->neg ? rnd_tiny(0, f, mode) : rnd_huge(0, f, mode); return 1; }
      return 0;
    }
    case K_EXPM1:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF) { *out = x->neg ? (SB | ONE) : INF; return 1; }
      /* e^x >= 2^(emax + 3): overflow; x <= -(p + 4) ln 2: -1 + e^x with 0 < e^x < 2^-(p+4) */
      if (!x->neg && ax >= (double)(f->emax + 3) * LN2_APPROX) { *out = rnd_huge(0, f, mode); return 1; }
      if (x->neg && ax >= (double)(f->p + 4) * LN2_APPROX) { *out = rnd_below_one(1, f, mode); return 1; }
      return 0;
    case K_LOG: case K_LOG2: case K_LOG10:
      if (x->cls == CL_ZERO) { *out = SB | INF; return 1; }
      if (x->neg) { *out = QN; return 1; }
      if (x->cls == CL_INF) { *out = INF; return 1; }
      if (xbits == ONE) { *out = 0; return 1; } /* log(1) = +0 */
      return 0;
    case K_LOG1P:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF) { *out = x->neg ? QN : INF; return 1; }
      if (x->neg && ax == 1.0) { *out = SB | INF; return 1; }
      if (x->neg && ax > 1.0) { *out = QN; return 1; }
      return 0;
    case K_SIN: case K_TAN:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF) { *out = QN; return 1; }
      return 0;
    case K_COS:
      if (x->cls == CL_ZERO) { *out = ONE; return 1; }
      if (x->cls == CL_INF) { *out = QN; return 1; }
      return 0;
    case K_ASIN:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF || ax > 1.0) { *out = QN; return 1; }
      return 0; /* |x| = 1 goes through the loop: 2 atan(1) */
    case K_ACOS:
      if (x->cls == CL_INF || ax > 1.0) { *out = QN; return 1; }
      if (!x->neg && ax == 1.0) { *out = 0; return 1; } /* acos(1) = +0 */
      return 0;
    case K_ATAN:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      return 0; /* +-inf handled in the evaluator */
    case K_SINH:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF) { *out = sgn | INF; return 1; }
      /* |x| >= (emax + 3) ln 2: e^|x| / 2 >= 2^(emax + 2) overflows */
      if (ax >= (double)(f->emax + 3) * LN2_APPROX) { *out = rnd_huge(x->neg, f, mode); return 1; }
      return 0;
    case K_COSH:
      if (x->cls == CL_ZERO) { *out = ONE; return 1; }
      if (x->cls == CL_INF) { *out = INF; return 1; }
      if (ax >= (double)(f->emax + 3) * LN2_APPROX) { *out = rnd_huge(0, f, mode); return 1; }
      return 0;
    case K_TANH:
      if (x->cls == CL_ZERO) { *out = xbits; return 1; }
      if (x->cls == CL_INF) { *out = sgn | ONE; return 1; }
      /* |x| >= (p + 4) ln 2 / 2: 0 < 1 - |tanh x| < 2 e^(-2|x|) <= 2^-(p+3) */
      if (ax >= (double)(f->p + 4) * LN2_APPROX / 2.0) { *out = rnd_below_one(x->neg, f, mode); return 1; }
      return 0;
    case K_RSQRT:
      if (x->cls == CL_ZERO) { *out = sgn | INF; return 1; }
      if (x->neg) { *out = QN; return 1; }
      if (x->cls == CL_INF) { *out = 0; return 1; }
      return 0;
  }
  return 0;
}

static void evaluate(int kind, const dec_t *x, int n, res_t *R) {
  switch (kind) {
    case K_EXP: ev_exp(R, x, n); break;
    case K_EXP2: ev_exp2(R, x, n); break;
    case K_EXP10: ev_exp10(R, x, n); break;
    case K_EXPM1: ev_expm1(R, x, n); break;
    case K_LOG: case K_LOG2: case K_LOG10: ev_log_any(R, x, n, kind); break;
    case K_LOG1P: ev_log1p(R, x, n); break;
    case K_SIN: case K_COS: case K_TAN: ev_trig(R, x, n, kind); break;
    case K_ASIN: ev_asin(R, x, n); break;
    case K_ACOS: ev_acos(R, x, n); break;
    case K_ATAN:
      if (x->cls == CL_INF) {
        const consts_t *C = get_consts(n);
        R->v = C->pio2;
        if (x->neg) iv_neg(&R->v, &R->v, n);
        R->E = 0;
      } else {
        ev_atan(R, x, n);
      }
      break;
    case K_SINH: case K_COSH: ev_sinh_cosh(R, x, n, kind); break;
    case K_TANH: ev_tanh(R, x, n); break;
    case K_RSQRT: ev_rsqrt(R, x, n); break;
  }
}

static const int LEVEL_LIMBS[] = {2, 3, 5, 9, 17, 33};
#define NLEVELS 6

/* The pattern of a positive normal number v of the format, v exact in binary64. */
static uint64_t fmt_bits(double v, const fmt_t *f) {
  int e;
  double m = frexp(v, &e); /* v = m 2^e, m in [1/2, 1) */
  uint64_t M = (uint64_t)ldexp(m, f->p);
  return ((uint64_t)(e - 1 + f->bias) << (f->p - 1)) + M - (1ull << (f->p - 1));
}

/* Results that are exact format numbers although the evaluator's interval around them
   is not degenerate: 10^k and log10(10^k) for the k with 10^k exact in the format.
   (exp2 of an integer, log2 of a power of two and rsqrt of a power of four come out as
   exact intervals; every other nonzero algebraic argument gives a transcendental value,
   Lindemann-Weierstrass.)  Rounding to nearest decides these through the loop; a directed
   mode needs them here. */
static int exact_case(int kind, const dec_t *x, const fmt_t *f, uint64_t *out) {
  /* 10^k = 2^k 5^k is exact while 5^k fits the precision */
  const int kmax = f->p == 53 ? 22 : (f->p == 24 ? 10 : (f->p == 11 ? 4 : 3));
  if (x->cls != CL_FINITE || x->neg) return 0;
  double v = approx(x), p10 = 1.0;
  if (kind == K_EXP10 && is_integer(x) && v <= kmax) {
    for (int i = 0; i < (int)v; i++) p10 *= 10.0;
    *out = fmt_bits(p10, f);
    return 1;
  }
  if (kind == K_LOG10) {
    for (int k = 1; k <= kmax; k++) {
      p10 *= 10.0;
      if (v == p10) {
        *out = fmt_bits((double)k, f);
        return 1;
      }
    }
  }
  return 0;
}

static int ziv(int kind, const dec_t *x, uint64_t xbits, const fmt_t *f, uint64_t *out, int mode) {
  if (special(kind, x, f, xbits, out, mode) || (mode != ORC_RN && exact_case(kind, x, f, out))) {
    g_last_level = -1;
    return ORC_OK;
  }
  /* 10^k for an integer 0 <= k <= 27 is the dyadic 5^k 2^k (5^k < 2^63), rounded directly:
     in binary64, 10^23 is a midpoint (5^23 is an odd 54-bit integer), which no interval
     around it can decide */
  if (kind == K_EXP10 && x->cls == CL_FINITE && !x->neg && is_integer(x) && approx(x) <= 27.0) {
    int64_t p5 = 1;
    for (int i = 0; i < (int)approx(x); i++) p5 *= 5;
    limb a[MAXL];
    fx_set_i64(a, p5, 2);
    *out = round_fixed(a, 2, (int64_t)approx(x), f, mode);
    g_last_level = -1;
    return ORC_OK;
  }
  /* acos(-1) = pi exactly as a real: round pi */
  for (int lvl = 0; lvl < NLEVELS; lvl++) {
    int n = LEVEL_LIMBS[lvl];
    res_t R;
    R.E = 0;
    g_fail = 0;
    if (kind == K_ACOS && x->neg && approx(x) == 1.0) {
      R.v = get_consts(n)->pi;
      R.E = 0;
    } else {
      evaluate(kind, x, n, &R);
    }
    if (g_fail) continue;
    uint64_t a = round_fixed(R.v.lo, n, R.E, f, mode), b = round_fixed(R.v.hi, n, R.E, f, mode);
    if (a == b) {
      *out = a;
      g_last_level = lvl;
      return ORC_OK;
    }
  }
  g_last_level = NLEVELS;
  return ORC_ERR_CAP;
}

/* ===================== public API ===================== */

static int kind_of(int func, int *is64) {
  static const int map[] = {K_EXP, K_EXP2, K_EXP10, K_EXPM1, K_LOG, K_LOG2, K_LOG10,
                            K_LOG1P, K_SIN, K_COS, -1 /*sincos*/, K_TAN, K_ASIN, K_ACOS,
                            K_ATAN, K_SINH, K_COSH, K_TANH, K_RSQRT, K_EXP2, K_LOG,
                            K_EXP, K_LOG2, K_LOG10, K_EXP10};
  if (func < 0 || func >= ORC_NUM_FUNCS) return -2;
  *is64 = func >= ORC_EXP2;
  return map[func];
}

int crm_oracle_f32(int func, uint32_t x, uint32_t *out) { return crm_oracle_f32_rm(func, x, ORC_RN, out); }
int crm_oracle_f64(int func, uint64_t x, uint64_t *out) { return crm_oracle_f64_rm(func, x, ORC_RN, out); }

int crm_oracle_f32_rm(int func, uint32_t x, int mode, uint32_t *out) {
  int is64;
  if (mode < ORC_RN || mode > ORC_RZ) return ORC_ERR_FUNC;
  int kind = kind_of(func, &is64);
  if (kind == -2 || is64) return ORC_ERR_FUNC;
  dec_t d = dec32(x);
  uint64_t r;
  if (func == ORC_SINCOSF) {
    int st = ziv(K_SIN, &d, x, &FMT32, &r, mode);
    if (st) return st;
    out[0] = (uint32_t)r;
    st = ziv(K_COS, &d, x, &FMT32, &r, mode);
    out[1] = (uint32_t)r;
    return st;
  }
  int st = ziv(kind, &d, x, &FMT32, &r, mode);
  out[0] = (uint32_t)r;
  return st;
}

int crm_oracle_f16_rm(int func, int fmt, uint32_t x, int mode, uint32_t *out) {
  int is64;
  int kind = kind_of(func, &is64);
  if (kind == -2 || is64 || (fmt != ORC_FMT_F16 && fmt != ORC_FMT_BF16) || mode < ORC_RN || mode > ORC_RZ)
    return ORC_ERR_FUNC;
  const fmt_t *f = fmt == ORC_FMT_F16 ? &FMT16 : &FMTB16;
  dec_t d = dec_fmt(x & 0xFFFFu, f);
  uint64_t r;
  if (func == ORC_SINCOSF) {
    int st = ziv(K_SIN, &d, x & 0xFFFFu, f, &r, mode);
    if (st) return st;
    out[0] = (uint32_t)r;
    st = ziv(K_COS, &d, x & 0xFFFFu, f, &r, mode);
    out[1] = (uint32_t)r;
    return st;
  }
  int st = ziv(kind, &d, x & 0xFFFFu, f, &r, mode);
  out[0] = (uint32_t)r;
  return st;
}

int crm_oracle_f16_array(int func, int fmt, const uint16_t *in, uint16_t *out, uint64_t n, int mode) {
  for (uint64_t i = 0; i < n; i++) {
    uint32_t r[2];
    int st = crm_oracle_f16_rm(func, fmt, in[i], mode, r);
    if (st) return st;
    out[i] = (uint16_t)r[0];
    if (func == ORC_SINCOSF) out[n + i] = (uint16_t)r[1];
  }
  return ORC_OK;
}

int crm_oracle_f64_rm(int func, uint64_t x, int mode, uint64_t *out) {
  int is64;
  if (mode < ORC_RN || mode > ORC_RZ) return ORC_ERR_FUNC;
  int kind = kind_of(func, &is64);
  if (kind < 0 || !is64) return ORC_ERR_FUNC;
  dec_t d = dec64(x);
  return ziv(kind, &d, x, &FMT64, out, mode);
}

int crm_oracle_last_level(void) { return g_last_level; }

/* How close f(x) lies to a rounding boundary of binary64 round-to-nearest (a midpoint
   between two consecutive binary64 numbers; in the top binade the overflow threshold
   2^1024 - 2^970 is one of them): *h = -log2(d), d the distance in units of the last place
   of the result's binade (0 < d <= 1/2).  A result within 2^-h ulp of a midpoint needs a
   working precision of about 53 + h bits before any evaluation can round it (the hard-to-
   round cases of Sec. II.B).  f(x) is enclosed at 9 limbs (512 fraction bits) and d is
   read from the 128 bits below the rounding position of the interval's lower end, so h is
   exact to far below 2^-60 relative and capped at 128.  Special inputs, results beyond the
   largest binade, and exact results (log(1), exp2 of an integer: d = 1/2) give h <= 1. */
int crm_oracle_f64_hardness(int func, uint64_t xb, double *h) {
  int is64;
  int kind = kind_of(func, &is64);
  if (kind < 0 || !is64) return ORC_ERR_FUNC;
  dec_t x = dec64(xb);
  uint64_t sp;
  *h = -1.0;
  if (special(kind, &x, &FMT64, xb, &sp, ORC_RN)) return ORC_OK;
  res_t R;
  int n = 9;
  for (;;) {
    R.E = 0;
    g_fail = 0;
    evaluate(kind, &x, n, &R);
    if (!g_fail) break;
    if (n == 33) return ORC_ERR_CAP;
    n = 2 * n - 1;
  }
  limb m[MAXL], t[MAXL];
  fx_abs(m, R.v.lo, n);
  int b = mag_bitlen(m, n);
  if (b == 0) return ORC_OK;
  const fmt_t *f = &FMT64;
  int64_t F = FB(n);
  int64_t ex = (int64_t)b - 1 + R.E - F;
  if (ex > f->emax) return ORC_OK;
  int64_t qe = (ex < f->emin ? f->emin : ex) - (f->p - 1);
  int64_t k = qe - (R.E - F); /* discarded bits below the last place */
  if (k < 2) return ORC_OK;
  /* the 128 bits just below the last place: floor(m / 2^(k - 128)) mod 2^128 */
  if (k >= 128) {
    mag_shr(t, m, n, k - 128);
  } else {
    mag_shl(t, m, n, 128 - k);
  }
  u128 w = ((u128)t[1] << 64) | t[0];
  const u128 half = (u128)1 << 127;
  u128 d = w >= half ? w - half : half - w;
  if (d == 0) {
    *h = 128.0;
    return ORC_OK;
  }
  /* -log2(d / 2^128) */
  double dd = (double)(uint64_t)(d >> 64) * 18446744073709551616.0 + (double)(uint64_t)d;
  *h = 128.0 - log2(dd);
  return ORC_OK;
}

/* ---- complex functions built from the real ones (the paper's application of Sec. III.A:
   cexpf, clogf and csinf over real and imaginary parts in [-40, 40]) ----
   cexp(x + iy) = e^x cos y + i e^x sin y;  csin(x + iy) = sin x cosh y + i cos x sinh y;
   clog(z) = log|z| + i atan2(y, x) with log|z| = log(x^2 + y^2) / 2.  Each component is the
   exact value rounded to nearest binary32, by the Ziv loop on its interval.  Finite inputs;
   clog also needs z != 0. */
enum { CX_EXP = 0, CX_LOG = 1, CX_SIN = 2 };

/* f(x) for a finite binary32 x as an interval times 2^E (zero: 0 or 1 exactly) */
static void cx_real(int kind, uint32_t xb, int n, res_t *R) {
  dec_t d = dec32(xb);
  R->E = 0;
  if (d.cls == CL_ZERO) {
    iv_set_i(&R->v, (kind == K_SIN || kind == K_SINH) ? 0 : 1, n);
    return;
  }
  evaluate(kind, &d, n, R);
}

static void cx_prod(int ka, uint32_t a, int kb, uint32_t b, int n, res_t *P) {
  res_t A, B;
  cx_real(ka, a, n, &A);
  cx_real(kb, b, n, &B);
  iv_mul(&P->v, &A.v, &B.v, n);
  P->E = A.E + B.E;
}

/* log|z| = (2 e ln 2 + log S) / 2 with x^2 + y^2 = S 2^(2e), S = Ma^2 + Mb^2 2^(2(eb - ea))
   (a the larger of |x|, |y| = Ma 2^ea); S's second term is truncated to the fraction bits,
   and log is evaluated at both ends of S's interval */
static void cx_logabs(uint32_t xr, uint32_t xi, int n, res_t *R) {
  dec_t a = dec32(xr & 0x7FFFFFFFu), b = dec32(xi & 0x7FFFFFFFu);
  if (approx(&b) > approx(&a)) {
    dec_t t = a;
    a = b;
    b = t;
  }
  const consts_t *C = get_consts(n);
  iv_t S, sb;
  iv_set_scaled(&S, 0, a.M * a.M, 0, n);
  if (b.cls != CL_ZERO) {
    iv_set_scaled(&sb, 0, b.M * b.M, 2 * (b.e - a.e), n);
    iv_add(&S, &S, &sb, n);
  }
  int64_t K1, K2;
  iv_t A1, A2, t;
  log_parts(S.lo, n, &K1, &A1);
  log_parts(S.hi, n, &K2, &A2);
  iv_t L1, L2;
  iv_mul_i(&t, &C->ln2, K1 + 2 * a.e, n);
  iv_add(&L1, &t, &A1, n);
  iv_mul_i(&t, &C->ln2, K2 + 2 * a.e, n);
  iv_add(&L2, &t, &A2, n);
  memcpy(R->v.lo, L1.lo, 8 * (size_t)n);
  memcpy(R->v.hi, L2.hi, 8 * (size_t)n);
  iv_shr(&R->v, &R->v, 1, n);
  R->E = 0;
}

/* atan2(y, x): theta = atan(|y| / |x|) (pi/2 - atan(|x| / |y|) when |y| > |x|), pi - theta for
   x < 0, negated for y < 0; the ratio's exponent difference is applied as a shift */
static void cx_arg(uint32_t xr, uint32_t xi, int n, res_t *R) {
  dec_t a = dec32(xr & 0x7FFFFFFFu), b = dec32(xi & 0x7FFFFFFFu);
  const consts_t *C = get_consts(n);
  iv_t th;
  if (a.cls == CL_ZERO) {
    th = C->pio2;
  } else if (b.cls == CL_ZERO) {
    iv_set_i(&th, 0, n);
  } else {
    const int big = approx(&b) > approx(&a);
    const dec_t *p = big ? &a : &b, *q = big ? &b : &a; /* ratio p / q <= 1 */
    iv_t mp, mq, r;
    iv_set_i(&mp, (int64_t)p->M, n);
    iv_set_i(&mq, (int64_t)q->M, n);
    iv_div(&r, &mp, &mq, n);
    const int64_t sh = p->e - q->e; /* <= 0, or small */
    if (sh >= 0)
      iv_shl(&r, &r, sh, n);
    else
      iv_shr(&r, &r, -sh, n);
    iv_atan(&th, &r, n);
    if (big) iv_sub(&th, &C->pio2, &th, n);
  }
  if (xr >> 31) iv_sub(&th, &C->pi, &th, n);
  if (xi >> 31) iv_neg(&th, &th, n);
  R->v = th;
  R->E = 0;
}

int crm_oracle_complex(int which, uint32_t xr, uint32_t xi, uint32_t out[2]) {
  if (which < CX_EXP || which > CX_SIN) return ORC_ERR_FUNC;
  for (int comp = 0; comp < 2; comp++) {
    int lvl;
    for (lvl = 0; lvl < NLEVELS; lvl++) {
      const int n = LEVEL_LIMBS[lvl];
      res_t R;
      g_fail = 0;
      if (which == CX_EXP)
        cx_prod(K_EXP, xr, comp ? K_SIN : K_COS, xi, n, &R);
      else if (which == CX_SIN)
        cx_prod(comp ? K_COS : K_SIN, xr, comp ? K_SINH : K_COSH, xi, n, &R);
      else if (comp == 0)
        cx_logabs(xr, xi, n, &R);
      else
        cx_arg(xr, xi, n, &R);
      if (g_fail) continue;
      uint64_t lo = round_fixed(R.v.lo, n, R.E, &FMT32, ORC_RN), hi = round_fixed(R.v.hi, n, R.E, &FMT32, ORC_RN);
      if (lo == hi) {
        out[comp] = (uint32_t)lo;
        break;
      }
    }
    if (lvl == NLEVELS) return ORC_ERR_CAP;
  }
  return ORC_OK;
}

int crm_oracle_complex_array(int which, const uint32_t *in, uint32_t *out, uint64_t n) {
  for (uint64_t i = 0; i < n; i++) {
    int st = crm_oracle_complex(which, in[2 * i], in[2 * i + 1], out + 2 * i);
    if (st) return st;
  }
  return ORC_OK;
}

/* ---- threaded array drivers ---- */
typedef struct {
  int func, is64, mode, hardness;
  const void *in;
  void *out;
  uint64_t n;
  uint64_t next; /* atomic work counter */
  int status;    /* first error (atomic) */
} job_t;

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  const uint64_t chunk = 256;
  for (;;) {
    uint64_t start = __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
    if (start >= J->n) break;
    uint64_t end = start + chunk < J->n ? start + chunk : J->n;
    for (uint64_t i = start; i < end; i++) {
      int st;
      if (J->hardness) {
        st = crm_oracle_f64_hardness(J->func, ((const uint64_t *)J->in)[i], ((double *)J->out) + i);
      } else if (J->is64) {
        st = crm_oracle_f64_rm(J->func, ((const uint64_t *)J->in)[i], J->mode, ((uint64_t *)J->out) + i);
      } else if (J->func == ORC_SINCOSF) {
        uint32_t sc[2];
        st = crm_oracle_f32_rm(J->func, ((const uint32_t *)J->in)[i], J->mode, sc);
        ((uint32_t *)J->out)[i] = sc[0];
        ((uint32_t *)J->out)[J->n + i] = sc[1];
      } else {
        st = crm_oracle_f32_rm(J->func, ((const uint32_t *)J->in)[i], J->mode, ((uint32_t *)J->out) + i);
      }
      if (st) {
        int zero = 0;
        __atomic_compare_exchange_n(&J->status, &zero, st, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED);
      }
    }
  }
  return NULL;
}

static int run_job(job_t *J, int nthreads) {
  if (nthreads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    nthreads = c > 0 ? (int)c : 1;
  }
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > J->n / 64 + 1) nthreads = (int)(J->n / 64 + 1);
  /* compute the constants once before the threads start */
  for (int l = 0; l < NLEVELS; l++) {
    get_consts(LEVEL_LIMBS[l]);
    get_consts(LEVEL_LIMBS[l] + 5);
  }
  pthread_t th[256];
  int started = 0;
  for (int t = 1; t < nthreads; t++)
    if (pthread_create(&th[started], NULL, worker, J) == 0) started++;
  worker(J);
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  return J->status;
}

int crm_oracle_f32_array_rm(int func, const uint32_t *in, uint32_t *out, uint64_t n, int nthreads, int mode) {
  int is64;
  int kind = kind_of(func, &is64);
  if (kind == -2 || is64 || mode < ORC_RN || mode > ORC_RZ) return ORC_ERR_FUNC;
  job_t J = {func, 0, mode, 0, in, out, n, 0, 0};
  return run_job(&J, nthreads);
}

int crm_oracle_f64_array_rm(int func, const uint64_t *in, uint64_t *out, uint64_t n, int nthreads, int mode) {
  int is64;
  int kind = kind_of(func, &is64);
  if (kind < 0 || !is64 || mode < ORC_RN || mode > ORC_RZ) return ORC_ERR_FUNC;
  job_t J = {func, 1, mode, 0, in, out, n, 0, 0};
  return run_job(&J, nthreads);
}

int crm_oracle_f64_hardness_array(int func, const uint64_t *in, double *out, uint64_t n, int nthreads) {
  int is64;
  int kind = kind_of(func, &is64);
  if (kind < 0 || !is64) return ORC_ERR_FUNC;
  job_t J = {func, 1, ORC_RN, 1, in, out, n, 0, 0};
  return run_job(&J, nthreads);
}

int crm_oracle_f32_array(int func, const uint32_t *in, uint32_t *out, uint64_t n, int nthreads) {
  return crm_oracle_f32_array_rm(func, in, out, n, nthreads, ORC_RN);
}
int crm_oracle_f64_array(int func, const uint64_t *in, uint64_t *out, uint64_t n, int nthreads) {
  return crm_oracle_f64_array_rm(func, in, out, n, nthreads, ORC_RN);
}

/* ---- diagnostics ---- */
static void put_iv(const iv_t *v, int n, uint64_t *lo, uint64_t *hi) {
  memcpy(lo, v->lo, 8 * (size_t)n);
  memcpy(hi, v->hi, 8 * (size_t)n);
}

int crm_oracle_constant(int which, int nlimbs, uint64_t *lo, uint64_t *hi) {
  if (nlimbs < 2 || nlimbs > MAXL) return ORC_ERR_FUNC;
  const consts_t *C = get_consts(nlimbs);
  switch (which) {
    case 0: put_iv(&C->ln2, nlimbs, lo, hi); break;
    case 1: put_iv(&C->ln10, nlimbs, lo, hi); break;
    case 2: put_iv(&C->pi, nlimbs, lo, hi); break;
    case 3: put_iv(&C->twoopi, nlimbs, lo, hi); break;
    default: return ORC_ERR_FUNC;
  }
  return ORC_OK;
}

int crm_oracle_constant_alt(int which, int n, uint64_t *lo, uint64_t *hi) {
  if (n < 2 || n > MAXL) return ORC_ERR_FUNC;
  iv_t r, t;
  if (which == 0) {
    /* ln 2 = sum_{k>=1} 1/(k 2^k), positive terms with ratio <= 1/2 */
    iv_t p, s;
    iv_set_i(&p, 1, n);
    iv_set_i(&s, 0, n);
    for (uint64_t k = 1;; k++) {
      iv_shr(&p, &p, 1, n);
      iv_div_u(&t, &p, k, n);
      limb mg[MAXL];
      iv_absmax(mg, &t, n);
      if (small_enough(mg, n)) {
        iv_widen_tail(&s, &t, n);
        break;
      }
      iv_add(&s, &s, &t, n);
    }
    r = s;
  } else if (which == 2) {
    /* pi = 48 atan(1/18) + 32 atan(1/57) - 20 atan(1/239)  (Gauss) */
    iv_t a;
    iv_atan_inv(&a, 18, n);
    iv_mul_u(&r, &a, 48, n);
    iv_atan_inv(&a, 57, n);
    iv_mul_u(&a, &a, 32, n);
    iv_add(&r, &r, &a, n);
    iv_atan_inv(&a, 239, n);
    iv_mul_u(&a, &a, 20, n);
    iv_sub(&r, &r, &a, n);
  } else {
    return ORC_ERR_FUNC;
  }
  put_iv(&r, n, lo, hi);
  return ORC_OK;
}

int crm_oracle_test_divmod(const uint32_t *u, int m, const uint32_t *v, int nv, uint32_t *q) {
  return divmod_d32(q, u, m, v, nv);
}

int crm_oracle_test_isqrt(const uint64_t *N, int nl, uint64_t *r) {
  if (nl > 2 * MAXL) return -1;
  return mag_isqrt(r, N, nl);
}
