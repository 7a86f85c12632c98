/*
 * crm_oracle.h -- correctly rounded reference evaluator (TEST INFRASTRUCTURE ONLY).
 *
 * This is the parity oracle for the GPU library: a plain, slow CPU implementation of
 *     out = RN_fmt(f(x))      (round to nearest, ties to even; binary32 or binary64)
 * for the one-input functions of the paper (Sec. II.A lists the 19 single-precision
 * functions, Sec. II.B the double-precision exp2 and log; exp, log2, log10 and exp10 in
 * binary64 extend that pair, as the paper's outlook asks for more double functions).  It follows Ziv's method
 * (Sec. I): evaluate an interval that provably encloses f(x) with multiprecision
 * integer (fixed-point) arithmetic, and raise the precision until both interval
 * ends round to the same floating-point number.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library; the product
 * path never does, and this code shares nothing with the CUDA sources.
 *
 * Function identifiers are the oracle's own; by design they carry the same numbers
 * as the public library's identifiers so that tests can pass one integer to both.
 */
#ifndef CRM_ORACLE_H
#define CRM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_EXPF = 0, ORC_EXP2F, ORC_EXP10F, ORC_EXPM1F, ORC_LOGF, ORC_LOG2F, ORC_LOG10F,
  ORC_LOG1PF, ORC_SINF, ORC_COSF, ORC_SINCOSF, ORC_TANF, ORC_ASINF, ORC_ACOSF,
  ORC_ATANF, ORC_SINHF, ORC_COSHF, ORC_TANHF, ORC_RSQRTF,
  ORC_EXP2 = 19, ORC_LOG = 20,
  /* more binary64 functions: the same formulas as expf, log2f, log10f and exp10f, in binary64 */
  ORC_EXP = 21, ORC_LOG2 = 22, ORC_LOG10 = 23, ORC_EXP10 = 24,
  ORC_NUM_FUNCS = 25
};

enum { ORC_OK = 0, ORC_ERR_FUNC = 1, ORC_ERR_CAP = 2 };

/* Rounding direction (IEEE 754 Sec. 4.3): to nearest, ties to even (the paper's mode and
   the library's); toward -inf; toward +inf; toward zero. */
enum { ORC_RN = 0, ORC_RD = 1, ORC_RU = 2, ORC_RZ = 3 };

/* One binary32 input (bit pattern) -> result bit pattern.  For ORC_SINCOSF, out[0]
   receives sin and out[1] cos.  Returns ORC_OK, ORC_ERR_FUNC (bad id / wrong
   format) or ORC_ERR_CAP (Ziv precision cap reached: never expected). */
int crm_oracle_f32(int func, uint32_t x, uint32_t *out);
int crm_oracle_f64(int func, uint64_t x, uint64_t *out);
/* The same in rounding direction mode (ORC_RN .. ORC_RZ; another value: ORC_ERR_FUNC). */
int crm_oracle_f32_rm(int func, uint32_t x, int mode, uint32_t *out);
int crm_oracle_f64_rm(int func, uint64_t x, int mode, uint64_t *out);

/* The binary32 function ids evaluated for 16-bit formats: IEEE binary16 (ORC_FMT_F16:
   11-bit precision, exponents -14..15) or bfloat16 (ORC_FMT_BF16: 8-bit precision,
   binary32's exponent range); inputs and results are 16-bit patterns.  The array form
   is single-threaded (sincosf: sin in out[0, n), cos in out[n, 2n)). */
enum { ORC_FMT_F16 = 0, ORC_FMT_BF16 = 1 };
int crm_oracle_f16_rm(int func, int fmt, uint32_t x, int mode, uint32_t *out);
int crm_oracle_f16_array(int func, int fmt, const uint16_t *in, uint16_t *out, uint64_t n, int mode);

/* Array forms, multithreaded with nthreads POSIX threads (<=0: one per online core).
   For ORC_SINCOSF, out holds 2n words: sin in [0,n), cos in [n,2n). */
int crm_oracle_f32_array(int func, const uint32_t *in, uint32_t *out, uint64_t n, int nthreads);
int crm_oracle_f64_array(int func, const uint64_t *in, uint64_t *out, uint64_t n, int nthreads);
int crm_oracle_f32_array_rm(int func, const uint32_t *in, uint32_t *out, uint64_t n, int nthreads, int mode);
int crm_oracle_f64_array_rm(int func, const uint64_t *in, uint64_t *out, uint64_t n, int nthreads, int mode);

/* Distance of f(x) from the nearest binary64 round-to-nearest boundary (a midpoint between
   consecutive binary64 numbers), for the binary64 functions: *h = -log2(distance in ulps),
   so a result within 2^-h ulp of a midpoint; capped at 128; h <= 1 for special inputs and
   exact results.  Used to select hard-to-round test inputs.  The array form is threaded. */
int crm_oracle_f64_hardness(int func, uint64_t x, double *h);
int crm_oracle_f64_hardness_array(int func, const uint64_t *in, double *out, uint64_t n, int nthreads);

/* Complex functions built from the real ones, the paper's second application (Sec. III.A):
   which 0: cexp(x + iy) = e^x cos y + i e^x sin y; 1: clog(z) = log|z| + i atan2(y, x);
   2: csin(x + iy) = sin x cosh y + i cos x sinh y.  Each component of the exact value is
   rounded to nearest binary32 (out[0] real, out[1] imaginary).  Finite inputs (clog: z != 0).
   The array form takes n interleaved (re, im) pairs. */
int crm_oracle_complex(int which, uint32_t xr, uint32_t xi, uint32_t out[2]);
int crm_oracle_complex_array(int which, const uint32_t *in, uint32_t *out, uint64_t n);

/* Diagnostics for the oracle's own tests: the Ziv level (0 = first precision) at which
   the last call on this thread finished, and the constants as scaled integers. */
int crm_oracle_last_level(void);
/* Writes floor and ceil of c * 2^bits for c in {0: ln2, 1: ln10, 2: pi, 3: 2/pi} into
   lo/hi as little-endian 64-bit limbs (nlimbs each); bits = 64*(nlimbs-1). */
int crm_oracle_constant(int which, int nlimbs, uint64_t *lo, uint64_t *hi);
/* Alternative formulas for the same constants (pi by Gauss's arctangent formula,
   ln2 by sum 1/(k 2^k)), for cross-checking in tests. */
int crm_oracle_constant_alt(int which, int nlimbs, uint64_t *lo, uint64_t *hi);
/* Big-integer long division used by the oracle: q = floor(u / v), returns 1 if the
   remainder is nonzero.  u has m 32-bit digits, v has nv digits (v[nv-1] != 0). */
int crm_oracle_test_divmod(const uint32_t *u, int m, const uint32_t *v, int nv, uint32_t *q);
/* Integer square root used by the oracle: r = floor(sqrt(N)); returns 1 if inexact. */
int crm_oracle_test_isqrt(const uint64_t *N, int nl, uint64_t *r);

#ifdef __cplusplus
}
#endif
#endif
