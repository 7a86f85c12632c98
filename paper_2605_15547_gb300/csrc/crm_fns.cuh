// crm_fns.cuh -- the per-function descriptors used by the array, slow and batch kernels:
// shared-memory table layout, the fast-tier evaluator for each form and the exact slow
// path (see the Fn interface in crm_kernels.cuh).
#pragma once
#include "crm_kernels.cuh"
#include "fam_atrig.cuh"
#include "fam_exp.cuh"
#include "fam_f64.cuh"
#include "fam_hyp.cuh"
#include "fam_log.cuh"
#include "fam_rsqrt.cuh"
#include "fam_trig.cuh"

namespace crm {

template <int KIND> struct FnExp {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return FORM == 1 ? 16 * 8 : 64 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_EXP2_T16_D : (const void *)CRM_EXP2_T64U_DF, tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h, int *sg = nullptr) {
    if (FORM == 1)
      y[0] = exp_plain<KIND>(x, (const double *)sm, h);
    else
      y[0] = exp_df<KIND>(x, (const float4 *)sm, h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { y[0] = exp_slow<KIND>(x, u, f, sg); }
  // Round to nearest, b^x is 1 for |x| <= 2^-25 (2^x: as 2^-25 < 2^-24.5 = 2^-25 / ln 2;
  // 10^x: |x| <= 2^-27 < 2^-25 / ln 10): b^x - 1 is then below 2^-25 + 2^-51 in magnitude,
  // inside the midpoints 1 + 2^-24 and 1 - 2^-25 (e^(-2^-25) = 1 - 2^-25 + 2^-51 - ...).
  static constexpr bool HAS_EASY = true;
  CRM_DEV static bool easy(float x, float *y) {
    y[0] = 1.0f;
    return fabsf(x) <= (KIND == 2 ? 0x1p-27f : 0x1p-25f);
  }
};

// The exp family's double-float tier with its 16-entry table in registers (Ctx: the
// lane's table entry, read by the other lanes through warp shuffles); the main kernel's
// register-table launch shape.  Same slow path and bits as FnExp.
template <int KIND> struct FnExpShfl {
  using T = float;
  using Ctx = float4;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 0; }
  template <int FORM> CRM_DEV static void load(unsigned char *) {}
  template <int FORM> CRM_DEV static Ctx make_ctx(const unsigned char *) {
    const float4 *t = (const float4 *)CRM_EXP2_T16U_DF;
    return t[threadIdx.x & 15];
  }
  template <int FORM> CRM_DEV static void eval(float x, const Ctx &R, float *y, bool &h) {
    y[0] = exp_df16<KIND>(x, R, h);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f) { y[0] = exp_slow<KIND>(x, u, f); }
};

template <int KIND> struct FnLog {
  using T = float;
  static constexpr int NOUT = 1;
  // plain: 97 (1/c_j, ln c_j) doubles; double-float: 193 (R_j, -ln R_j in three words)
  // float4s (every kind: log2 and log10 scale the natural logarithm)
  template <int FORM> static constexpr int tab_bytes() { return FORM == 1 ? 97 * 16 : 193 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_LN_T97_D : (const void *)CRM_LN_T193M_DF, tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h, int *sg = nullptr) {
    if (FORM == 1)
      y[0] = log_plain<KIND>(x, (const double2 *)sm, h);
    else
      y[0] = log_df<KIND>(x, (const float4 *)sm, h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { y[0] = log_slow<KIND>(x, u, f, sg); }
  // log1p x = x - x^2/2 + ... rounds to x for |x| < 2^-26: with 2^e <= |x| < 2^(e+1),
  // e <= -27, x^2/2 < 2^(2e+1) is below a quarter ulp of x, 2^(e-25) (the distance to the
  // midpoint toward zero when x is a power of two; half an ulp otherwise).  ln, log2 and
  // log10 have no such range.
  static constexpr bool HAS_EASY = KIND == 3;
  CRM_DEV static bool easy(float x, float *y) {
    y[0] = x;
    return fabsf(x) < 0x1p-26f;
  }
};

template <int H> struct FnHyp {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return FORM == 1 ? 16 * 8 : 64 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_EXP2_T16_D : (const void *)CRM_EXP2_T64U_DF, tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h, int *sg = nullptr) {
    if (FORM == 1)
      y[0] = hyp_plain<H>(x, (const double *)sm, h);
    else
      y[0] = hyp_df<H>(x, (const float4 *)sm, h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { y[0] = hyp_slow<H>(x, u, f, sg); }
  // Round to nearest: expm1 x = x + x^2/2 + ... is x for |x| < 2^-26 (the bound of log1p);
  // sinh x = x + x^3/6 + ... and tanh x = x - x^3/3 + ... are x for |x| < 2^-12 (with
  // 2^e <= |x| < 2^(e+1), e <= -13: x^3/3 < 2^(3e+3)/3 <= 2^(e-24), half an ulp, and for x
  // a power of two x^3/3 = 2^(3e)/3 < 2^(e-25), a quarter); cosh x = 1 + x^2/2 + ... is 1
  // for |x| < 2^-12 (x^2/2 < 2^-25, below the midpoint 1 + 2^-24).
  static constexpr bool HAS_EASY = true;
  CRM_DEV static bool easy(float x, float *y) {
    y[0] = H == HYP_COSH ? 1.0f : x;
    return fabsf(x) < (H == HYP_EXPM1 ? 0x1p-26f : 0x1p-12f);
  }
};

template <int KIND> struct FnTrig {
  using T = float;
  static constexpr int NOUT = KIND == TRIG_SINCOS ? 2 : 1;
  // shared memory: 16 words of 2/pi, the (sin, cos) table (FP64 form: 32 double pairs of
  // j pi/64; double-float form: 128 float quadruples (hi, lo, hi, lo) of j pi/256; 16 bytes
  // each), 8 window entries of four consecutive words of 2/pi (PW[k] = words k .. k+3, zero
  // beyond the 16), and for tan the (tan hi, lo)(j pi/256) float pairs
  static constexpr int OFF_PW = 64 + 128 * 16, OFF_TT = OFF_PW + 8 * 16;
  template <int FORM> static constexpr int tab_bytes() { return OFF_TT + (KIND == TRIG_TAN ? 128 * 8 : 0); }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, CRM_TWO_OVER_PI_W, 64);
    if (FORM == 1)
      copy_tab(sm + 64, CRM_SINCOS_T32_D, 32 * 16);
    else
      copy_tab(sm + 64, CRM_SINCOS_T128_DF, 128 * 16);
    uint32_t *pw = (uint32_t *)(sm + OFF_PW);
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
      const int w = (i >> 2) + (i & 3);
      pw[i] = w < 16 ? CRM_TWO_OVER_PI_W[w] : 0u;
    }
    if (KIND == TRIG_TAN && FORM == 2) copy_tab(sm + OFF_TT, CRM_TAN_T128_DF, 128 * 8);
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h, int *sg = nullptr) {
    const unsigned char *b = (const unsigned char *)sm;
    if (FORM == 1)
      trig_plain<KIND>(x, (const uint32_t *)b, (const double *)(b + 64), y, h);
    else
      trig_df<KIND>(x, (const uint4 *)(b + OFF_PW), (const float4 *)(b + 64), (const float2 *)(b + OFF_TT), y,
                    h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { trig_slow<KIND>(x, y, u, f, sg); }
  // Round to nearest: sin x = x - x^3/6 + ... and tan x = x + x^3/3 + ... are x, cos x =
  // 1 - x^2/2 + ... is 1, for |x| < 2^-12 (the bounds of sinh, tanh and cosh).
  static constexpr bool HAS_EASY = true;
  CRM_DEV static bool easy(float x, float *y) {
    y[0] = KIND == TRIG_COS ? 1.0f : x;
    y[1] = 1.0f;
    return fabsf(x) < 0x1p-12f;
  }
  // warp-uniform choice of the double-float reduction (see trig_reduce_df)
  CRM_DEV static bool path_ok(float x) { return trig_cw_ok(x); }
  template <int FORM, int PATH> CRM_DEV static void eval_path(float x, const void *sm, float *y, bool &h) {
    const unsigned char *b = (const unsigned char *)sm;
    trig_df<KIND, PATH>(x, (const uint4 *)(b + OFF_PW), (const float4 *)(b + 64), (const float2 *)(b + OFF_TT), y, h);
  }
};

template <int KIND> struct FnAtrig {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 18 * 8; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_ATAN_T17_D : (const void *)CRM_ATAN_T17_DF, 18 * 8);
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h, int *sg = nullptr) {
    if (FORM == 1)
      y[0] = atrig_plain<KIND>(x, (const double *)sm, h);
    else
      y[0] = atrig_df<KIND>(x, (const float2 *)sm, h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { y[0] = atrig_slow<KIND>(x, u, f, sg); }
  // Round to nearest: asin x = x + x^3/6 + ... and atan x = x - x^3/3 + ... are x for
  // |x| < 2^-12 (the bounds of sinh and tanh).  With P = RN(pi/2) = pi/2 + 2^-24.45 and its
  // midpoints P -+ 2^-24: acos x = pi/2 - x - x^3/6 - ... lies between them for
  // |x| < 2^-26, and atan x = +-(pi/2 - 1/|x| + ...) for 2^26 <= |x| < inf (1/|x| <= 2^-26 <
  // 2^-24 - 2^-24.45 = 2^-25.9).
  static constexpr bool HAS_EASY = true;
  CRM_DEV static bool easy(float x, float *y) {
    const float ax = fabsf(x), P = bitsf(0x3FC90FDBu);
    if (KIND == AT_ACOS) {
      y[0] = P;
      return ax < 0x1p-26f;
    }
    const bool big = KIND == AT_ATAN && ax >= 0x1p26f;
    y[0] = big ? copysignf(P, x) : x;
    return ax < 0x1p-12f || (big && ax < CRM_INF_F);
  }
};

struct FnRsqrt {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 0; }
  template <int FORM> CRM_DEV static void load(unsigned char *) {}
  template <int FORM> CRM_DEV static void eval(float x, const void *, float *y, bool &h, int *sg = nullptr) {
    y[0] = FORM == 1 ? rsqrt_plain(x, h) : rsqrt_df(x, h, sg);
  }
  CRM_DEV static void slow(float x, float *y, int &u, bool f, int *sg = nullptr) { y[0] = rsqrt_slow(x, u, f, sg); }
};

// binary64 pair: one main path (double-double), used for both form slots
struct FnExp2D {
  using T = double;
  static constexpr int NOUT = 1;
  // form 1: double-double in FP64; form 2: FP64-free (128-bit fixed point)
  template <int FORM> static constexpr int tab_bytes() { return FORM == 2 ? 1024 * 16 : 96 * 8; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    if (FORM == 2)
      copy_tab(sm, CRM_EXP2I_T, 1024 * 16);
    else
      copy_tab(sm, CRM_EXP2D_T, 96 * 8);
  }
  template <int FORM> CRM_DEV static void eval(double x, const void *sm, double *y, bool &h, int *sg = nullptr) {
    if (FORM == 2)
      y[0] = exp2d_int(x, (const ulonglong2 *)sm, h, sg);
    else
      y[0] = exp2d_main(x, (const double *)sm, h, sg);
  }
  CRM_DEV static void slow(double x, double *y, int &u, bool f, int *sg = nullptr) { y[0] = exp2d_slow(x, u, f, sg); }
};
struct FnLogD {
  using T = double;
  static constexpr int NOUT = 1;
  // form 1: double-double in FP64; form 2: FP64-free (128-bit fixed point), with the
  // tables -log(R_j 2^-9) (193 x 16 bytes) and R_j (194 x 2 bytes) in shared memory
  static constexpr int LBYTES = 193 * 16;
  template <int FORM> static constexpr int tab_bytes() { return FORM == 2 ? LBYTES + 194 * 2 + 12 : 0; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    if (FORM == 2) {
      copy_tab(sm, CRM_LOGI_L, LBYTES);
      copy_tab(sm + LBYTES, CRM_LOGI_R, 194 * 2);
    }
  }
  template <int FORM> CRM_DEV static void eval(double x, const void *sm, double *y, bool &h, int *sg = nullptr) {
    if (FORM == 2)
      y[0] = logd_int(x, (const ulonglong2 *)sm, (const unsigned short *)((const unsigned char *)sm + LBYTES), h,
                      sg);
    else
      y[0] = logd_main(x, h, sg);
  }
  CRM_DEV static void slow(double x, double *y, int &u, bool f, int *sg = nullptr) { y[0] = logd_slow(x, u, f, sg); }
};

// More binary64 functions on the fixed-point cores: e^x and 10^x (KIND 0, 2) on the exp2
// core with the 1024-entry table, log2 and log10 (KIND 1, 2) on the log core; the slow path
// is the exact 192-bit tier.  One form (the FP64-free one).
template <int KIND> struct FnExpBD {
  using T = double;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 1024 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) { copy_tab(sm, CRM_EXP2I_T, 1024 * 16); }
  template <int FORM> CRM_DEV static void eval(double x, const void *sm, double *y, bool &h, int *sg = nullptr) {
    y[0] = expbd_int<KIND>(x, (const ulonglong2 *)sm, h, sg);
  }
  CRM_DEV static void slow(double x, double *y, int &u, bool f, int *sg = nullptr) {
    y[0] = expbd_slow<KIND>(x, u, f, sg);
  }
};
template <int KIND> struct FnLogBD {
  using T = double;
  static constexpr int NOUT = 1;
  static constexpr int LBYTES = 193 * 16;
  template <int FORM> static constexpr int tab_bytes() { return LBYTES + 194 * 2 + 12; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, CRM_LOGI_L, LBYTES);
    copy_tab(sm + LBYTES, CRM_LOGI_R, 194 * 2);
  }
  template <int FORM> CRM_DEV static void eval(double x, const void *sm, double *y, bool &h, int *sg = nullptr) {
    y[0] = logbd_int<KIND>(x, (const ulonglong2 *)sm, (const unsigned short *)((const unsigned char *)sm + LBYTES),
                           h, sg);
  }
  CRM_DEV static void slow(double x, double *y, int &u, bool f, int *sg = nullptr) {
    y[0] = logbd_slow<KIND>(x, u, f, sg);
  }
};

}  // namespace crm
