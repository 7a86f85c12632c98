// k_trig.cu -- sinf, cosf, sincosf, tanf kernels.
#include "crm_registry.h"
#include "fam_trig.cuh"

namespace crm {

template <int KIND> struct FnTrig {
  using T = float;
  static constexpr int NOUT = KIND == TRIG_SINCOS ? 2 : 1;
  // shared memory: 16 words of 2/pi, then the (sin, cos)(j pi/64) table (double or
  // float-pair entries, 16 bytes each)
  template <int FORM> static constexpr int tab_bytes() { return 64 + 32 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, CRM_TWO_OVER_PI_W, 64);
    copy_tab(sm + 64, FORM == 1 ? (const void *)CRM_SINCOS_T32_D : (const void *)CRM_SINCOS_T32_DF, 32 * 16);
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    const unsigned char *b = (const unsigned char *)sm;
    if (FORM == 1)
      trig_plain<KIND>(x, (const uint32_t *)b, (const double *)(b + 64), y, h);
    else
      trig_df<KIND>(x, (const uint32_t *)b, (const float4 *)(b + 64), y, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { trig_slow<KIND>(x, y, u); }
};

void register_trig(FuncEntry *t) {
  set_entry<FnTrig<TRIG_SIN>, true, true>(t[8]);      // CRM_SINF
  set_entry<FnTrig<TRIG_COS>, true, true>(t[9]);      // CRM_COSF
  set_entry<FnTrig<TRIG_SINCOS>, true, true>(t[10]);  // CRM_SINCOSF
  set_entry<FnTrig<TRIG_TAN>, true, true>(t[11]);     // CRM_TANF
}

}  // namespace crm
