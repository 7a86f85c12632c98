// k_exp.cu -- expf, exp2f, exp10f kernels (all tiers).
#include "crm_registry.h"
#include "fam_exp.cuh"

namespace crm {

template <int KIND> struct FnExp {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return FORM == 1 ? 16 * 8 : 64 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_EXP2_T16_D : (const void *)CRM_EXP2_T64U_DF, tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    if (FORM == 1)
      y[0] = exp_plain<KIND>(x, (const double *)sm, h);
    else
      y[0] = exp_df<KIND>(x, (const float4 *)sm, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = exp_slow<KIND>(x, u); }
};

void register_exp(FuncEntry *t) {
  set_entry<FnExp<0>, true, true>(t[0]);  // CRM_EXPF
  set_entry<FnExp<1>, true, true>(t[1]);  // CRM_EXP2F
  set_entry<FnExp<2>, true, true>(t[2]);  // CRM_EXP10F
}

}  // namespace crm
