// k_hyp.cu -- expm1f, sinhf, coshf, tanhf kernels.
#include "crm_registry.h"
#include "fam_hyp.cuh"

namespace crm {

template <int H> struct FnHyp {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return FORM == 1 ? 16 * 8 : 64 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_EXP2_T16_D : (const void *)CRM_EXP2_T64U_DF, tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    if (FORM == 1)
      y[0] = hyp_plain<H>(x, (const double *)sm, h);
    else
      y[0] = hyp_df<H>(x, (const float4 *)sm, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = hyp_slow<H>(x, u); }
};

void register_hyp(FuncEntry *t) {
  set_entry<FnHyp<HYP_EXPM1>, true, true>(t[3]);   // CRM_EXPM1F
  set_entry<FnHyp<HYP_SINH>, true, true>(t[15]);   // CRM_SINHF
  set_entry<FnHyp<HYP_COSH>, true, true>(t[16]);   // CRM_COSHF
  set_entry<FnHyp<HYP_TANH>, true, true>(t[17]);   // CRM_TANHF
}

}  // namespace crm
