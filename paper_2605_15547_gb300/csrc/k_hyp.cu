// k_hyp.cu -- expm1f, sinhf, coshf, tanhf kernels.
#include "crm_registry.h"
#include "fam_hyp.cuh"

namespace crm {

template <int H> struct FnHyp {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 16 * 8; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) { copy_tab(sm, (const void *)CRM_EXP2_T16_D, tab_bytes<FORM>()); }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    y[0] = hyp_plain<H>(x, (const double *)sm, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = hyp_slow<H>(x, u); }
};

void register_hyp(FuncEntry *t) {
  set_entry<FnHyp<HYP_EXPM1>, true, false>(t[3]);   // CRM_EXPM1F
  set_entry<FnHyp<HYP_SINH>, true, false>(t[15]);   // CRM_SINHF
  set_entry<FnHyp<HYP_COSH>, true, false>(t[16]);   // CRM_COSHF
  set_entry<FnHyp<HYP_TANH>, true, false>(t[17]);   // CRM_TANHF
}

}  // namespace crm
