// k_hyp.cu -- expm1f, sinhf, coshf, tanhf kernels.
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_hyp(FuncEntry *t) {
  set_entry<FnHyp<HYP_EXPM1>, true, true>(t[3]);   // CRM_EXPM1F
  set_entry<FnHyp<HYP_SINH>, true, true>(t[15]);   // CRM_SINHF
  set_entry<FnHyp<HYP_COSH>, true, true>(t[16]);   // CRM_COSHF
  set_entry<FnHyp<HYP_TANH>, true, true>(t[17]);   // CRM_TANHF
}

}  // namespace crm
