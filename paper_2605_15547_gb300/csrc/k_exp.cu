// k_exp.cu -- expf, exp2f, exp10f kernels (all tiers).
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_exp(FuncEntry *t) {
  set_entry<FnExp<0>, true, true>(t[0]);  // CRM_EXPF
  set_entry<FnExp<1>, true, true>(t[1]);  // CRM_EXP2F
  set_entry<FnExp<2>, true, true>(t[2]);  // CRM_EXP10F
  set_regtab_variant<FnExpShfl<0>>(t[0]);
  set_regtab_variant<FnExpShfl<1>>(t[1]);
  set_regtab_variant<FnExpShfl<2>>(t[2]);
}

}  // namespace crm
