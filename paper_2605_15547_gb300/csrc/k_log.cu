// k_log.cu -- logf, log2f, log10f, log1pf kernels (all tiers).
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_log(FuncEntry *t) {
  set_entry<FnLog<0>, true, true>(t[4]);  // CRM_LOGF
  set_entry<FnLog<1>, true, true>(t[5]);  // CRM_LOG2F
  set_entry<FnLog<2>, true, true>(t[6]);  // CRM_LOG10F
  set_entry<FnLog<3>, true, true>(t[7]);  // CRM_LOG1PF
}

}  // namespace crm
