// k_atrig.cu -- atanf, asinf, acosf, rsqrtf kernels.
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_atrig(FuncEntry *t) {
  set_entry<FnAtrig<AT_ASIN>, true, true>(t[12]);  // CRM_ASINF
  set_entry<FnAtrig<AT_ACOS>, true, true>(t[13]);  // CRM_ACOSF
  set_entry<FnAtrig<AT_ATAN>, true, true>(t[14]);  // CRM_ATANF
  set_entry<FnRsqrt, true, true>(t[18]);           // CRM_RSQRTF
}

}  // namespace crm
