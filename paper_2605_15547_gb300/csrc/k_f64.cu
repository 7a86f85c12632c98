// k_f64.cu -- binary64 exp2 and log kernels (double-double main path, exact slow path).
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_f64(FuncEntry *t) {
  set_entry<FnExp2D, true, true>(t[19]);  // CRM_EXP2
  set_entry<FnLogD, true, true>(t[20]);   // CRM_LOG
}

}  // namespace crm
