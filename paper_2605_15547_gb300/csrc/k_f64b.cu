// k_f64b.cu -- more binary64 functions: e^x, log2, log10, 10^x (FP64-free main path on the
// fixed-point cores, exact 192-bit slow path).
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_f64b(FuncEntry *t) {
  set_entry_default<FnExpBD<0>>(t[21]);  // CRM_EXP
  set_entry_default<FnLogBD<1>>(t[22]);  // CRM_LOG2
  set_entry_default<FnLogBD<2>>(t[23]);  // CRM_LOG10
  set_entry_default<FnExpBD<2>>(t[24]);  // CRM_EXP10
}

}  // namespace crm
