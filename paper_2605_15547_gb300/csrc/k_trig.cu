// k_trig.cu -- sinf, cosf, sincosf, tanf kernels.
#include "crm_fns.cuh"
#include "crm_registry.h"

namespace crm {

void register_trig(FuncEntry *t) {
  set_entry<FnTrig<TRIG_SIN>, true, true>(t[8]);      // CRM_SINF
  set_entry<FnTrig<TRIG_COS>, true, true>(t[9]);      // CRM_COSF
  set_entry<FnTrig<TRIG_SINCOS>, true, true>(t[10]);  // CRM_SINCOSF
  set_entry<FnTrig<TRIG_TAN>, true, true>(t[11]);     // CRM_TANF
}

}  // namespace crm
