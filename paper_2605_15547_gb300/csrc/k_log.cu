// k_log.cu -- logf, log2f, log10f, log1pf kernels (all tiers).
#include "crm_registry.h"
#include "fam_log.cuh"

namespace crm {

template <int KIND> struct FnLog {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 97 * 16; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) {
    copy_tab(sm, FORM == 1 ? (const void *)CRM_LN_T97_D : (const void *)log_tab_df<KIND>(), tab_bytes<FORM>());
  }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    if (FORM == 1)
      y[0] = log_plain<KIND>(x, (const double2 *)sm, h);
    else
      y[0] = log_df<KIND>(x, (const float4 *)sm, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = log_slow<KIND>(x, u); }
};

void register_log(FuncEntry *t) {
  set_entry<FnLog<0>, true, true>(t[4]);  // CRM_LOGF
  set_entry<FnLog<1>, true, true>(t[5]);  // CRM_LOG2F
  set_entry<FnLog<2>, true, true>(t[6]);  // CRM_LOG10F
  set_entry<FnLog<3>, true, true>(t[7]);  // CRM_LOG1PF
}

}  // namespace crm
