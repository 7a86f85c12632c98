// k_atrig.cu -- atanf, asinf, acosf, rsqrtf kernels.
#include "crm_registry.h"
#include "fam_atrig.cuh"
#include "fam_rsqrt.cuh"

namespace crm {

template <int KIND> struct FnAtrig {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 18 * 8; }
  template <int FORM> CRM_DEV static void load(unsigned char *sm) { copy_tab(sm, CRM_ATAN_T17_D, 18 * 8); }
  template <int FORM> CRM_DEV static void eval(float x, const void *sm, float *y, bool &h) {
    y[0] = atrig_plain<KIND>(x, (const double *)sm, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = atrig_slow<KIND>(x, u); }
};

struct FnRsqrt {
  using T = float;
  static constexpr int NOUT = 1;
  template <int FORM> static constexpr int tab_bytes() { return 0; }
  template <int FORM> CRM_DEV static void load(unsigned char *) {}
  template <int FORM> CRM_DEV static void eval(float x, const void *, float *y, bool &h) {
    y[0] = FORM == 1 ? rsqrt_plain(x, h) : rsqrt_df(x, h);
  }
  CRM_DEV static void slow(float x, float *y, bool &u) { y[0] = rsqrt_slow(x, u); }
};

void register_atrig(FuncEntry *t) {
  set_entry<FnAtrig<AT_ASIN>, true, false>(t[12]);  // CRM_ASINF
  set_entry<FnAtrig<AT_ACOS>, true, false>(t[13]);  // CRM_ACOSF
  set_entry<FnAtrig<AT_ATAN>, true, false>(t[14]);  // CRM_ATANF
  set_entry<FnRsqrt, true, true>(t[18]);           // CRM_RSQRTF
}

}  // namespace crm
