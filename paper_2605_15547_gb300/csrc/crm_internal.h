// crm_internal.h -- runtime helpers shared between the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include "crm_registry.h"

namespace crm {
void ensure_init();
const FuncEntry &func_entry(int func);
int resolve_form(const FuncEntry &fe, int form);
int check_args(int func, int dtype, const void *in, void *out, uint64_t n);
int variant_of(int func, int form);
int main_blocks_per_sm(const FuncEntry &fe, int form, int vi);
int force_slow_flag();
int cuda_fail_code(cudaError_t e);
// Head/vector split for vb-byte vectors; false (everything scalar) unless in and out are
// vb-byte congruent (and the second output row too).
bool fill_geometry(const FuncEntry &fe, const void *in, void *out, uint64_t n, KArgs &a, int vb);
int main_grid(const FuncEntry &fe, const KArgs &a, int vi, int sms, int bps);
}  // namespace crm
