// crm_registry.h -- launchers exported by each family's translation unit.
#pragma once
#include <cuda_runtime.h>

#include "crm_kernels.cuh"

namespace crm {

typedef cudaError_t (*launch_fn)(const KArgs &, int grid, cudaStream_t);
typedef int (*occ_fn)(void);

enum { NUNROLL = 4 };  // variants: unroll 1, 2, 4 (vectors in flight per thread), 3 = pipelined

struct FuncEntry {
  launch_fn main[3][NUNROLL];  // [form][unroll]; form 0 unused; null when unavailable
  const void *main_sym[3][NUNROLL];
  launch_fn slow;
  int nout;   // 1, or 2 for sincosf
  int dtype;  // 0 binary32, 1 binary64
};

template <class Fn, int FORM, int U>
cudaError_t launch_main(const KArgs &a, int grid, cudaStream_t s) {
  k_main<Fn, FORM, U><<<grid, KBLOCK, 0, s>>>(a);
  return cudaGetLastError();
}
template <class Fn>
cudaError_t launch_slow(const KArgs &a, int grid, cudaStream_t s) {
  k_slow<Fn><<<grid, KBLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Fn, int FORM>
cudaError_t launch_pipe(const KArgs &a, int grid, cudaStream_t s) {
  k_pipe<Fn, FORM><<<grid, KBLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Fn, int FORM>
void set_form(FuncEntry &e) {
  e.main[FORM][0] = launch_main<Fn, FORM, 1>;
  e.main[FORM][1] = launch_main<Fn, FORM, 2>;
  e.main[FORM][2] = launch_main<Fn, FORM, 4>;
  e.main[FORM][3] = launch_pipe<Fn, FORM>;
  e.main_sym[FORM][0] = (const void *)k_main<Fn, FORM, 1>;
  e.main_sym[FORM][1] = (const void *)k_main<Fn, FORM, 2>;
  e.main_sym[FORM][2] = (const void *)k_main<Fn, FORM, 4>;
  e.main_sym[FORM][3] = (const void *)k_pipe<Fn, FORM>;
}

template <class Fn, bool HAS_PLAIN, bool HAS_DF>
void set_entry(FuncEntry &e) {
  e = FuncEntry();
  if (HAS_PLAIN) set_form<Fn, 1>(e);
  if (HAS_DF) set_form<Fn, 2>(e);
  e.slow = launch_slow<Fn>;
  e.nout = Fn::NOUT;
  e.dtype = sizeof(typename Fn::T) == 8 ? 1 : 0;
}

// one per family translation unit
void register_exp(FuncEntry *table);
void register_log(FuncEntry *table);
void register_hyp(FuncEntry *table);
void register_trig(FuncEntry *table);
void register_atrig(FuncEntry *table);
void register_f64(FuncEntry *table);

}  // namespace crm
