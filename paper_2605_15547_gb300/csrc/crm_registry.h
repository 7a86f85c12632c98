// crm_registry.h -- launchers exported by each family's translation unit.
#pragma once
#include <cuda_runtime.h>

#include "crm_kernels.cuh"

namespace crm {

typedef cudaError_t (*launch_fn)(const KArgs &, int grid, cudaStream_t);
typedef int (*occ_fn)(void);

// Launch shapes of the main kernel that the autotuner chooses among: vectors per thread
// per iteration, threads per block, register prefetch of the next iteration, a register
// cap (minimum resident blocks), the vector width (16- or 32-byte accesses: 4 or 8
// binary32 elements), or the shared-memory pipelined kernel.
struct VariantInfo {
  int unroll, block, prefetch, pipelined, min_blocks, vec_bytes;
};
enum { NVARIANT = 10, DEFAULT_VARIANT = 1 };
constexpr VariantInfo VARIANTS[NVARIANT] = {
    {1, 256, 0, 0, 1, 16}, {2, 256, 0, 0, 1, 16}, {4, 256, 0, 0, 1, 16}, {PVPT, KBLOCK, 0, 1, 1, 16},
    {2, 256, 1, 0, 4, 16}, {1, 256, 1, 0, 1, 16}, {2, 128, 1, 0, 1, 16}, {2, 512, 1, 0, 1, 16},
    {1, 256, 1, 0, 1, 32}, {1, 512, 1, 0, 1, 32}};

struct FuncEntry {
  launch_fn main[3][NVARIANT];  // [form][variant]; form 0 unused; null when unavailable
  const void *main_sym[3][NVARIANT];
  launch_fn slow;
  int nout;   // 1, or 2 for sincosf
  int dtype;  // 0 binary32, 1 binary64
};

template <class Fn, int FORM, int U, int BS, bool PF, bool WIDE>
cudaError_t launch_main(const KArgs &a, int grid, cudaStream_t s) {
  k_main<Fn, FORM, U, BS, PF, WIDE><<<grid, BS, 0, s>>>(a);
  return cudaGetLastError();
}
template <class Fn, int FORM, int U, int BS, bool PF, int MINB>
cudaError_t launch_main_capped(const KArgs &a, int grid, cudaStream_t s) {
  k_main_capped<Fn, FORM, U, BS, PF, MINB><<<grid, BS, 0, s>>>(a);
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

template <class Fn, int FORM, int V>
void set_variant(FuncEntry &e) {
  constexpr VariantInfo I = VARIANTS[V];
  if constexpr (I.pipelined) {
    e.main[FORM][V] = launch_pipe<Fn, FORM>;
    e.main_sym[FORM][V] = (const void *)k_pipe<Fn, FORM>;
  } else if constexpr (I.min_blocks > 1) {
    e.main[FORM][V] = launch_main_capped<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.min_blocks>;
    e.main_sym[FORM][V] = (const void *)k_main_capped<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.min_blocks>;
  } else {
    e.main[FORM][V] = launch_main<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.vec_bytes == 32>;
    e.main_sym[FORM][V] = (const void *)k_main<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.vec_bytes == 32>;
  }
}

// The double-float form gets every launch shape; the plain FP64 form, bound by the FP64
// pipe whatever the shape, only the default one.
template <class Fn, int FORM>
void set_form(FuncEntry &e) {
  set_variant<Fn, FORM, DEFAULT_VARIANT>(e);
  if constexpr (FORM == 2) {
    set_variant<Fn, FORM, 0>(e);
    set_variant<Fn, FORM, 2>(e);
    set_variant<Fn, FORM, 3>(e);
    set_variant<Fn, FORM, 4>(e);
    set_variant<Fn, FORM, 5>(e);
    set_variant<Fn, FORM, 6>(e);
    set_variant<Fn, FORM, 7>(e);
    set_variant<Fn, FORM, 8>(e);
    set_variant<Fn, FORM, 9>(e);
  }
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
