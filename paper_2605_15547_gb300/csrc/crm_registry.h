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
// binary32 elements), the shared-memory pipelined kernel, or (reg_table) the evaluator
// variant whose table of at most 16 entries lives in registers and is read by warp
// shuffles instead of shared-memory loads (the exp family), or (easy) the main kernel
// that packs the elements needing the evaluator across the warp (eval_vecs, functions
// with easy arguments only).
struct VariantInfo {
  int unroll, block, prefetch, pipelined, min_blocks, vec_bytes, reg_table, easy;
};
enum { NVARIANT = 13, DEFAULT_VARIANT = 1, REGTAB_VARIANT = 10 };
constexpr VariantInfo VARIANTS[NVARIANT] = {
    {1, 256, 0, 0, 1, 16, 0, 0}, {2, 256, 0, 0, 1, 16, 0, 0}, {4, 256, 0, 0, 1, 16, 0, 0},
    {PVPT, KBLOCK, 0, 1, 1, 16, 0, 0}, {2, 256, 1, 0, 4, 16, 0, 0}, {1, 256, 1, 0, 1, 16, 0, 0},
    {2, 128, 1, 0, 1, 16, 0, 0}, {2, 512, 1, 0, 1, 16, 0, 0}, {1, 256, 1, 0, 1, 32, 0, 0},
    {1, 512, 1, 0, 1, 32, 0, 0}, {2, 512, 1, 0, 1, 16, 1, 0}, {1, 512, 1, 0, 1, 32, 0, 1},
    {2, 512, 1, 0, 1, 16, 0, 1}};

// The packing shapes are shapes 9 and 7 with packing (host-memory calls map them back).
constexpr bool same_shape(const VariantInfo &a, const VariantInfo &b) {
  return a.unroll == b.unroll && a.block == b.block && a.prefetch == b.prefetch && a.pipelined == b.pipelined &&
         a.min_blocks == b.min_blocks && a.vec_bytes == b.vec_bytes && a.reg_table == b.reg_table;
}
static_assert(same_shape(VARIANTS[11], VARIANTS[9]) && same_shape(VARIANTS[12], VARIANTS[7]) &&
                  VARIANTS[11].easy && VARIANTS[12].easy && !VARIANTS[9].easy && !VARIANTS[7].easy,
              "packing shapes 11 and 12 are shapes 9 and 7 with packing");

struct FuncEntry {
  launch_fn main[3][NVARIANT];  // [form][variant]; form 0 unused; null when unavailable
  const void *main_sym[3][NVARIANT];
  launch_fn slow;
  launch_fn dmain, dslow;  // directed rounding and 16-bit formats (k_dir, k_dir_slow)
  const void *dmain_sym;
  int nout;   // 1, or 2 for sincosf
  int dtype;  // 0 binary32, 1 binary64
};

template <class Fn, int FORM, int U, int BS, bool PF, bool WIDE, bool EASY = false>
cudaError_t launch_main(const KArgs &a, int grid, cudaStream_t s) {
  k_main<Fn, FORM, U, BS, PF, WIDE, EASY><<<grid, BS, 0, s>>>(a);
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

template <class Fn>
cudaError_t launch_dir(const KArgs &a, int grid, cudaStream_t s) {
  k_dir<Fn><<<grid, KBLOCK, 0, s>>>(a);
  return cudaGetLastError();
}
template <class Fn>
cudaError_t launch_dir_slow(const KArgs &a, int grid, cudaStream_t s) {
  k_dir_slow<Fn><<<grid, KBLOCK, 0, s>>>(a);
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
    e.main[FORM][V] = launch_main<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.vec_bytes == 32, (bool)I.easy>;
    e.main_sym[FORM][V] =
        (const void *)k_main<Fn, FORM, I.unroll, I.block, (bool)I.prefetch, I.vec_bytes == 32, (bool)I.easy>;
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
    if constexpr (EasyOf<Fn>::value) {
      set_variant<Fn, FORM, 11>(e);
      set_variant<Fn, FORM, 12>(e);
    }
  }
}

// The register-table evaluator FnR of the same function, in the FP64-free form's slot
// REGTAB_VARIANT (the shape of VARIANTS[REGTAB_VARIANT]).
template <class FnR>
void set_regtab_variant(FuncEntry &e) {
  constexpr VariantInfo I = VARIANTS[REGTAB_VARIANT];
  e.main[2][REGTAB_VARIANT] = launch_main<FnR, 2, I.unroll, I.block, (bool)I.prefetch, false>;
  e.main_sym[2][REGTAB_VARIANT] = (const void *)k_main<FnR, 2, I.unroll, I.block, (bool)I.prefetch, false>;
}

template <class Fn, bool HAS_PLAIN, bool HAS_DF>
void set_entry(FuncEntry &e) {
  e = FuncEntry();
  if constexpr (HAS_PLAIN) set_form<Fn, 1>(e);
  if constexpr (HAS_DF) set_form<Fn, 2>(e);
  e.slow = launch_slow<Fn>;
  e.dmain = launch_dir<Fn>;
  e.dslow = launch_dir_slow<Fn>;
  e.dmain_sym = (const void *)k_dir<Fn>;
  e.nout = Fn::NOUT;
  e.dtype = sizeof(typename Fn::T) == 8 ? 1 : 0;
}

// A function with the FP64-free form in the default launch shape only (fewer kernels to
// build for the later binary64 functions).
template <class Fn>
void set_entry_default(FuncEntry &e) {
  e = FuncEntry();
  set_variant<Fn, 2, DEFAULT_VARIANT>(e);
  e.slow = launch_slow<Fn>;
  e.dmain = launch_dir<Fn>;
  e.dslow = launch_dir_slow<Fn>;
  e.dmain_sym = (const void *)k_dir<Fn>;
  e.nout = Fn::NOUT;
  e.dtype = 1;
}

// one per family translation unit
void register_exp(FuncEntry *table);
void register_log(FuncEntry *table);
void register_hyp(FuncEntry *table);
void register_trig(FuncEntry *table);
void register_atrig(FuncEntry *table);
void register_f64(FuncEntry *table);
void register_f64b(FuncEntry *table);

}  // namespace crm
