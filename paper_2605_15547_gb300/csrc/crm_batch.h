// crm_batch.h -- device descriptors of the batching form.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "crm_ws.h"

namespace crm {

// One array of a batch, as the kernels see it (32 bytes).
struct BatchDesc {
  const void *in;
  void *out;
  uint64_t n;
  uint64_t tile0;  // index of the array's first tile in the whole batch
  int32_t func;
  int32_t flags;   // bit 0: input and output(s) 16-byte aligned (vector loop allowed)
};

struct BatchArgs {
  const BatchDesc *descs;
  int count;
  int tile_shift;           // tiles of 2^tile_shift elements
  uint64_t total_tiles;
  uint64_t tiles_per_block;
  crm_ws_header *hdr;
  crm_queue_entry *q;
  uint64_t cap;
  unsigned long long *qcount;  // sub-queue counters (see crm_ws.h)
  int nsubq;
  int force_hard;
  uint32_t aid_base;  // index of descs[0] in the whole batch (grouped mode)
};

// Mixed mode: one kernel over all arrays (function switch per tile) + the slow pass.
cudaError_t launch_batch(const BatchArgs &b, int form, int grid, int slow_grid, cudaStream_t s);
const void *batch_kernel_symbol(int form);
// Grouped mode: one kernel specialised for `func` over that function's arrays; the slow
// pass runs once after all groups (launch_batch_slow, descs = the whole batch).  easy: the
// kernel packs the elements that need the evaluator across the warp (as the main kernel's
// packing shapes; functions without easy arguments ignore it).
cudaError_t launch_batch_group(int func, const BatchArgs &b, int form, int grid, cudaStream_t s, bool easy);
const void *batch_group_symbol(int func, int form, bool easy);
cudaError_t launch_batch_slow(const BatchArgs &b, int slow_grid, cudaStream_t s);

}  // namespace crm
