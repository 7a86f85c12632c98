// crm_ws.h -- device workspace layout shared by the runtime and the kernels.
#pragma once
#include <stdint.h>

// Header at the start of each workspace.  The totals accumulate until crm_stats_reset();
// `count` is the last call's number of hard lanes.
typedef struct crm_ws_header {
  unsigned long long count;            // lanes that failed the fast-path test this call
  unsigned long long hard_total;       // sum of count over calls
  unsigned long long unresolved_total; // lanes no tier could decide (never expected)
  unsigned long long inline_total;     // lanes finished inline because the queue was full
  unsigned long long timeouts;         // bounded waits that gave up (never expected)
  unsigned long long fp64_total;       // queued lanes whose slow path ran an FP64 tier
  unsigned long long pad[2];
} crm_ws_header;

// One queued hard lane: element index (array id in bits 40..63 for the batch form) and
// the input's bit pattern (kept so that in-place calls still see the original input).
typedef struct crm_queue_entry {
  uint64_t idx;
  uint64_t x;
} crm_queue_entry;

// The hard-case queue is split into CRM_NSUBQ sub-queues of equal capacity, each with its
// own counter on its own 128-byte line (so that the warps' atomicAdds spread over many
// addresses instead of serialising on one); warp w of the grid uses sub-queue
// w % CRM_NSUBQ.  The counters follow the header at byte offset CRM_SUBQ_OFFSET and are
// cleared before every call.
#define CRM_NSUBQ 64
#define CRM_SUBQ_STRIDE 16  /* unsigned long longs between counters: 128 bytes */
#define CRM_SUBQ_OFFSET 128
#define CRM_WS_HEADER_BYTES (CRM_SUBQ_OFFSET + CRM_NSUBQ * CRM_SUBQ_STRIDE * 8)
