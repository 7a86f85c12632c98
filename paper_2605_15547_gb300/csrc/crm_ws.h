// crm_ws.h -- device workspace layout shared by the runtime and the kernels.
#pragma once
#include <stdint.h>

// Header at the start of each workspace.  `count` is cleared before every call; the
// totals accumulate until crm_stats_reset().
typedef struct crm_ws_header {
  unsigned long long count;            // lanes that failed the fast-path test this call
  unsigned long long hard_total;       // sum of count over calls
  unsigned long long unresolved_total; // lanes no tier could decide (never expected)
  unsigned long long inline_total;     // lanes finished inline because the queue was full
  unsigned long long timeouts;         // bounded waits that gave up (never expected)
  unsigned long long pad[3];
} crm_ws_header;

// One queued hard lane: element index (array id in bits 40..63 for the batch form) and
// the input's bit pattern (kept so that in-place calls still see the original input).
typedef struct crm_queue_entry {
  uint64_t idx;
  uint64_t x;
} crm_queue_entry;
