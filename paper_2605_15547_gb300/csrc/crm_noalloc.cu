// crm_noalloc.cu -- crm_eval_noalloc: the same evaluation as crm_eval_form, with its
// scratch memory (workspace counters and hard-case queue) in a statically reserved
// device array instead of memory the library allocates on first use.
//
// Who needs it: code that must not allocate device memory when it calls the library --
// work recorded under stream capture (cudaMalloc is not permitted while a stream is
// being captured), serving processes that budget every device byte at start-up and
// forbid allocation afterwards, and callers running inside another component's memory
// manager that owns all allocation.  The caller still provides the input and output.
//
// The array below is created when the library is loaded and every GPU that loads the
// library keeps it until the process exits.  It is sized so that every lane of the
// largest accepted call fits in the queue.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/crm.h"
#include "crm_internal.h"

namespace crm {

constexpr uint64_t kNoAllocMaxElems = CRM_NOALLOC_MAX_ELEMS;
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocBytes = kNoAllocHeader + kNoAllocMaxElems * sizeof(crm_queue_entry);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Per-device set-up, done once with the device current: the device address of the
// array (the host-side symbol is only a stand-in and must never reach a kernel) and the
// SM count.  Fixed-size host table, so set-up allocates nothing either.
struct NoAllocDevice {
  unsigned char *scratch;
  int sms;
  int ready;
};
static NoAllocDevice g_nadev[128];
static std::mutex g_namu;

static int noalloc_setup(NoAllocDevice **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail_code(e);
  if (dev < 0 || dev >= 128) return CRM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_namu);
  NoAllocDevice &d = g_nadev[dev];
  if (!d.ready) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail_code(e);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail_code(e);
    d.scratch = (unsigned char *)p;
    d.sms = sms > 0 ? sms : 1;
    d.ready = 1;
  }
  *out = &d;
  return CRM_OK;
}

}  // namespace crm

using namespace crm;

extern "C" int crm_eval_noalloc(int func_id, int dtype, int form, const void *in, void *out,
                                uint64_t n, void *stream) {
  ensure_init();
  int st = check_args(func_id, dtype, in, out, n);
  if (st) return st;
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  const FuncEntry &fe = func_entry(func_id);
  int fm = resolve_form(fe, form);
  if (fm < 0) return CRM_ERR_FORM;
  if (n == 0) return CRM_OK;
  if (n > kNoAllocMaxElems) return CRM_ERR_SIZE;
  NoAllocDevice *d = nullptr;
  st = noalloc_setup(&d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  KArgs a;
  int vi = variant_of(func_id, fm);
  if (!fill_geometry(fe, in, out, n, a, VARIANTS[vi].vec_bytes) && VARIANTS[vi].vec_bytes != 16) {
    vi = DEFAULT_VARIANT;
    fill_geometry(fe, in, out, n, a, 16);
  }
  a.hdr = (crm_ws_header *)d->scratch;
  a.q = (crm_queue_entry *)(d->scratch + kNoAllocHeader);
  a.cap = kNoAllocMaxElems;
  a.qcount = &a.hdr->count;  // one queue: every lane of a call fits in it
  a.nsubq = 1;
  a.force_hard = force_slow_flag();
  a.desc = 0;
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fe.main_sym[fm][vi], VARIANTS[vi].block, 0);
  if (e != cudaSuccess) return cuda_fail_code(e);
  int grid = main_grid(fe, a, vi, d->sms, bps > 0 ? bps : 1);
  // The array keeps the previous call's contents: the queue count must start at zero.
  e = cudaMemsetAsync(&a.hdr->count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  e = fe.main[fm][vi](a, grid, s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  e = fe.slow(a, d->sms * 2, s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  return CRM_OK;
}

// Counters of the static scratch of the current device (the header of
// g_noalloc_scratch, which every crm_eval_noalloc call on the device adds to).  Reading
// them allocates nothing either: one small copy into the caller's struct.
extern "C" int crm_noalloc_stats(void *stream, crm_stats_t *out) {
  ensure_init();
  if (!out) return CRM_ERR_NULL;
  NoAllocDevice *d = nullptr;
  int st = noalloc_setup(&d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  crm_ws_header h;
  cudaError_t e = cudaMemcpyAsync(&h, d->scratch, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  out->hard_total = h.hard_total;
  out->unresolved_total = h.unresolved_total;
  out->inline_total = h.inline_total;
  out->last_count = h.count;
  out->timeouts = h.timeouts;
  out->fp64_total = h.fp64_total;
  return CRM_OK;
}

extern "C" int crm_noalloc_stats_reset(void *stream) {
  ensure_init();
  NoAllocDevice *d = nullptr;
  int st = noalloc_setup(&d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(d->scratch, 0, sizeof(crm_ws_header), s);
  if (e != cudaSuccess) return cuda_fail_code(e);
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? CRM_OK : cuda_fail_code(e);
}
