// crm_runtime.cu -- the C ABI of include/crm.h: argument checks, per-(device, stream)
// workspaces, launch configuration, the host-buffer and batch entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/crm.h"
#include "crm_batch.h"
#include "crm_internal.h"
#include "crm_registry.h"

namespace crm {

static FuncEntry g_table[CRM_NUM_FUNCS];
static std::once_flag g_init_once;
// Process-wide settings: plain atomics, so that a setter racing with calls on other
// threads is well defined (a call sees either the old or the new value).
static std::atomic<int> g_default_form{CRM_FORM_AUTO};
static std::atomic<int> g_force_slow{0};
static thread_local int g_last_cuda = 0;

static void init_table() {
  memset(g_table, 0, sizeof(g_table));
  register_exp(g_table);
  register_log(g_table);
  register_hyp(g_table);
  register_trig(g_table);
  register_atrig(g_table);
  register_f64(g_table);
  register_f64b(g_table);
  const char *f = getenv("CRM_FORM");
  if (f) {
    if (!strcmp(f, "plain")) g_default_form = CRM_FORM_PLAIN_FP64;
    if (!strcmp(f, "df")) g_default_form = CRM_FORM_DF32;
  }
  const char *fs = getenv("CRM_FORCE_SLOW");
  if (fs && atoi(fs)) g_force_slow = 1;
}
void ensure_init() { std::call_once(g_init_once, init_table); }
const FuncEntry &func_entry(int func) { return g_table[func]; }
int force_slow_flag() { return g_force_slow; }
int cuda_fail_code(cudaError_t e) {
  g_last_cuda = (int)e;
  return CRM_ERR_CUDA;
}

// ------------------------------------------------------------------ workspaces
struct Workspace {
  crm_ws_header *hdr = nullptr;  // device
  crm_queue_entry *q = nullptr;  // device
  uint64_t cap = 0;
  // batching form: device descriptors and their page-locked host staging copy
  BatchDesc *bdesc = nullptr;
  BatchDesc *bstage = nullptr;
  int bcap = 0;
  cudaEvent_t bcopied = nullptr;  // the last descriptor upload has completed
  // A captured batch call re-reads bstage and rewrites bdesc at every replay of its
  // graph: the capture takes both buffers for itself (bcaptured), and the next batch
  // call outside capture, or crm_reserve, gives the workspace new ones.  The captured
  // pairs stay allocated until crm_shutdown.
  bool bcaptured = false;
  std::vector<std::pair<BatchDesc *, BatchDesc *>> retired;
  std::vector<crm_queue_entry *> retired_q;  // queues replaced by a larger one
};

struct DevInfo {
  int sms = 0;
  std::map<const void *, int> occ;  // kernel symbol -> resident blocks per SM
};

static std::mutex g_mu;
static std::map<std::pair<int, uintptr_t>, Workspace> g_ws;
static std::map<int, DevInfo> g_dev;

static const uint64_t kDefaultCap = 1ull << 21;  // 2M hard lanes (32 MiB) per workspace

static unsigned long long *subq_counts(Workspace *w) {
  return (unsigned long long *)((char *)w->hdr + CRM_SUBQ_OFFSET);
}

static int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return CRM_ERR_CUDA;
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// Workspace of (current device, stream) with at least `cap` queue entries.
static int get_ws(cudaStream_t s, uint64_t cap, Workspace **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace &w = g_ws[{dev, (uintptr_t)s}];
  if (w.hdr && w.cap >= cap) {
    *out = &w;
    return CRM_OK;
  }
  if (capturing(s)) return CRM_ERR_CAPTURE;
  if (w.hdr) {  // grow: keep the header (counters), replace the queue
    // a CUDA graph captured earlier may still address the old queue: keep it allocated
    // until crm_shutdown instead of freeing it
    w.retired_q.push_back(w.q);
    w.q = nullptr;
  } else {
    e = cudaMalloc((void **)&w.hdr, CRM_WS_HEADER_BYTES);
    if (e != cudaSuccess) {
      w.hdr = nullptr;
      return e == cudaErrorMemoryAllocation ? CRM_ERR_NOMEM : cuda_fail(e);
    }
    e = cudaMemset(w.hdr, 0, CRM_WS_HEADER_BYTES);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = cudaMalloc((void **)&w.q, cap * sizeof(crm_queue_entry));
  if (e != cudaSuccess) {
    w.q = nullptr;
    w.cap = 0;
    return e == cudaErrorMemoryAllocation ? CRM_ERR_NOMEM : cuda_fail(e);
  }
  w.cap = cap;
  *out = &w;
  return CRM_OK;
}

static int dev_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo &d = g_dev[dev];
  if (!d.sms) {
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || d.sms <= 0)
      d.sms = 1;
  }
  return d.sms;
}

static int blocks_per_sm(const void *sym, int block) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo &d = g_dev[dev];
  auto it = d.occ.find(sym);
  if (it != d.occ.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sym, block, 0) != cudaSuccess || nb <= 0) nb = 1;
  d.occ[sym] = nb;
  return nb;
}

// Launch shape per (function, form): the default, the env CRM_VARIANT, crm_set_variant
// or the autotuner's choice.  A shape the form does not provide falls back to the default.
static std::atomic<int> g_variant[CRM_NUM_FUNCS][3];
static std::once_flag g_variant_once;

static void variant_init() {
  int def = DEFAULT_VARIANT;
  const char *u = getenv("CRM_VARIANT");
  if (u && atoi(u) >= 0 && atoi(u) < NVARIANT) def = atoi(u);
  for (int f = 0; f < CRM_NUM_FUNCS; f++)
    for (int m = 0; m < 3; m++) g_variant[f][m] = def;
}

int variant_of(int func, int form) {
  std::call_once(g_variant_once, variant_init);
  int v = g_variant[func][form];
  return g_table[func].main[form][v] ? v : DEFAULT_VARIANT;
}

static void set_variant_of(int func, int form, int v) {
  std::call_once(g_variant_once, variant_init);
  g_variant[func][form] = v;
}

int resolve_form(const FuncEntry &fe, int form) {
  if (form == CRM_FORM_AUTO) {
    if (fe.main[CRM_FORM_DF32][DEFAULT_VARIANT]) return CRM_FORM_DF32;
    if (fe.main[CRM_FORM_PLAIN_FP64][DEFAULT_VARIANT]) return CRM_FORM_PLAIN_FP64;
    return -1;
  }
  if (form != CRM_FORM_PLAIN_FP64 && form != CRM_FORM_DF32) return -1;
  return fe.main[form][DEFAULT_VARIANT] ? form : -1;
}

int check_args(int func, int dtype, const void *in, void *out, uint64_t n) {
  if (func < 0 || func >= CRM_NUM_FUNCS) return CRM_ERR_FUNC;
  const FuncEntry &fe = g_table[func];
  int want = func >= CRM_EXP2 ? CRM_F64 : CRM_F32;
  if (dtype != CRM_F32 && dtype != CRM_F64) return CRM_ERR_DTYPE;
  if (dtype != want) return CRM_ERR_DTYPE;
  if (n == 0) return CRM_OK;
  if (!in || !out) return CRM_ERR_NULL;
  size_t es = dtype == CRM_F64 ? 8 : 4;
  if (((uintptr_t)in % es) || ((uintptr_t)out % es)) return CRM_ERR_ARG;
  if (n > (1ull << 40)) return CRM_ERR_ARG;
  uintptr_t a0 = (uintptr_t)in, a1 = a0 + n * es;
  uintptr_t b0 = (uintptr_t)out, b1 = b0 + n * es * (func == CRM_SINCOSF ? 2 : 1);
  if (a0 != b0 && a0 < b1 && b0 < a1) return CRM_ERR_OVERLAP;
  (void)fe;
  return CRM_OK;
}

// Vector geometry: the vector loop needs input and output(s) at the same offset modulo
// 16 bytes; the scalar loop covers the unaligned head and the tail.
bool fill_geometry(const FuncEntry &fe, const void *in, void *out, uint64_t n, KArgs &a, int vb) {
  const size_t es = fe.dtype ? 8 : 4;
  const int W = vb / (int)es;
  a.in = in;
  a.out = out;
  a.n = n;
  uintptr_t ia = (uintptr_t)in, oa = (uintptr_t)out;
  bool vec = ((ia - oa) % vb) == 0 && (fe.nout == 1 || (n * es) % vb == 0);
  if (vec) {
    uint64_t head = ((vb - ia % vb) % vb) / es;
    if (head > n) head = n;
    a.head = head;
    a.nvec = (n - head) / W;
  } else {
    a.head = 0;
    a.nvec = 0;
  }
  return vec;
}

// Grid of the main kernel: enough blocks for the work, at most one full wave of
// resident blocks (the kernel loops over the rest).
int main_grid(const FuncEntry &fe, const KArgs &a, int vi, int sms, int bps) {
  const int W = VARIANTS[vi].vec_bytes / (fe.dtype ? 8 : 4);
  const uint64_t U = (uint64_t)VARIANTS[vi].unroll, B = (uint64_t)VARIANTS[vi].block;
  uint64_t want = (a.nvec + B * U - 1) / (B * U);
  uint64_t nscal = a.head + (a.n - a.head - (uint64_t)W * a.nvec);
  uint64_t want_s = (nscal + B - 1) / B;
  if (want_s > want) want = want_s;
  uint64_t cap_blocks = (uint64_t)sms * bps;
  return (int)(want < cap_blocks ? (want ? want : 1) : cap_blocks);
}

int main_blocks_per_sm(const FuncEntry &fe, int form, int vi) {
  return blocks_per_sm(fe.main_sym[form][vi], VARIANTS[vi].block);
}

// Enqueue one evaluation (arguments already checked, n > 0).
static int enqueue(int func, int form, const void *in, void *out, uint64_t n, cudaStream_t s,
                   uint32_t desc, int variant = -1) {
  const FuncEntry &fe = g_table[func];
  int fm = resolve_form(fe, form);
  if (fm < 0) return CRM_ERR_FORM;
  Workspace *w = nullptr;
  int st = get_ws(s, kDefaultCap, &w);
  if (st) return st;
  KArgs a;
  int vi = variant >= 0 ? variant : variant_of(func, fm);
  // a 32-byte shape needs in and out 32-byte congruent; else the default 16-byte shape
  if (!fill_geometry(fe, in, out, n, a, VARIANTS[vi].vec_bytes) && VARIANTS[vi].vec_bytes != 16) {
    vi = DEFAULT_VARIANT;
    fill_geometry(fe, in, out, n, a, 16);
  }
  a.hdr = w->hdr;
  a.q = w->q;
  a.cap = w->cap;
  a.qcount = subq_counts(w);
  a.nsubq = CRM_NSUBQ;
  a.force_hard = g_force_slow;
  a.desc = desc;
  int sms = dev_sms();
  int grid = main_grid(fe, a, vi, sms, main_blocks_per_sm(fe, fm, vi));
  cudaError_t e = cudaMemsetAsync(a.qcount, 0, CRM_NSUBQ * CRM_SUBQ_STRIDE * 8, s);
  if (e != cudaSuccess) return cuda_fail(e);
  e = fe.main[fm][vi](a, grid, s);
  if (e != cudaSuccess) return cuda_fail(e);
  e = fe.slow(a, sms * 2, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return CRM_OK;
}

// ------------------------------------------------------------------ batch buffers
static std::atomic<int> g_batch_tile_shift{14};  // the autotuner may change it (crm_set_batch_tile)
static std::atomic<int> g_batch_mode{CRM_BATCH_GROUPED};  // crm_set_batch_mode / the autotuner

static int batch_buffers(cudaStream_t s, Workspace *w, int count) {
  if (w->bcap >= count && !w->bcaptured) return CRM_OK;
  if (capturing(s)) return CRM_ERR_CAPTURE;
  cudaError_t e;
  int want = count < 1024 ? 1024 : count;
  if (w->bcaptured) {
    // a graph owns the current pair: keep it for that graph, start a new one
    w->retired.push_back({w->bdesc, w->bstage});
    if (want < w->bcap) want = w->bcap;
    w->bdesc = nullptr;
    w->bstage = nullptr;
    w->bcap = 0;
    w->bcaptured = false;
  } else if (w->bdesc) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaFree(w->bdesc);
    cudaFreeHost(w->bstage);
    w->bdesc = nullptr;
    w->bstage = nullptr;
    w->bcap = 0;
  }
  if (cudaMalloc((void **)&w->bdesc, (size_t)want * sizeof(BatchDesc)) != cudaSuccess) return CRM_ERR_NOMEM;
  if (cudaMallocHost((void **)&w->bstage, (size_t)want * sizeof(BatchDesc)) != cudaSuccess) return CRM_ERR_NOMEM;
  if (!w->bcopied) {
    e = cudaEventCreateWithFlags(&w->bcopied, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  w->bcap = want;
  return CRM_OK;
}

// ------------------------------------------------------------------ host-buffer path
// Chunks of the host array go through two internal streams: while one stream computes a
// chunk, the copy engines move the neighbouring chunks in and out (H2D and D2H overlap
// with compute and with each other).
struct HostStage {
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t ev = nullptr;
  void *din[2] = {nullptr, nullptr}, *dout[2] = {nullptr, nullptr};
  size_t bytes = 0;  // per input buffer
};
static std::map<int, HostStage> g_stage;
static const uint64_t kChunkElems = 1ull << 22;

static int host_pipeline(int func, int form, const void *in, void *out, uint64_t n, cudaStream_t user) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  const FuncEntry &fe = g_table[func];
  const size_t es = fe.dtype ? 8 : 4;
  const int nout = fe.nout;
  HostStage *hs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    hs = &g_stage[dev];
  }
  if (!hs->st[0]) {
    for (int i = 0; i < 2; i++) {
      if ((e = cudaStreamCreateWithFlags(&hs->st[i], cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e);
    }
    if ((e = cudaEventCreateWithFlags(&hs->ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
  }
  size_t need = kChunkElems * 8;
  if (hs->bytes < need) {
    for (int i = 0; i < 2; i++) {
      if (hs->din[i]) cudaFree(hs->din[i]);
      if (hs->dout[i]) cudaFree(hs->dout[i]);
      hs->din[i] = hs->dout[i] = nullptr;
      if (cudaMalloc(&hs->din[i], need) != cudaSuccess || cudaMalloc(&hs->dout[i], 2 * need) != cudaSuccess)
        return CRM_ERR_NOMEM;
    }
    hs->bytes = need;
  }
  // order after the caller's prior work on `user`
  if ((e = cudaEventRecord(hs->ev, user)) != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < 2; i++)
    if ((e = cudaStreamWaitEvent(hs->st[i], hs->ev, 0)) != cudaSuccess) return cuda_fail(e);
  const char *hin = (const char *)in;
  char *hout = (char *)out;
  uint64_t c = 0;
  for (uint64_t off = 0; off < n; off += kChunkElems, c++) {
    uint64_t m = n - off < kChunkElems ? n - off : kChunkElems;
    int b = (int)(c & 1);
    cudaStream_t s = hs->st[b];
    if ((e = cudaMemcpyAsync(hs->din[b], hin + off * es, m * es, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e);
    int st = enqueue(func, form, hs->din[b], hs->dout[b], m, s, 0);
    if (st) return st;
    for (int r = 0; r < nout; r++) {
      if ((e = cudaMemcpyAsync(hout + (r * n + off) * es, (char *)hs->dout[b] + r * m * es, m * es,
                               cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e);
    }
  }
  for (int i = 0; i < 2; i++)
    if ((e = cudaStreamSynchronize(hs->st[i])) != cudaSuccess) return cuda_fail(e);
  return CRM_OK;
}

}  // namespace crm

using namespace crm;

// Times `reps` back-to-back runs of fn() on stream s (after one untimed run).
template <class F> static int time_runs(cudaStream_t s, int reps, float *ms, F fn) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e);
  }
  int st = fn();
  if (!st && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_fail(e);
  for (int r = 0; r < reps && !st; r++) st = fn();
  if (!st && (e = cudaEventRecord(e1, s)) != cudaSuccess) st = cuda_fail(e);
  if (!st && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(e);
  float t = 0.0f;
  if (!st && (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) st = cuda_fail(e);
  if (!st) *ms = t / (float)reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

extern "C" {

int crm_eval_form(int func_id, int dtype, int form, const void *in, void *out, uint64_t n, void *stream) {
  ensure_init();
  int st = check_args(func_id, dtype, in, out, n);
  if (st) return st;
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  if (resolve_form(g_table[func_id], form) < 0) return CRM_ERR_FORM;
  if (n == 0) return CRM_OK;
  return enqueue(func_id, form, in, out, n, (cudaStream_t)stream, 0);
}

int crm_eval(int func_id, int dtype, const void *in, void *out, uint64_t n, void *stream) {
  ensure_init();
  return crm_eval_form(func_id, dtype, g_default_form, in, out, n, stream);
}

int crm_eval_rm(int func_id, int dtype, int rmode, const void *in, void *out, uint64_t n, void *stream) {
  ensure_init();
  if (func_id < 0 || func_id >= CRM_NUM_FUNCS) return CRM_ERR_FUNC;
  if (rmode < CRM_RN || rmode > CRM_RZ) return CRM_ERR_ARG;
  const bool f64 = func_id >= CRM_EXP2;
  if (dtype == CRM_F16 || dtype == CRM_BF16) {
    if (f64) return CRM_ERR_DTYPE;  // the 16-bit formats take the binary32 functions
  } else {
    int st = check_args(func_id, dtype, in, out, n);
    if (st) return st;
    if (rmode == CRM_RN) return crm_eval_form(func_id, dtype, CRM_FORM_AUTO, in, out, n, stream);
  }
  if (n == 0) return CRM_OK;
  if (!in || !out) return CRM_ERR_NULL;
  const size_t es = dtype == CRM_F64 ? 8 : (dtype == CRM_F32 ? 4 : 2);
  if (((uintptr_t)in % es) || ((uintptr_t)out % es) || n > (1ull << 40)) return CRM_ERR_ARG;
  const uintptr_t a0 = (uintptr_t)in, a1 = a0 + n * es;
  const uintptr_t b0 = (uintptr_t)out, b1 = b0 + n * es * (func_id == CRM_SINCOSF ? 2 : 1);
  if (a0 != b0 && a0 < b1 && b0 < a1) return CRM_ERR_OVERLAP;
  const FuncEntry &fe = g_table[func_id];
  if (!fe.dmain) return CRM_ERR_FORM;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w = nullptr;
  int st = get_ws(s, kDefaultCap, &w);
  if (st) return st;
  KArgs a;
  memset(&a, 0, sizeof(a));
  a.in = in;
  a.out = out;
  a.n = n;
  a.hdr = w->hdr;
  a.q = w->q;
  a.cap = w->cap;
  a.qcount = subq_counts(w);
  a.nsubq = CRM_NSUBQ;
  a.force_hard = g_force_slow;
  a.rm = rmode;
  a.fmt = dtype == CRM_F16 ? 1 : (dtype == CRM_BF16 ? 2 : 0);
  // 16-byte vectors between a scalar head and tail (k_main's geometry): 4 binary32 or 2
  // binary64 elements, or 8 halves for the 16-bit formats (in and out congruent modulo 16
  // bytes, and for sincosf the second output too)
  uint64_t W = dtype == CRM_F64 ? 2 : 4;
  if (a.fmt == 0) {
    fill_geometry(fe, in, out, n, a, 16);
  } else {
    W = 8;
    const uintptr_t ia = (uintptr_t)in, oa = (uintptr_t)out;
    const bool vec = ((ia - oa) % 16) == 0 && (fe.nout == 1 || (n * 2) % 16 == 0);
    a.head = vec ? ((16 - ia % 16) % 16) / 2 : 0;
    if (a.head > n) a.head = n;
    a.nvec = vec ? (n - a.head) / 8 : 0;
    if (a.nvec >= (1ull << 31)) a.nvec = (1ull << 31) - 1;  // 32-bit vector indices; the rest is the tail
  }
  const int sms = dev_sms();
  const uint64_t nscal = a.head + (n - a.head - W * a.nvec);
  const uint64_t want_v = (a.nvec + KBLOCK - 1) / KBLOCK;
  const uint64_t want_s = (nscal + (uint64_t)KBLOCK * DIR_UNROLL - 1) / ((uint64_t)KBLOCK * DIR_UNROLL);
  uint64_t want = want_v > want_s ? want_v : want_s;
  if (want == 0) want = 1;
  const uint64_t cap_blocks = (uint64_t)sms * blocks_per_sm(fe.dmain_sym, KBLOCK);
  const int grid = (int)(want < cap_blocks ? want : cap_blocks);
  cudaError_t e = cudaMemsetAsync(a.qcount, 0, CRM_NSUBQ * CRM_SUBQ_STRIDE * 8, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = fe.dmain(a, grid, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = fe.dslow(a, sms * 2, s)) != cudaSuccess) return cuda_fail(e);
  return CRM_OK;
}

int crm_set_form(int form) {
  ensure_init();
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  g_default_form = form;
  return CRM_OK;
}

int crm_set_force_slow(int on) {
  ensure_init();
  g_force_slow = on == 2 ? 2 : (on ? 1 : 0);
  return CRM_OK;
}

// Queue entries reserved for calls of up to max_elems elements: one entry per 64
// elements (room for a hard-case rate of 1/64 before any lane is finished inline), at
// least the default 2^21 entries and at most 2^26 (1 GiB).
static uint64_t queue_cap_for(uint64_t max_elems) {
  uint64_t cap = (max_elems + 63) / 64;
  cap = (cap + CRM_NSUBQ - 1) / CRM_NSUBQ * CRM_NSUBQ;
  if (cap < kDefaultCap) cap = kDefaultCap;
  if (cap > (1ull << 26)) cap = 1ull << 26;
  return cap;
}

int crm_reserve(uint64_t max_elems, int max_arrays, void *stream) {
  ensure_init();
  if (max_arrays < 0) return CRM_ERR_ARG;
  Workspace *w;
  int st = get_ws((cudaStream_t)stream, queue_cap_for(max_elems), &w);
  if (st) return st;
  return max_arrays > 0 ? batch_buffers((cudaStream_t)stream, w, max_arrays) : CRM_OK;
}

int crm_hard_case_count(void *stream, uint64_t *host_out) {
  if (!host_out) return CRM_ERR_NULL;
  crm_stats_t st;
  const int r = crm_stats(stream, &st);
  if (r == CRM_OK) *host_out = st.last_count;
  return r;
}

int crm_stats(void *stream, crm_stats_t *out) {
  ensure_init();
  if (!out) return CRM_ERR_NULL;
  Workspace *w;
  int st = get_ws((cudaStream_t)stream, kDefaultCap, &w);
  if (st) return st;
  crm_ws_header h;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemcpy(&h, w->hdr, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  out->hard_total = h.hard_total;
  out->unresolved_total = h.unresolved_total;
  out->inline_total = h.inline_total;
  out->last_count = h.count;
  out->timeouts = h.timeouts;
  out->fp64_total = h.fp64_total;
  return CRM_OK;
}

int crm_stats_reset(void *stream) {
  ensure_init();
  Workspace *w;
  int st = get_ws((cudaStream_t)stream, kDefaultCap, &w);
  if (st) return st;
  cudaError_t e = cudaMemsetAsync(w->hdr, 0, sizeof(crm_ws_header), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? CRM_OK : cuda_fail(e);
}

// Page-locked host memory that the device addresses directly (cudaHostAlloc on a system
// with unified addressing reports it as host memory with a device pointer): the device
// address is returned in dp.  Anything else (pageable memory, device memory) is false.
static bool device_mapped_host(const void *p, void **dp) {
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    (void)cudaGetLastError();  // a failed query leaves a (non-sticky) last error: clear it
    return false;
  }
  if (pa.type != cudaMemoryTypeHost || pa.devicePointer == nullptr) return false;
  *dp = pa.devicePointer;
  return true;
}

int crm_eval_host(int func_id, int dtype, int form, const void *in, void *out, uint64_t n, void *stream) {
  ensure_init();
  if (func_id < 0 || func_id >= CRM_NUM_FUNCS) return CRM_ERR_FUNC;
  int want = func_id >= CRM_EXP2 ? CRM_F64 : CRM_F32;
  if (dtype != want) return CRM_ERR_DTYPE;
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  if (resolve_form(g_table[func_id], form) < 0) return CRM_ERR_FORM;
  if (n == 0) return CRM_OK;
  if (!in || !out) return CRM_ERR_NULL;
  void *din = nullptr, *dout = nullptr;
  if (device_mapped_host(in, &din) && device_mapped_host(out, &dout)) {
    // both buffers mapped: the kernels stream them in place over the host link (on
    // GB300, NVLink-C2C), without staging copies
    cudaStream_t s = (cudaStream_t)stream;
    int st = check_args(func_id, dtype, din, dout, n);
    if (st) return st;
    // the packing shapes store the packed elements' results one by one, in small writes
    // that the host link serves slowly: take the same shape without packing
    const int fm = resolve_form(g_table[func_id], form);
    int v = variant_of(func_id, fm);
    if (VARIANTS[v].easy) v = VARIANTS[v].vec_bytes == 32 ? 9 : 7;
    st = enqueue(func_id, form, din, dout, n, s, 0, v);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? CRM_OK : cuda_fail(e);
  }
  return host_pipeline(func_id, form, in, out, n, (cudaStream_t)stream);
}

int crm_eval_batch(const crm_desc_t *descs, int count, int form, void *stream) {
  ensure_init();
  if (count < 0) return CRM_ERR_ARG;
  if (count == 0) return CRM_OK;
  if (!descs) return CRM_ERR_NULL;
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  if (count > (1 << 23)) return CRM_ERR_ARG;
  bool has64 = false;
  for (int i = 0; i < count; i++) {
    const crm_desc_t &d = descs[i];
    int st = check_args(d.func_id, d.dtype, d.in, d.out, d.n);
    if (st) return st;
    if (resolve_form(g_table[d.func_id], form) < 0) return CRM_ERR_FORM;
    if (d.func_id > CRM_LOG) return CRM_ERR_FUNC;  // the batching form takes the paper's 21
    if (d.func_id >= CRM_EXP2) has64 = true;
  }
  int fm = form == CRM_FORM_PLAIN_FP64 ? 1 : 2;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w = nullptr;
  int st = get_ws(s, kDefaultCap, &w);
  if (st) return st;
  st = batch_buffers(s, w, count);
  if (st) return st;
  bool cap = capturing(s);
  cudaError_t e;
  if (!cap) {  // the staging copy of the previous batch must have been consumed
    e = cudaEventSynchronize(w->bcopied);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const int shift = g_batch_tile_shift;
  const bool grouped = g_batch_mode == CRM_BATCH_GROUPED || has64;  // binary64: grouped only
  // Staging: the mixed mode keeps the caller's order; the grouped mode orders the arrays by
  // function (stable), with tile indices counted from the start of each function's group.
  int gstart[CRM_NUM_FUNCS], gcount[CRM_NUM_FUNCS];
  uint64_t gtiles[CRM_NUM_FUNCS];
  const int NF = CRM_NUM_FUNCS;
  for (int f = 0; f < NF; f++) gcount[f] = 0, gtiles[f] = 0;
  for (int i = 0; i < count; i++)
    if (descs[i].n) gcount[grouped ? descs[i].func_id : 0]++;
  int used = 0;
  for (int f = 0; f < NF; f++) {
    gstart[f] = used;
    used += gcount[f];
  }
  if (used == 0) return CRM_OK;
  int fill[CRM_NUM_FUNCS];
  for (int f = 0; f < NF; f++) fill[f] = gstart[f];
  for (int i = 0; i < count; i++) {
    const crm_desc_t &d = descs[i];
    if (d.n == 0) continue;
    const int g = grouped ? d.func_id : 0;
    BatchDesc &b = w->bstage[fill[g]++];
    b.in = d.in;
    b.out = d.out;
    b.n = d.n;
    b.tile0 = gtiles[g];
    b.func = d.func_id;
    uintptr_t ia = (uintptr_t)d.in, oa = (uintptr_t)d.out;
    bool vec = (ia % 16) == 0 && (oa % 16) == 0 && (d.func_id != CRM_SINCOSF || (d.n * 4) % 16 == 0);
    b.flags = vec ? 1 : 0;
    gtiles[g] += (d.n + (1ull << shift) - 1) >> shift;  // (binary64 vectors: 2 elements)
  }
  e = cudaMemcpyAsync(w->bdesc, w->bstage, used * sizeof(BatchDesc), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!cap) {
    e = cudaEventRecord(w->bcopied, s);
    if (e != cudaSuccess) return cuda_fail(e);
  } else {
    w->bcaptured = true;  // this graph now owns bstage and bdesc
  }
  int sms = dev_sms();
  BatchArgs a;
  a.descs = w->bdesc;
  a.count = used;
  a.tile_shift = shift;
  a.hdr = w->hdr;
  a.q = w->q;
  a.cap = w->cap;
  a.qcount = subq_counts(w);
  a.nsubq = CRM_NSUBQ;
  a.force_hard = g_force_slow;
  a.aid_base = 0;
  e = cudaMemsetAsync(a.qcount, 0, CRM_NSUBQ * CRM_SUBQ_STRIDE * 8, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!grouped) {
    const uint64_t tiles = gtiles[0];
    uint64_t grid = (uint64_t)sms * blocks_per_sm(batch_kernel_symbol(fm), KBLOCK);
    if (grid > tiles) grid = tiles;
    a.total_tiles = tiles;
    a.tiles_per_block = (tiles + grid - 1) / grid;
    e = launch_batch(a, fm, (int)grid, sms * 2, s);
    return e == cudaSuccess ? CRM_OK : cuda_fail(e);
  }
  for (int f = 0; f < NF; f++) {
    if (!gcount[f]) continue;
    BatchArgs g = a;
    g.descs = w->bdesc + gstart[f];
    g.count = gcount[f];
    g.aid_base = (uint32_t)gstart[f];
    g.total_tiles = gtiles[f];
    // the function's arrays are packed when its chosen launch shape packs (crm_autotune
    // found packing faster on its data)
    const bool easy = fm == 2 && VARIANTS[variant_of(f, fm)].easy != 0;
    uint64_t grid = (uint64_t)sms * blocks_per_sm(batch_group_symbol(f, fm, easy), KBLOCK);
    if (grid > gtiles[f]) grid = gtiles[f];
    g.tiles_per_block = (gtiles[f] + grid - 1) / grid;
    e = launch_batch_group(f, g, fm, (int)grid, s, easy);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = launch_batch_slow(a, sms * 2, s);
  return e == cudaSuccess ? CRM_OK : cuda_fail(e);
}

int crm_set_batch_mode(int mode) {
  ensure_init();
  if (mode != CRM_BATCH_MIXED && mode != CRM_BATCH_GROUPED) return CRM_ERR_ARG;
  g_batch_mode = mode;
  return CRM_OK;
}

int crm_set_batch_tile(int log2_elems) {
  ensure_init();
  if (log2_elems < 8 || log2_elems > 24) return CRM_ERR_ARG;
  g_batch_tile_shift = log2_elems;
  return CRM_OK;
}

int crm_variant_info(int variant, int *unroll, int *block, int *prefetch, int *pipelined, int *min_blocks,
                     int *vec_bytes, int *reg_table, int *easy) {
  if (variant < 0 || variant >= NVARIANT) return CRM_ERR_ARG;
  if (reg_table) *reg_table = VARIANTS[variant].reg_table;
  if (easy) *easy = VARIANTS[variant].easy;
  if (unroll) *unroll = VARIANTS[variant].unroll;
  if (block) *block = VARIANTS[variant].block;
  if (prefetch) *prefetch = VARIANTS[variant].prefetch;
  if (pipelined) *pipelined = VARIANTS[variant].pipelined;
  if (min_blocks) *min_blocks = VARIANTS[variant].min_blocks;
  if (vec_bytes) *vec_bytes = VARIANTS[variant].vec_bytes;
  return CRM_OK;
}

int crm_set_variant(int func_id, int form, int variant) {
  ensure_init();
  if (func_id < 0 || func_id >= CRM_NUM_FUNCS) return CRM_ERR_FUNC;
  int fm = resolve_form(g_table[func_id], form);
  if (fm < 0) return CRM_ERR_FORM;
  if (variant < 0 || variant >= NVARIANT || !g_table[func_id].main[fm][variant]) return CRM_ERR_ARG;
  set_variant_of(func_id, fm, variant);
  return CRM_OK;
}

int crm_get_variant(int func_id, int form, int *variant) {
  ensure_init();
  if (func_id < 0 || func_id >= CRM_NUM_FUNCS) return CRM_ERR_FUNC;
  if (!variant) return CRM_ERR_NULL;
  int fm = resolve_form(g_table[func_id], form);
  if (fm < 0) return CRM_ERR_FORM;
  *variant = variant_of(func_id, fm);
  return CRM_OK;
}

int crm_autotune(int func_id, int dtype, int form, const void *in, void *out, uint64_t n, int reps,
                 void *stream, int *best, float *ms) {
  ensure_init();
  int st = check_args(func_id, dtype, in, out, n);
  if (st) return st;
  if (form < CRM_FORM_AUTO || form > CRM_FORM_DF32) return CRM_ERR_FORM;
  const FuncEntry &fe = g_table[func_id];
  int fm = resolve_form(fe, form);
  if (fm < 0) return CRM_ERR_FORM;
  cudaStream_t s = (cudaStream_t)stream;
  if (capturing(s)) return CRM_ERR_CAPTURE;
  if (reps < 1) reps = 1;
  int bv = variant_of(func_id, fm);
  float bms = 0.0f;
  bool have = false;
  for (int v = 0; v < NVARIANT; v++) {
    if (ms) ms[v] = -1.0f;
    if (!fe.main[fm][v] || n == 0) continue;
    float t = 0.0f;
    st = time_runs(s, reps, &t, [&]() { return enqueue(func_id, fm, in, out, n, s, 0, v); });
    if (st) return st;
    if (ms) ms[v] = t;
    if (!have || t < bms) {
      bms = t;
      bv = v;
      have = true;
    }
  }
  set_variant_of(func_id, fm, bv);
  if (best) *best = bv;
  return CRM_OK;
}

int crm_autotune_batch(const crm_desc_t *descs, int count, int form, int reps, void *stream, int *best_mode,
                       int *best_shift, float *ms) {
  ensure_init();
  if (capturing((cudaStream_t)stream)) return CRM_ERR_CAPTURE;
  if (reps < 1) reps = 1;
  const int keep_shift = g_batch_tile_shift, keep_mode = g_batch_mode;
  int bs = keep_shift, bm = keep_mode;
  float bms = 0.0f;
  bool have = false;
  const int ntiles = CRM_BATCH_TILE_MAX - CRM_BATCH_TILE_MIN + 1;
  for (int mode = CRM_BATCH_MIXED; mode <= CRM_BATCH_GROUPED; mode++) {
    for (int sh = CRM_BATCH_TILE_MIN; sh <= CRM_BATCH_TILE_MAX; sh++) {
      g_batch_tile_shift = sh;
      g_batch_mode = mode;
      float t = 0.0f;
      int st = time_runs((cudaStream_t)stream, reps, &t, [&]() { return crm_eval_batch(descs, count, form, stream); });
      if (st) {
        g_batch_tile_shift = keep_shift;
        g_batch_mode = keep_mode;
        return st;
      }
      if (ms) ms[mode * ntiles + sh - CRM_BATCH_TILE_MIN] = t;
      if (!have || t < bms) {
        bms = t;
        bs = sh;
        bm = mode;
        have = true;
      }
    }
  }
  g_batch_tile_shift = bs;
  g_batch_mode = bm;
  if (best_shift) *best_shift = bs;
  if (best_mode) *best_mode = bm;
  return CRM_OK;
}

const char *crm_status_str(int status) {
  switch (status) {
    case CRM_OK: return "ok";
    case CRM_ERR_FUNC: return "unknown function id";
    case CRM_ERR_DTYPE: return "dtype does not match the function";
    case CRM_ERR_NULL: return "null pointer";
    case CRM_ERR_OVERLAP: return "input and output overlap partially";
    case CRM_ERR_CUDA: return "CUDA runtime error";
    case CRM_ERR_NOMEM: return "out of device memory";
    case CRM_ERR_FORM: return "form not available for this function";
    case CRM_ERR_CAPTURE: return "workspace must grow during stream capture";
    case CRM_ERR_ARG: return "invalid argument";
    case CRM_ERR_NODEV: return "no CUDA device";
    case CRM_ERR_SIZE: return "n exceeds CRM_NOALLOC_MAX_ELEMS for crm_eval_noalloc";
  }
  return "unknown status";
}

int crm_last_cuda_error(void) { return g_last_cuda; }

void crm_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &kv : g_ws) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first.first);
    if (kv.second.q) cudaFree(kv.second.q);
    if (kv.second.hdr) cudaFree(kv.second.hdr);
    if (kv.second.bdesc) cudaFree(kv.second.bdesc);
    if (kv.second.bstage) cudaFreeHost(kv.second.bstage);
    if (kv.second.bcopied) cudaEventDestroy(kv.second.bcopied);
    for (auto &r : kv.second.retired) {
      cudaFree(r.first);
      cudaFreeHost(r.second);
    }
    for (auto *q : kv.second.retired_q) cudaFree(q);
    cudaSetDevice(cur);
  }
  g_ws.clear();
  g_dev.clear();
}

const char *crm_version(void) { return "crm 0.1 (sm_103a)"; }

}  // extern "C"
