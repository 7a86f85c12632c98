// crm_kernels.cuh -- the array kernels.
//
// k_main: one pass over the array, 128-bit coalesced loads and stores (4 binary32 per
//   vector, UNROLL vectors in flight per thread), the chosen tier's evaluator per element,
//   and hard-case compaction: a warp-uniform __any_sync test; when some lane failed its
//   rounding test, __ballot_sync + __popc reserve queue slots with one atomicAdd per warp
//   and the failing lanes write (index, input bits).  This is the paper's Sec. II.B
//   pattern (only failing lanes go to the slow path) mapped to warps.
// k_slow: stream-ordered after k_main, a fixed grid drains the queue with the exact
//   slow path.  If the queue was full, k_main evaluates those lanes inline instead, so no
//   lane is ever dropped.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "crm_common.cuh"
#include "crm_ws.h"

namespace crm {

constexpr int KBLOCK = 256;

struct KArgs {
  const void *in;
  void *out;
  uint64_t n;        // elements
  uint64_t head;     // leading elements handled by the scalar loop (alignment)
  uint64_t nvec;     // float4 / double2 vectors after the head (k_dir, 16-bit formats: 8-half vectors)
  crm_ws_header *hdr;
  crm_queue_entry *q;
  uint64_t cap;      // queue capacity (entries)
  unsigned long long *qcount;  // sub-queue counters, CRM_SUBQ_STRIDE apart
  int nsubq;         // sub-queues (each of cap / nsubq entries)
  int force_hard;    // test hook: every lane takes the slow path (1: and every tier of it)
  uint32_t desc;     // array id recorded in queue entries (batch form)
  int rm;            // rounding direction of the directed kernels (CRM_RM_*)
  int fmt;           // their element format: 0 the function's own, 1 binary16, 2 bfloat16
};

// 32-byte vectors (one 256-bit access per thread: ld/st.global.v8.f32, .v4.f64)
struct alignas(32) float8v {
  float v[8];
};
struct alignas(32) double4v {
  double v[4];
};

// The vector a thread moves per access: 16 bytes, or 32 bytes when WIDE.
template <class T, bool WIDE = false> struct VecOf;
template <> struct VecOf<float, false> { using V = float4; static constexpr int W = 4; };
template <> struct VecOf<double, false> { using V = double2; static constexpr int W = 2; };
template <> struct VecOf<float, true> { using V = float8v; static constexpr int W = 8; };
template <> struct VecOf<double, true> { using V = double4v; static constexpr int W = 4; };

CRM_DEV float8v ld_stream(const float8v *p) {
  float8v r;
  asm volatile("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
                 "=f"(r.v[6]), "=f"(r.v[7])
               : "l"(p));
  return r;
}
CRM_DEV void st_stream(float8v *p, const float8v &a) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.v[0]), "f"(a.v[1]),
               "f"(a.v[2]), "f"(a.v[3]), "f"(a.v[4]), "f"(a.v[5]), "f"(a.v[6]), "f"(a.v[7])
               : "memory");
}
CRM_DEV double4v ld_stream(const double4v *p) {
  double4v r;
  asm volatile("ld.global.cs.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(r.v[0]), "=d"(r.v[1]), "=d"(r.v[2]), "=d"(r.v[3])
               : "l"(p));
  return r;
}
CRM_DEV void st_stream(double4v *p, const double4v &a) {
  asm volatile("st.global.cs.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a.v[0]), "d"(a.v[1]), "d"(a.v[2]),
               "d"(a.v[3])
               : "memory");
}
CRM_DEV float vget(const float8v &a, int j) { return a.v[j]; }
CRM_DEV double vget(const double4v &a, int j) { return a.v[j]; }
CRM_DEV void vset(float8v &a, int j, float x) { a.v[j] = x; }
CRM_DEV void vset(double4v &a, int j, double x) { a.v[j] = x; }

CRM_DEV float4 ld_stream(const float4 *p) { return __ldcs(p); }
CRM_DEV double2 ld_stream(const double2 *p) { return __ldcs(p); }
CRM_DEV void st_stream(float4 *p, float4 v) { __stcs(p, v); }
CRM_DEV void st_stream(double2 *p, double2 v) { __stcs(p, v); }
CRM_DEV float vget(const float4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
CRM_DEV double vget(const double2 &v, int j) { return j == 0 ? v.x : v.y; }
CRM_DEV void vset(float4 &v, int j, float a) {
  if (j == 0) v.x = a; else if (j == 1) v.y = a; else if (j == 2) v.z = a; else v.w = a;
}
CRM_DEV void vset(double2 &v, int j, double a) {
  if (j == 0) v.x = a; else v.y = a;
}
CRM_DEV uint64_t xbits_of(float x) { return fbits(x); }
CRM_DEV uint64_t xbits_of(double x) { return dbits(x); }
template <class T> CRM_DEV T x_from_bits(uint64_t b);
template <> CRM_DEV float x_from_bits<float>(uint64_t b) { return bitsf((uint32_t)b); }
template <> CRM_DEV double x_from_bits<double>(uint64_t b) { return bitsd(b); }

// Reserve queue slots for up to W lanes per thread with one atomicAdd per warp on the
// warp's sub-queue counter (the whole warp calls this; hm holds the thread's hard bits).
// Lanes beyond the sub-queue's capacity are returned in the result mask and must be
// finished inline.
template <int W>
CRM_DEV unsigned push_hard(unsigned hm, const uint64_t *idx, const uint64_t *xb, const KArgs &a) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned m[W];
  unsigned total = 0;
#pragma unroll
  for (int j = 0; j < W; j++) {
    m[j] = __ballot_sync(0xFFFFFFFFu, (hm >> j) & 1u);
    total += __popc(m[j]);
  }
  const unsigned sq = a.nsubq == 1 ? 0u
                                    : (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % (unsigned)a.nsubq;
  const uint64_t subcap = a.cap / (uint64_t)a.nsubq;
  crm_queue_entry *q = a.q + sq * subcap;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&a.qcount[sq * CRM_SUBQ_STRIDE], (unsigned long long)total);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  unsigned over = 0;
#pragma unroll
  for (int j = 0; j < W; j++) {
    if ((hm >> j) & 1u) {
      unsigned long long pos = base + __popc(m[j] & lt);
      if (pos < subcap) {
        crm_queue_entry e;
        e.idx = ((uint64_t)a.desc << 40) | idx[j];
        e.x = xb[j];
        q[pos] = e;
      } else {
        over |= 1u << j;
      }
    }
    base += __popc(m[j]);
  }
  return over;
}

// Fn interface (one struct per function, see the k_*.cu files):
//   using T = float | double;  static constexpr int NOUT = 1 | 2;
//   template <int FORM> static constexpr int tab_bytes();   (shared memory bytes)
//   template <int FORM> CRM_DEV static void load(unsigned char *sm);  (fill it)
//   template <int FORM> CRM_DEV static void eval(T x, const void *sm, T *y, bool &hard);
//     (or, for a table held in registers: using Ctx = ...; make_ctx<FORM>(sm) once per
//     thread, and eval takes the Ctx instead of sm)
//   CRM_DEV static void slow(T x, T *y, int &status, bool force);  (status: bit 0 no tier
//     decided, bit 1 an FP64 tier ran; force: skip
//     the first tier's early exit, so that every deeper tier runs -- the test hook)

template <class Fn, int FORM>
CRM_DEV void load_tab(unsigned char *sm) {
  Fn::template load<FORM>(sm);
  __syncthreads();
}

// What each thread passes to the evaluator: the shared-memory table, or, for an Fn that
// keeps its table in registers (it declares a Ctx type and make_ctx), the thread's share of
// the table, loaded once before the loop.
template <class Fn, int FORM, class = void> struct CtxOf {
  using type = const void *;
  CRM_DEV static type make(const unsigned char *sm) { return sm; }
};
template <class Fn, int FORM> struct CtxOf<Fn, FORM, std::void_t<typename Fn::Ctx>> {
  using type = typename Fn::Ctx;
  CRM_DEV static type make(const unsigned char *sm) { return Fn::template make_ctx<FORM>(sm); }
};

template <class Fn>
__device__ __noinline__ void slow_store(typename Fn::T x, uint64_t i, const KArgs &a) {
  using T = typename Fn::T;
  T y[2];
  int st;
  Fn::slow(x, y, st, a.force_hard == 1);
  T *out = (T *)a.out;
  out[i] = y[0];
  if (Fn::NOUT == 2) out[a.n + i] = y[1];
  atomicAdd(&a.hdr->inline_total, 1ull);
  if (st & 1) atomicAdd(&a.hdr->unresolved_total, 1ull);
  if (st & 2) atomicAdd(&a.hdr->fp64_total, 1ull);
}

// Evaluates the W elements of one vector: y0 (and y1 for two outputs) and the hard
// flags; returns whether any lane of the vector is hard (the flags stay predicates, the
// queue mask is built from them only on the rare path, hard_mask).
// An Fn with two ways to evaluate its fast tier, one valid only for some arguments
// (path_ok) and cheaper, declares path_ok and eval_path<FORM, PATH> (PATH 1: the cheaper
// way, every lane of the warp having passed path_ok; PATH 2: the general way): eval_vec
// then takes one warp vote per vector and evaluates the whole vector on one path.
template <class Fn, class = void> struct HasPaths : std::false_type {};
template <class Fn> struct HasPaths<Fn, std::void_t<decltype(Fn::path_ok(typename Fn::T()))>> : std::true_type {};

template <class Fn, int FORM, int PATH, class V, class C>
CRM_DEV bool eval_vec_on(const V &xv, const C &sm, V &y0, V &y1, bool *h) {
  using T = typename Fn::T;
  constexpr int W = sizeof(V) / sizeof(T);
  bool any = false;
#pragma unroll
  for (int j = 0; j < W; j++) {
    T y[2];
    if constexpr (PATH == 0)
      Fn::template eval<FORM>(vget(xv, j), sm, y, h[j]);
    else
      Fn::template eval_path<FORM, PATH>(vget(xv, j), sm, y, h[j]);
    any = any || h[j];
    vset(y0, j, y[0]);
    if (Fn::NOUT == 2) vset(y1, j, y[1]);
  }
  return any;
}
// Called by whole warps (the vector loops keep every lane of a warp together).
template <class Fn, int FORM, class V, class C>
CRM_DEV bool eval_vec(const V &xv, const C &sm, V &y0, V &y1, bool *h) {
  if constexpr (HasPaths<Fn>::value && FORM != 1) {
    using T = typename Fn::T;
    constexpr int W = sizeof(V) / sizeof(T);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < W; j++) ok = ok && Fn::path_ok(vget(xv, j));
    if (__all_sync(0xFFFFFFFFu, ok)) return eval_vec_on<Fn, FORM, 1>(xv, sm, y0, y1, h);
    return eval_vec_on<Fn, FORM, 2>(xv, sm, y0, y1, h);
  } else {
    return eval_vec_on<Fn, FORM, 0>(xv, sm, y0, y1, h);
  }
}
// ---- compaction of the elements that need the evaluator
// An Fn may declare HAS_EASY and easy(x, y): true when RN(f(x)) is known without evaluating
// f (tiny arguments: x, 1 or RN(pi/2); the proofs are beside each easy()), with y set to it.
// On inputs with a wide range of magnitudes most elements can be of that kind, yet in a
// warp every lane would still pay the full evaluation.  easy_vector resolves them first,
// packs the others of the whole warp's vector (32 W elements) densely into a per-warp
// shared-memory buffer, evaluates them there, one per lane per round, and each evaluating
// lane stores its result (and queues its hard lanes) itself: ceil(M / 32) rounds for M
// elements instead of W.
template <class Fn, class = void> struct EasyOf : std::false_type {};
template <class Fn> struct EasyOf<Fn, std::void_t<decltype(Fn::HAS_EASY)>> : std::bool_constant<Fn::HAS_EASY> {};

// Buffer words per warp: x and the element's place (lane W + j) for 32 W elements.
template <class Fn, int W> constexpr int easy_words() { return EasyOf<Fn>::value ? 2 * 32 * W : 0; }

template <class Fn, int FORM, class C>
CRM_DEV void eval_one(float x, const C &sm, float *y, bool &h) {
  if constexpr (HasPaths<Fn>::value && FORM != 1) {
    if (__all_sync(0xFFFFFFFFu, Fn::path_ok(x)))
      Fn::template eval_path<FORM, 1>(x, sm, y, h);
    else
      Fn::template eval_path<FORM, 2>(x, sm, y, h);
  } else {
    Fn::template eval<FORM>(x, sm, y, h);
  }
}

// One vector per lane of a whole warp: v0 is the warp's first vector of the segment, this
// lane's is v0 + lane (act: it exists).  Returns false, having stored nothing, when more
// than 32 (W - 1) elements need the evaluator (packing would save no round): the caller
// then evaluates the vector as usual.  Otherwise stores every result, queues the hard lanes
// and returns true.  cw: this warp's buffer (easy_words<Fn, W>() words).
template <class Fn, int FORM, class V, class C>
CRM_DEV bool easy_vector(const V &xv, uint32_t v0, bool act, V *out4, V *out4b, uint64_t seg, const C &sm,
                         const KArgs &a, float *cw) {
  using T = typename Fn::T;
  constexpr int W = sizeof(V) / sizeof(T);
  const int lane = threadIdx.x & 31;
  T y[2];
  // a sample first: with fewer than 8 easy elements among the warp's first slot, the
  // vector is taken to have too few to repay the packing (one vote per vector)
  if (__popc(__ballot_sync(0xFFFFFFFFu, act && Fn::easy(vget(xv, 0), y))) < 8) return false;
  // one pass: each element's easy result, and the others packed into the buffer at their
  // place among the warp's (ballot prefix), whatever their count (at most 32 W)
  const unsigned lt = (1u << lane) - 1u;
  uint32_t *ci = (uint32_t *)(cw + 32 * W);
  V y0, y1;
  int M = 0;
#pragma unroll
  for (int j = 0; j < W; j++) {
    const T x = vget(xv, j);
    const bool need = act && !Fn::easy(x, y);  // no lane past the end
    vset(y0, j, y[0]);
    if (Fn::NOUT == 2) vset(y1, j, y[1]);
    const unsigned nb = __ballot_sync(0xFFFFFFFFu, need);
    if (need) {
      const int k = M + __popc(nb & lt);
      cw[k] = x;
      ci[k] = (uint32_t)(lane * W + j);
    }
    M += __popc(nb);
  }
  if (M > 32 * (W - 1)) {  // packing saves no round: the buffer's contents are dropped
    __syncwarp();
    return false;
  }
  if (act) {  // the easy results; the others are overwritten below, in warp order
    st_stream(out4 + v0 + lane, y0);
    if (Fn::NOUT == 2) st_stream(out4b + v0 + lane, y1);
  }
  if (M == 0) return true;
  __syncwarp();  // also orders the vector stores above before the element stores below
  const uint64_t e0 = a.head + (seg + v0) * W;  // the warp's first element
  T *out = (T *)a.out;
  for (int k0 = 0; k0 < M; k0 += 32) {  // every lane runs every round (warp-level votes inside)
    const int k = k0 + lane;
    const bool on = k < M;
    const T x = on ? cw[k] : T(1);
    uint64_t i = e0 + (on ? ci[k] : 0u);
    bool hh;
    eval_one<Fn, FORM>(x, sm, y, hh);
    if (on) {
      out[i] = y[0];
      if (Fn::NOUT == 2) out[a.n + i] = y[1];
    }
    const bool hq = on && hh;
    if (__any_sync(0xFFFFFFFFu, hq)) {
      uint64_t xb = xbits_of(x);
      if (push_hard<1>(hq ? 1u : 0u, &i, &xb, a)) slow_store<Fn>(x, i, a);
    }
  }
  __syncwarp();  // the buffer is refilled by the next vector
  return true;
}

template <int W> CRM_DEV unsigned hard_mask(const bool *h, bool force) {
  unsigned hm = 0;
#pragma unroll
  for (int j = 0; j < W; j++) hm |= (unsigned)(h[j] || force) << j;
  return hm;
}

// The vector loop addresses vectors with 32-bit indices inside segments of at most
// 2^31 vectors (an array below 2^33 binary32 elements is one segment): one add, compare
// and wide multiply-add per vector instead of their 64-bit pairs.  Queue indices stay
// 64-bit (rare path).
constexpr uint64_t KSEG = 1ull << 31;

// Loads the UNROLL vectors of one iteration (zero past the end).
template <class V, int UNROLL, int BS>
CRM_DEV void load_vecs(V *xv, const V *in4, uint32_t base, uint32_t nv) {
#pragma unroll
  for (int u = 0; u < UNROLL; u++) {
    const uint32_t v = base + (uint32_t)(u * BS) + threadIdx.x;
    xv[u] = v < nv ? ld_stream(in4 + v) : V();
  }
}

// Evaluates and stores the UNROLL vectors of one iteration of a segment (nv vectors from
// vector `seg` of the array; out4, out4b point at the segment), queueing the hard lanes.
template <class Fn, int FORM, int UNROLL, int BS, bool WIDE, bool EASY, class C>
CRM_DEV void eval_vecs(const typename VecOf<typename Fn::T, WIDE>::V *xv, uint32_t base, uint32_t nv,
                       typename VecOf<typename Fn::T, WIDE>::V *out4, typename VecOf<typename Fn::T, WIDE>::V *out4b,
                       uint64_t seg, const C &sm, const KArgs &a, float *cw) {
  using T = typename Fn::T;
  using V = typename VecOf<T, WIDE>::V;
  constexpr int W = VecOf<T, WIDE>::W;
#pragma unroll
  for (int u = 0; u < UNROLL; u++) {
    const uint32_t v = base + (uint32_t)(u * BS) + threadIdx.x;
    bool act = v < nv;
    if constexpr (EASY && EasyOf<Fn>::value && FORM == 2) {  // whole warps (force_hard is per launch)
      if (!a.force_hard && easy_vector<Fn, FORM>(xv[u], v - (threadIdx.x & 31), act, out4, out4b, seg, sm, a, cw))
        continue;
    }
    V y0, y1;
    bool h[W];
    const bool any = (eval_vec<Fn, FORM>(xv[u], sm, y0, y1, h) || a.force_hard) && act;
    if (act) {
      st_stream(out4 + v, y0);
      if (Fn::NOUT == 2) st_stream(out4b + v, y1);
    }
    if (__any_sync(0xFFFFFFFFu, any)) {
      const unsigned hm = act ? hard_mask<W>(h, a.force_hard != 0) : 0u;
      uint64_t ii[W], xb[W];
#pragma unroll
      for (int j = 0; j < W; j++) {
        ii[j] = a.head + (seg + v) * W + j;
        xb[j] = xbits_of(vget(xv[u], j));
      }
      unsigned over = push_hard<W>(hm, ii, xb, a);
      if (over) {
#pragma unroll
        for (int j = 0; j < W; j++)
          if ((over >> j) & 1u) slow_store<Fn>(vget(xv[u], j), ii[j], a);
      }
    }
  }
}

// UNROLL vectors per thread per iteration, BS threads per block; with PF the next
// iteration's vectors are loaded
// before this iteration is evaluated (software prefetch: the loads' latency overlaps the
// thread's own arithmetic).
template <class Fn, int FORM, int UNROLL, int BS, bool PF, bool WIDE, bool EASY = false>
CRM_DEV void main_body(const KArgs &a) {
  using T = typename Fn::T;
  using V = typename VecOf<T, WIDE>::V;
  constexpr int W = VecOf<T, WIDE>::W;
  __shared__ __align__(16) unsigned char smem[(Fn::template tab_bytes<FORM>() > 0) ? Fn::template tab_bytes<FORM>() : 16];
  // the per-warp buffers of eval_vec_easy (binary32 functions with easy arguments)
  constexpr int EW = EASY && FORM == 2 ? easy_words<Fn, W>() : 0;
  __shared__ __align__(16) float ebuf[EW > 0 ? (BS / 32) * EW : 1];
  float *cw = ebuf + (EW > 0 ? (threadIdx.x >> 5) * EW : 0);
  load_tab<Fn, FORM>(smem);
  const typename CtxOf<Fn, FORM>::type sm = CtxOf<Fn, FORM>::make(smem);

  // base < nv <= 2^31 and stride = grid * BS * UNROLL < 2^26 (at most one wave of
  // resident blocks): base + stride stays below 2^32
  const uint32_t stride = gridDim.x * (uint32_t)(BS * UNROLL);
  for (uint64_t seg = 0; seg < a.nvec; seg += KSEG) {
    const uint32_t nv = (uint32_t)(a.nvec - seg < KSEG ? a.nvec - seg : KSEG);  // >= 1
    const V *in4 = (const V *)((const T *)a.in + a.head) + seg;
    V *out4 = (V *)((T *)a.out + a.head) + seg;
    V *out4b = (V *)((T *)a.out + a.n + a.head) + seg;  // second output (sincos)
    uint32_t base = blockIdx.x * (uint32_t)(BS * UNROLL);
    if (PF) {
      V xv[UNROLL];
      load_vecs<V, UNROLL, BS>(xv, in4, base, nv);
      for (; base < nv; base += stride) {
        V nx[UNROLL];
        load_vecs<V, UNROLL, BS>(nx, in4, base + stride, nv);
        eval_vecs<Fn, FORM, UNROLL, BS, WIDE, EASY>(xv, base, nv, out4, out4b, seg, sm, a, cw);
#pragma unroll
        for (int u = 0; u < UNROLL; u++) xv[u] = nx[u];
      }
    } else {
      for (; base < nv; base += stride) {
        V xv[UNROLL];
        load_vecs<V, UNROLL, BS>(xv, in4, base, nv);
        eval_vecs<Fn, FORM, UNROLL, BS, WIDE, EASY>(xv, base, nv, out4, out4b, seg, sm, a, cw);
      }
    }
  }
  // scalar part: the head [0, head) and the tail [head + W nvec, n)
  const uint64_t tail0 = a.head + (uint64_t)W * a.nvec;
  const uint64_t nscal = a.head + (a.n - tail0);
  const T *in = (const T *)a.in;
  T *out = (T *)a.out;
  const uint64_t sstride = (uint64_t)gridDim.x * BS;
  for (uint64_t b = (uint64_t)blockIdx.x * BS; b < nscal; b += sstride) {
    uint64_t k = b + threadIdx.x;
    bool act = k < nscal;
    uint64_t i = k < a.head ? k : tail0 + (k - a.head);
    T x = act ? in[i] : T(0);
    T y[2];
    bool h;
    Fn::template eval<FORM>(x, sm, y, h);
    h = (h || a.force_hard) && act;
    if (act) {
      out[i] = y[0];
      if (Fn::NOUT == 2) out[a.n + i] = y[1];
    }
    if (__any_sync(0xFFFFFFFFu, h)) {
      uint64_t xb = xbits_of(x);
      if (push_hard<1>(h ? 1u : 0u, &i, &xb, a)) slow_store<Fn>(x, i, a);
    }
  }
}

// Binary32 kernels are held to 64 registers (two 512-thread blocks per SM): their fast
// path needs 47-57, and what would raise the count is the rarely called inline slow path
// (queue overflow), which may spill instead.  The binary64 fixed-point kernels keep the
// compiler's choice.
template <class Fn> constexpr int min_blocks_64regs(int bs) {
  return sizeof(typename Fn::T) == 4 ? 65536 / (bs * 64) : 1;
}
template <class Fn, int FORM, int UNROLL, int BS, bool PF, bool WIDE = false, bool EASY = false>
__global__ void __launch_bounds__(BS, min_blocks_64regs<Fn>(BS)) k_main(KArgs a) {
  main_body<Fn, FORM, UNROLL, BS, PF, WIDE, EASY>(a);
}
// The same with a register cap: at least MINB blocks of BS threads resident per SM.
template <class Fn, int FORM, int UNROLL, int BS, bool PF, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_main_capped(KArgs a) {
  main_body<Fn, FORM, UNROLL, BS, PF, false>(a);
}

// ------------------------------------------------------------------ pipelined variant
// The same work with the inputs staged through shared memory by bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), a ring of PSTAGES chunks per block:
// the bytes in flight no longer depend on registers, so each SM keeps enough reads
// outstanding to cover HBM latency.  Thread 0 issues the copies; every wait is bounded
// by the global timer (1 s), after which the block records a timeout, waits (bounded)
// for its copies still in flight and returns.
constexpr int PSTAGES = 4;
constexpr int PVPT = 2;  // 16-byte vectors per thread per chunk
constexpr unsigned long long PWAIT_NS = 1000000000ull;

CRM_DEV unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
CRM_DEV void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
CRM_DEV void mbar_arm_and_copy(uint64_t *bar, void *dst, const void *src, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
CRM_DEV bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
CRM_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the given phase parity; false if the global-timer limit ran out first.
CRM_DEV bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > PWAIT_NS) return false;
  return true;
}

template <class Fn, int FORM>
__global__ void __launch_bounds__(KBLOCK) k_pipe(KArgs a) {
  using T = typename Fn::T;
  using V = typename VecOf<T>::V;
  constexpr int W = VecOf<T>::W;
  constexpr int CH = KBLOCK * PVPT;  // vectors per chunk
  __shared__ __align__(16) unsigned char sm[(Fn::template tab_bytes<FORM>() > 0) ? Fn::template tab_bytes<FORM>() : 16];
  __shared__ __align__(128) V buf[PSTAGES][CH];
  __shared__ uint64_t bars[PSTAGES];
  Fn::template load<FORM>(sm);
  if (threadIdx.x == 0) {
    for (int s = 0; s < PSTAGES; s++) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const V *in4 = (const V *)((const T *)a.in + a.head);
  V *out4 = (V *)((T *)a.out + a.head);
  V *out4b = (V *)((T *)a.out + a.n + a.head);
  const uint64_t nchunks = (a.nvec + CH - 1) / CH;
  const uint64_t mine = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto chunk_of = [&](uint64_t i) { return blockIdx.x + i * gridDim.x; };
  auto issue = [&](uint64_t i) {
    uint64_t c = chunk_of(i);
    uint64_t v0 = c * CH;
    uint64_t nv = a.nvec - v0 < (uint64_t)CH ? a.nvec - v0 : (uint64_t)CH;
    mbar_arm_and_copy(&bars[i % PSTAGES], buf[i % PSTAGES], in4 + v0, (unsigned)(nv * sizeof(V)));
  };
  if (threadIdx.x == 0)
    for (uint64_t i = 0; i < mine && i < (uint64_t)PSTAGES; i++) issue(i);
  bool failed = false;
  for (uint64_t i = 0; i < mine; i++) {
    const int st = (int)(i % PSTAGES);
    bool ok = mbar_wait_bounded(&bars[st], (unsigned)((i / PSTAGES) & 1));
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const uint64_t v0 = chunk_of(i) * CH;
#pragma unroll
    for (int u = 0; u < PVPT; u++) {
      const uint64_t vl = (uint64_t)u * KBLOCK + threadIdx.x;
      const uint64_t v = v0 + vl;
      const bool act = v < a.nvec;
      V xv = act ? buf[st][vl] : V();
      V y0, y1;
      bool h[W];
      const bool any = (eval_vec<Fn, FORM>(xv, sm, y0, y1, h) || a.force_hard) && act;
      if (act) {
        st_stream(out4 + v, y0);
        if (Fn::NOUT == 2) st_stream(out4b + v, y1);
      }
      if (__any_sync(0xFFFFFFFFu, any)) {
        const unsigned hm = act ? hard_mask<W>(h, a.force_hard != 0) : 0u;
        uint64_t ii[W], xb[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
          ii[j] = a.head + v * W + j;
          xb[j] = xbits_of(vget(xv, j));
        }
        unsigned over = push_hard<W>(hm, ii, xb, a);
        if (over) {
#pragma unroll
          for (int j = 0; j < W; j++)
            if ((over >> j) & 1u) slow_store<Fn>(vget(xv, j), ii[j], a);
        }
      }
    }
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0 && i + PSTAGES < mine) issue(i + PSTAGES);
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicAdd(&a.hdr->timeouts, 1ull);
      // bounded wait for copies still in flight into this block's shared memory
      for (int s = 0; s < PSTAGES; s++) {
        uint64_t last = (uint64_t)-1;
        for (uint64_t i = 0; i < mine; i++)
          if ((int)(i % PSTAGES) == s) last = i;
        if (last != (uint64_t)-1) mbar_wait_bounded(&bars[s], (unsigned)((last / PSTAGES) & 1));
      }
    }
    __syncthreads();
    return;
  }
  // scalar head and tail, as in k_main
  const uint64_t tail0 = a.head + (uint64_t)W * a.nvec;
  const uint64_t nscal = a.head + (a.n - tail0);
  const T *in = (const T *)a.in;
  T *out = (T *)a.out;
  for (uint64_t b = (uint64_t)blockIdx.x * KBLOCK; b < nscal; b += (uint64_t)gridDim.x * KBLOCK) {
    uint64_t k = b + threadIdx.x;
    bool act = k < nscal;
    uint64_t i = k < a.head ? k : tail0 + (k - a.head);
    T x = act ? in[i] : T(0);
    T y[2];
    bool h;
    Fn::template eval<FORM>(x, sm, y, h);
    h = (h || a.force_hard) && act;
    if (act) {
      out[i] = y[0];
      if (Fn::NOUT == 2) out[a.n + i] = y[1];
    }
    if (__any_sync(0xFFFFFFFFu, h)) {
      uint64_t xb = xbits_of(x);
      if (push_hard<1>(h ? 1u : 0u, &i, &xb, a)) slow_store<Fn>(x, i, a);
    }
  }
}

// Calls f(entry) for every queued entry: the sub-queues are spread over the grid
// (virtual blocks: sub-queue = vb % nsubq, part = vb / nsubq), and each sub-queue's
// entries below its count are taken by its blocks in turn.  Block 0's first warp then
// adds the call's total to hard_total and records it as the last count.
template <class F>
CRM_DEV void for_each_queued(const crm_queue_entry *q, unsigned long long *qcount, int nsubq, uint64_t cap,
                             crm_ws_header *hdr, F f) {
  const uint64_t subcap = cap / (uint64_t)nsubq;
  const unsigned parts = gridDim.x >= (unsigned)nsubq ? gridDim.x / (unsigned)nsubq : 1u;
  for (unsigned vb = blockIdx.x; vb < (unsigned)nsubq * parts; vb += gridDim.x) {
    const unsigned sq = vb % (unsigned)nsubq, part = vb / (unsigned)nsubq;
    unsigned long long cnt = qcount[sq * CRM_SUBQ_STRIDE];
    if (cnt > subcap) cnt = subcap;
    for (uint64_t i = (uint64_t)part * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)parts * blockDim.x)
      f(q[sq * subcap + i]);
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    // the first warp sums the counters (independent loads, then a shuffle reduction:
    // a serial loop would wait for one L2 round trip per counter)
    unsigned long long total = 0;
    for (int sq = (int)threadIdx.x; sq < nsubq; sq += 32) total += qcount[sq * CRM_SUBQ_STRIDE];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(0xFFFFFFFFu, total, o);
    if (threadIdx.x == 0) {
      atomicAdd(&hdr->hard_total, total);
      hdr->count = total;
    }
  }
}

template <class Fn>
__global__ void __launch_bounds__(KBLOCK) k_slow(KArgs a) {
  using T = typename Fn::T;
  T *out = (T *)a.out;
  for_each_queued(a.q, a.qcount, a.nsubq, a.cap, a.hdr, [&](const crm_queue_entry &e) {
    uint64_t idx = e.idx & ((1ull << 40) - 1);
    T x = x_from_bits<T>(e.x);
    T y[2];
    int st;
    Fn::slow(x, y, st, a.force_hard == 1);
    out[idx] = y[0];
    if (Fn::NOUT == 2) out[a.n + idx] = y[1];
    if (st & 1) atomicAdd(&a.hdr->unresolved_total, 1ull);
    if (st & 2) atomicAdd(&a.hdr->fp64_total, 1ull);
  });
}

}  // namespace crm

namespace crm {

// ------------------------------------------------------------------ directed rounding and 16-bit formats
// k_dir: the same evaluation, run with the sign output (Fn::eval with sg): each element's
// candidate c and sign(f(x) - c) go through the finisher of the requested direction and
// format (crm_common.cuh).  Lanes whose sign the fast tier cannot decide (f(x) too close to
// a binary32 number, or on one) are queued as in k_main, and k_dir_slow finishes them.
// Elements are processed one per thread per step (UNROLL steps in flight), with coalesced
// 4-, 8- or 2-byte accesses; 16-bit inputs are widened to binary32 exactly.
template <class T> CRM_DEV T dir_load(const KArgs &a, uint64_t i) { return ((const T *)a.in)[i]; }
template <> CRM_DEV float dir_load<float>(const KArgs &a, uint64_t i) {
  if (a.fmt == 0) return ((const float *)a.in)[i];
  const uint16_t h = ((const uint16_t *)a.in)[i];
  return a.fmt == 2 ? from16<true>(h) : from16<false>(h);
}
CRM_DEV void dir_store(const KArgs &a, uint64_t i, const float *y, const int *sg, int nout) {
  for (int r = 0; r < nout; r++) {
    const uint64_t o = i + (uint64_t)r * a.n;
    if (a.fmt == 0)
      ((float *)a.out)[o] = finish_f32(y[r], sg[r], a.rm);
    else
      ((uint16_t *)a.out)[o] = a.fmt == 2 ? finish_16<true>(y[r], sg[r], a.rm) : finish_16<false>(y[r], sg[r], a.rm);
  }
}
CRM_DEV void dir_store(const KArgs &a, uint64_t i, const double *y, const int *sg, int) {
  ((double *)a.out)[i] = finish_f64(y[0], sg[0], a.rm);
}

template <class Fn>
__device__ __noinline__ void dir_slow_store(typename Fn::T x, uint64_t i, const KArgs &a) {
  using T = typename Fn::T;
  T y[2];
  int sg[2] = {0, 0}, st;
  Fn::slow(x, y, st, a.force_hard == 1, sg);
  dir_store(a, i, y, sg, Fn::NOUT);
  atomicAdd(&a.hdr->inline_total, 1ull);
  if (st & 1) atomicAdd(&a.hdr->unresolved_total, 1ull);
  if (st & 2) atomicAdd(&a.hdr->fp64_total, 1ull);
}

constexpr int DIR_UNROLL = 4;

// One element in a directed mode: candidate, signs and hard flag.
template <class Fn>
CRM_DEV bool dir_eval(typename Fn::T x, const unsigned char *sm, typename Fn::T *y, int *sg, const KArgs &a) {
  bool h;
  sg[0] = sg[1] = 0;
  Fn::template eval<2>(x, sm, y, h, sg);
  return h || a.force_hard;
}

// Binary32 / binary64 results: 16-byte vectors [head, head + W nvec) of the array (the
// geometry of k_main), one vector per thread per step with the next one loaded ahead;
// every element's (candidate, sign) goes through the finisher, hard lanes are queued
// (their stored value is replaced by k_dir_slow).  The 16-bit formats take 16-byte vectors
// of 8 halves instead (nvec counts those).  The scalar loop takes the head and the tail.
template <class Fn>
__global__ void __launch_bounds__(KBLOCK) k_dir(KArgs a) {
  using T = typename Fn::T;
  using V = typename VecOf<T, false>::V;
  constexpr int W = VecOf<T, false>::W;
  __shared__ __align__(16) unsigned char sm[(Fn::template tab_bytes<2>() > 0) ? Fn::template tab_bytes<2>() : 16];
  load_tab<Fn, 2>(sm);
  const uint32_t stride = gridDim.x * (uint32_t)KBLOCK;
  const uint64_t nvec_own = a.fmt == 0 ? a.nvec : 0;  // vectors of the function's own format
  for (uint64_t seg = 0; seg < nvec_own; seg += KSEG) {
    const uint32_t nv = (uint32_t)(nvec_own - seg < KSEG ? nvec_own - seg : KSEG);
    const V *in4 = (const V *)((const T *)a.in + a.head) + seg;
    V *out4 = (V *)((T *)a.out + a.head) + seg;
    V *out4b = (V *)((T *)a.out + a.n + a.head) + seg;  // second output (sincos)
    uint32_t base = blockIdx.x * (uint32_t)KBLOCK;
    V xv = base + threadIdx.x < nv ? ld_stream(in4 + base + threadIdx.x) : V();
    for (; base < nv; base += stride) {  // whole warps: base is block-uniform
      const uint32_t v = base + threadIdx.x, vn = v + stride;
      const V nx = vn < nv ? ld_stream(in4 + vn) : V();
      const bool act = v < nv;
      V y0, y1;
      bool h[W];
      bool any = false;
#pragma unroll
      for (int j = 0; j < W; j++) {
        T y[2];
        int sg[2];
        h[j] = dir_eval<Fn>(vget(xv, j), sm, y, sg, a) && act;
        any = any || h[j];
        if constexpr (sizeof(T) == 4) {
          vset(y0, j, finish_f32(y[0], sg[0], a.rm));
          if (Fn::NOUT == 2) vset(y1, j, finish_f32(y[1], sg[1], a.rm));
        } else {
          vset(y0, j, finish_f64(y[0], sg[0], a.rm));
        }
      }
      if (act) {
        st_stream(out4 + v, y0);
        if (Fn::NOUT == 2) st_stream(out4b + v, y1);
      }
      if (__any_sync(0xFFFFFFFFu, any)) {
        const unsigned hm = hard_mask<W>(h, false);
        uint64_t ii[W], xb[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
          ii[j] = a.head + (seg + v) * W + j;
          xb[j] = xbits_of(vget(xv, j));
        }
        const unsigned over = push_hard<W>(hm, ii, xb, a);
        if (over) {
#pragma unroll
          for (int j = 0; j < W; j++)
            if ((over >> j) & 1u) dir_slow_store<Fn>(vget(xv, j), ii[j], a);
        }
      }
      xv = nx;
    }
  }
  // 16-bit formats: 16-byte vectors of 8 inputs (widened to binary32 exactly), the results
  // finished into the format and stored 8 at a time
  if constexpr (sizeof(T) == 4) {
    if (a.fmt != 0) {
      const uint32_t nv = (uint32_t)a.nvec;  // below 2^31 (crm_eval_rm caps it; the rest is the tail)
      const uint4 *in8 = (const uint4 *)((const uint16_t *)a.in + a.head);
      uint4 *out8 = (uint4 *)((uint16_t *)a.out + a.head);
      uint4 *out8b = (uint4 *)((uint16_t *)a.out + a.n + a.head);
      for (uint32_t base = blockIdx.x * (uint32_t)KBLOCK; base < nv; base += stride) {  // whole warps
        const uint32_t v = base + threadIdx.x;
        const bool act = v < nv;
        const uint4 raw = act ? __ldcs(in8 + v) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
        uint32_t o0[4] = {0u, 0u, 0u, 0u}, o1[4] = {0u, 0u, 0u, 0u};
        float xs[8];
        bool h[8];
        bool any = false;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const uint16_t hb = (uint16_t)(w[j >> 1] >> (16 * (j & 1)));
          xs[j] = a.fmt == 2 ? from16<true>(hb) : from16<false>(hb);
          float y[2];
          int sg[2];
          h[j] = dir_eval<Fn>(xs[j], sm, y, sg, a) && act;
          any = any || h[j];
          const uint32_t r0 = a.fmt == 2 ? finish_16<true>(y[0], sg[0], a.rm) : finish_16<false>(y[0], sg[0], a.rm);
          o0[j >> 1] |= r0 << (16 * (j & 1));
          if (Fn::NOUT == 2) {
            const uint32_t r1 = a.fmt == 2 ? finish_16<true>(y[1], sg[1], a.rm) : finish_16<false>(y[1], sg[1], a.rm);
            o1[j >> 1] |= r1 << (16 * (j & 1));
          }
        }
        if (act) {
          __stcs(out8 + v, make_uint4(o0[0], o0[1], o0[2], o0[3]));
          if (Fn::NOUT == 2) __stcs(out8b + v, make_uint4(o1[0], o1[1], o1[2], o1[3]));
        }
        if (__any_sync(0xFFFFFFFFu, any)) {
          const unsigned hm = hard_mask<8>(h, false);
          uint64_t ii[8], xb[8];
#pragma unroll
          for (int j = 0; j < 8; j++) {
            ii[j] = a.head + (uint64_t)v * 8 + j;
            xb[j] = fbits(xs[j]);
          }
          const unsigned over = push_hard<8>(hm, ii, xb, a);
          if (over) {
#pragma unroll
            for (int j = 0; j < 8; j++)
              if ((over >> j) & 1u) dir_slow_store<Fn>(xs[j], ii[j], a);
          }
        }
      }
    }
  }
  // scalar part: the head [0, head) and the tail [head + Wv nvec, n)
  const uint64_t Wv = sizeof(T) == 4 && a.fmt != 0 ? 8 : (uint64_t)W;
  const uint64_t tail0 = a.head + Wv * a.nvec;
  const uint64_t nscal = a.head + (a.n - tail0);
  const uint64_t sstride = (uint64_t)gridDim.x * KBLOCK * DIR_UNROLL;
  for (uint64_t b = (uint64_t)blockIdx.x * KBLOCK * DIR_UNROLL; b < nscal; b += sstride) {
    T xs[DIR_UNROLL];
    uint64_t is[DIR_UNROLL];
#pragma unroll
    for (int u = 0; u < DIR_UNROLL; u++) {
      const uint64_t k = b + (uint64_t)u * KBLOCK + threadIdx.x;
      is[u] = k < a.head ? k : tail0 + (k - a.head);
      xs[u] = k < nscal ? dir_load<T>(a, is[u]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < DIR_UNROLL; u++) {
      const bool act = b + (uint64_t)u * KBLOCK + threadIdx.x < nscal;
      T y[2];
      int sg[2];
      const bool h = dir_eval<Fn>(xs[u], sm, y, sg, a) && act;
      if (act && !h) dir_store(a, is[u], y, sg, Fn::NOUT);
      if (__any_sync(0xFFFFFFFFu, h)) {
        uint64_t xb = xbits_of(xs[u]);
        if (push_hard<1>(h ? 1u : 0u, &is[u], &xb, a)) dir_slow_store<Fn>(xs[u], is[u], a);
      }
    }
  }
}

template <class Fn>
__global__ void __launch_bounds__(KBLOCK) k_dir_slow(KArgs a) {
  using T = typename Fn::T;
  for_each_queued(a.q, a.qcount, a.nsubq, a.cap, a.hdr, [&](const crm_queue_entry &e) {
    const uint64_t idx = e.idx & ((1ull << 40) - 1);
    T y[2];
    int sg[2] = {0, 0}, st;
    Fn::slow(x_from_bits<T>(e.x), y, st, a.force_hard == 1, sg);
    dir_store(a, idx, y, sg, Fn::NOUT);
    if (st & 1) atomicAdd(&a.hdr->unresolved_total, 1ull);
    if (st & 2) atomicAdd(&a.hdr->fp64_total, 1ull);
  });
}

}  // namespace crm
