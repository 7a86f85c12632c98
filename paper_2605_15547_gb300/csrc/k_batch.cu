// k_batch.cu -- the batching form: one persistent kernel over many arrays of uneven
// length and mixed functions, and the matching slow-path kernel.
//
// The host cuts every array into tiles of 2^tile_shift elements and gives each array
// the index of its first tile (a prefix over the tile counts).  Block b owns the
// contiguous tile range [b * tpb, (b + 1) * tpb): one binary search finds the array of
// its first tile, then it walks forward.  A block-uniform switch on the array's function
// selects the evaluator; the function's small table is (re)loaded into shared memory when
// the function changes between consecutive tiles.  Hard lanes of every array go to one
// queue tagged with the array index (bits 40..63 of the entry's index).
#include "crm_batch.h"
#include "crm_fns.cuh"

namespace crm {

constexpr int BATCH_SMEM = FnTrig<TRIG_TAN>::tab_bytes<2>();  // largest binary32 table (tanf's)
static_assert(FnLog<0>::tab_bytes<2>() <= BATCH_SMEM && FnTrig<TRIG_TAN>::tab_bytes<2>() <= BATCH_SMEM &&
                  FnExp<0>::tab_bytes<2>() <= BATCH_SMEM && FnHyp<0>::tab_bytes<2>() <= BATCH_SMEM &&
                  FnAtrig<0>::tab_bytes<2>() <= BATCH_SMEM,
              "the mixed batch kernel's shared memory holds every binary32 table");

template <class Fn, int FORM, bool EASY = false>
CRM_DEV void batch_tile(const BatchDesc &d, uint32_t aid, uint64_t off, uint64_t m, const unsigned char *sm,
                        const BatchArgs &b, float *cw = nullptr) {
  using T = typename Fn::T;
  KArgs a;
  a.in = d.in;
  a.out = d.out;
  a.n = d.n;
  a.hdr = b.hdr;
  a.q = b.q;
  a.cap = b.cap;
  a.qcount = b.qcount;
  a.nsubq = b.nsubq;
  a.force_hard = b.force_hard;
  a.desc = aid;
  const T *in = (const T *)d.in;
  T *out = (T *)d.out;
  using V = typename VecOf<T>::V;
  constexpr int W = VecOf<T>::W;
  if ((d.flags & 1) && (off % W) == 0) {
    // vectors: 16-byte aligned array, tile offset a multiple of the vector width
    const uint32_t nv = (uint32_t)(m / W);  // a tile is at most 2^16 elements: 32-bit indices
    const V *in4 = (const V *)(in + off);
    V *out4 = (V *)(out + off);
    V *out4b = (V *)(out + d.n + off);
    // two vectors per thread per iteration, and the next iteration's two loaded before
    // this one is evaluated (register prefetch)
    V nx[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const uint32_t v = (uint32_t)(u * KBLOCK) + threadIdx.x;
      nx[u] = v < nv ? ld_stream(in4 + v) : V();
    }
    for (uint32_t base = 0; base < nv; base += 2 * KBLOCK) {
      V xv[2] = {nx[0], nx[1]};
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t v = base + (uint32_t)(2 * KBLOCK + u * KBLOCK) + threadIdx.x;
        nx[u] = v < nv ? ld_stream(in4 + v) : V();
      }
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const uint32_t v = base + (uint32_t)(u * KBLOCK) + threadIdx.x;
        bool act = v < nv;
        if constexpr (EASY && EasyOf<Fn>::value && FORM == 2) {  // whole warps; element off + v W + j
          a.head = off;
          if (!a.force_hard && easy_vector<Fn, FORM>(xv[u], v - (threadIdx.x & 31), act, out4, out4b, 0, sm, a, cw))
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
            ii[j] = off + (uint64_t)v * W + j;
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
    off += (uint64_t)nv * W;
    m -= nv * W;
  }
  // scalar elements (unaligned arrays and the last partial vector)
  for (uint64_t base = 0; base < m; base += KBLOCK) {
    uint64_t k = base + threadIdx.x;
    bool act = k < m;
    uint64_t i = off + k;
    T x = act ? in[i] : T(0);
    T y[2];
    bool h;
    Fn::template eval<FORM>(x, sm, y, h);
    h = (h || a.force_hard) && act;
    if (act) {
      out[i] = y[0];
      if (Fn::NOUT == 2) out[d.n + i] = y[1];
    }
    if (__any_sync(0xFFFFFFFFu, h)) {
      uint64_t xb = xbits_of(x);
      if (push_hard<1>(h ? 1u : 0u, &i, &xb, a)) slow_store<Fn>(x, i, a);
    }
  }
}

// Calls F.template operator()<Fn>() for the function id (block-uniform).
#define CRM_FOR_FUNC(func, F)                                 \
  switch (func) {                                             \
    case 0: F.template run<FnExp<0>>(); break;                \
    case 1: F.template run<FnExp<1>>(); break;                \
    case 2: F.template run<FnExp<2>>(); break;                \
    case 3: F.template run<FnHyp<HYP_EXPM1>>(); break;        \
    case 4: F.template run<FnLog<0>>(); break;                \
    case 5: F.template run<FnLog<1>>(); break;                \
    case 6: F.template run<FnLog<2>>(); break;                \
    case 7: F.template run<FnLog<3>>(); break;                \
    case 8: F.template run<FnTrig<TRIG_SIN>>(); break;        \
    case 9: F.template run<FnTrig<TRIG_COS>>(); break;        \
    case 10: F.template run<FnTrig<TRIG_SINCOS>>(); break;    \
    case 11: F.template run<FnTrig<TRIG_TAN>>(); break;       \
    case 12: F.template run<FnAtrig<AT_ASIN>>(); break;       \
    case 13: F.template run<FnAtrig<AT_ACOS>>(); break;       \
    case 14: F.template run<FnAtrig<AT_ATAN>>(); break;       \
    case 15: F.template run<FnHyp<HYP_SINH>>(); break;        \
    case 16: F.template run<FnHyp<HYP_COSH>>(); break;        \
    case 17: F.template run<FnHyp<HYP_TANH>>(); break;        \
    case 18: F.template run<FnRsqrt>(); break;                \
    default: break;                                           \
  }

// The same over all 21 functions (grouped mode and the slow pass; binary64 included).
#define CRM_FOR_FUNC_ALL(func, F)                              \
  switch (func) {                                             \
    case 19: F.template run<FnExp2D>(); break;                \
    case 20: F.template run<FnLogD>(); break;                 \
    default: CRM_FOR_FUNC(func, F);                           \
  }

template <int FORM> struct LoadOp {
  unsigned char *sm;
  template <class Fn> CRM_DEV void run() { Fn::template load<FORM>(sm); }
};
template <int FORM> struct TileOp {
  const BatchDesc *d;
  uint32_t aid;
  uint64_t off, m;
  const unsigned char *sm;
  const BatchArgs *b;
  template <class Fn> CRM_DEV void run() { batch_tile<Fn, FORM>(*d, aid, off, m, sm, *b); }
};
struct SlowOp {
  uint64_t xbits;
  bool force;
  const BatchDesc *d;
  uint64_t idx;
  unsigned long long *unres, *fp64;
  template <class Fn> CRM_DEV void run() {
    using T = typename Fn::T;
    T y[2];
    int u;
    Fn::slow(x_from_bits<T>(xbits), y, u, force);
    T *out = (T *)d->out;
    out[idx] = y[0];
    if (Fn::NOUT == 2) out[d->n + idx] = y[1];
    if (u & 1) atomicAdd(unres, 1ull);
    if (u & 2) atomicAdd(fp64, 1ull);
  }
};

CRM_DEV uint64_t tiles_of(const BatchDesc &d, int shift) { return (d.n + (1ull << shift) - 1) >> shift; }

template <int FORM>
__global__ void __launch_bounds__(KBLOCK) k_batch(BatchArgs b) {
  __shared__ __align__(16) unsigned char sm[BATCH_SMEM];
  const uint64_t t0 = (uint64_t)blockIdx.x * b.tiles_per_block;
  uint64_t t1 = t0 + b.tiles_per_block;
  if (t1 > b.total_tiles) t1 = b.total_tiles;
  if (t0 >= t1) return;
  // the array holding tile t0: last array with tile0 <= t0
  int lo = 0, hi = b.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.descs[mid].tile0 <= t0) lo = mid; else hi = mid - 1;
  }
  int aidx = lo;
  int cur = -1;
  for (uint64_t t = t0; t < t1; t++) {
    while (t >= b.descs[aidx].tile0 + tiles_of(b.descs[aidx], b.tile_shift)) aidx++;
    const BatchDesc d = b.descs[aidx];
    if (d.func != cur) {
      __syncthreads();
      LoadOp<FORM> L{sm};
      CRM_FOR_FUNC(d.func, L);
      __syncthreads();
      cur = d.func;
    }
    uint64_t off = (t - d.tile0) << b.tile_shift;
    uint64_t m = d.n - off;
    if (m > (1ull << b.tile_shift)) m = 1ull << b.tile_shift;
    TileOp<FORM> op{&d, b.aid_base + (uint32_t)aidx, off, m, sm, &b};
    CRM_FOR_FUNC(d.func, op);
  }
}

// Grouped mode: every array of b has function Fn; the table is loaded once.
template <class Fn, int FORM, bool EASY = false>
__global__ void __launch_bounds__(KBLOCK) k_batch_group(BatchArgs b) {
  __shared__ __align__(16) unsigned char sm[(Fn::template tab_bytes<FORM>() > 0) ? Fn::template tab_bytes<FORM>() : 16];
  constexpr int EW = EASY && FORM == 2 ? easy_words<Fn, VecOf<typename Fn::T>::W>() : 0;
  __shared__ __align__(16) float ebuf[EW > 0 ? (KBLOCK / 32) * EW : 1];
  float *cw = ebuf + (EW > 0 ? (threadIdx.x >> 5) * EW : 0);
  Fn::template load<FORM>(sm);
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * b.tiles_per_block;
  uint64_t t1 = t0 + b.tiles_per_block;
  if (t1 > b.total_tiles) t1 = b.total_tiles;
  if (t0 >= t1) return;
  int lo = 0, hi = b.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.descs[mid].tile0 <= t0) lo = mid; else hi = mid - 1;
  }
  int aidx = lo;
  for (uint64_t t = t0; t < t1; t++) {
    while (t >= b.descs[aidx].tile0 + tiles_of(b.descs[aidx], b.tile_shift)) aidx++;
    const BatchDesc d = b.descs[aidx];
    uint64_t off = (t - d.tile0) << b.tile_shift;
    uint64_t m = d.n - off;
    if (m > (1ull << b.tile_shift)) m = 1ull << b.tile_shift;
    batch_tile<Fn, FORM, EASY>(d, b.aid_base + (uint32_t)aidx, off, m, sm, b, cw);
  }
}

__global__ void __launch_bounds__(KBLOCK) k_batch_slow(BatchArgs b) {
  for_each_queued(b.q, b.qcount, b.nsubq, b.cap, b.hdr, [&](const crm_queue_entry &e) {
    uint32_t aid = (uint32_t)(e.idx >> 40);
    uint64_t idx = e.idx & ((1ull << 40) - 1);
    const BatchDesc *d = &b.descs[aid];
    SlowOp op{e.x, b.force_hard == 1, d, idx, &b.hdr->unresolved_total, &b.hdr->fp64_total};
    CRM_FOR_FUNC_ALL(d->func, op);
  });
}

cudaError_t launch_batch(const BatchArgs &b, int form, int grid, int slow_grid, cudaStream_t s) {
  if (form == 1)
    k_batch<1><<<grid, KBLOCK, 0, s>>>(b);
  else
    k_batch<2><<<grid, KBLOCK, 0, s>>>(b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_batch_slow(b, slow_grid, s);
}

cudaError_t launch_batch_slow(const BatchArgs &b, int slow_grid, cudaStream_t s) {
  k_batch_slow<<<slow_grid, KBLOCK, 0, s>>>(b);
  return cudaGetLastError();
}

// Per-function launchers and symbols of the grouped kernel, indexed by function id.
struct GroupLaunch {
  int form;
  const BatchArgs *b;
  int grid;
  cudaStream_t s;
  bool easy;
  template <class Fn> void run() {
    if (form == 1)
      k_batch_group<Fn, 1><<<grid, KBLOCK, 0, s>>>(*b);
    else if (EasyOf<Fn>::value && easy)
      k_batch_group<Fn, 2, true><<<grid, KBLOCK, 0, s>>>(*b);
    else
      k_batch_group<Fn, 2><<<grid, KBLOCK, 0, s>>>(*b);
  }
};
struct GroupSymbol {
  int form;
  const void *sym;
  bool easy;
  template <class Fn> void run() {
    sym = form == 1 ? (const void *)k_batch_group<Fn, 1>
                    : (EasyOf<Fn>::value && easy ? (const void *)k_batch_group<Fn, 2, true>
                                                 : (const void *)k_batch_group<Fn, 2>);
  }
};

cudaError_t launch_batch_group(int func, const BatchArgs &b, int form, int grid, cudaStream_t s, bool easy) {
  GroupLaunch L{form, &b, grid, s, easy};
  CRM_FOR_FUNC_ALL(func, L);
  return cudaGetLastError();
}

const void *batch_group_symbol(int func, int form, bool easy) {
  GroupSymbol G{form, nullptr, easy};
  CRM_FOR_FUNC_ALL(func, G);
  return G.sym;
}

const void *batch_kernel_symbol(int form) {
  return form == 1 ? (const void *)k_batch<1> : (const void *)k_batch<2>;
}

}  // namespace crm
