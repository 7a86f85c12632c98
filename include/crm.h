/*
 * crm.h -- correctly rounded array math for GB300 (sm_103a): the C ABI.
 *
 * Operation.  For every element x of an input array, store RN(f(x)): f evaluated exactly
 * and rounded once to the nearest binary32 (or binary64) number, ties to even, with
 * gradual underflow and overflow to infinity.  This is the correct-rounding goal of
 * Sec. I and Sec. II of "Correctly Rounded Functions For Vector Applications: A
 * Performance Study"; the GPU runs of Sec. III.C use round-to-nearest-even only, and so
 * does this library.  The single-precision function set is the one of Sec. II.A; the
 * double-precision pair (exp2, log) is the one of Sec. II.B; exp, log2, log10 and exp10 in
 * binary64 extend it (the paper's outlook: more double-precision functions).
 *
 * Evaluation forms (crm_form_t):
 *   CRM_FORM_PLAIN_FP64 -- FP64 internal arithmetic, as the paper's single-precision
 *                          algorithms do (Sec. II.A), plus a rounding test;
 *   CRM_FORM_DF32       -- the FP64-free form: no FP64 on the main path.  Binary32
 *                          functions: FP32 double-float fast path with a rounding test
 *                          and an FP64 / double-double fallback (the FP32 fast path with
 *                          FP64 fallback suggested in Sec. II.A and Sec. IV).  Binary64
 *                          exp2 and log: 128-bit fixed-point integer arithmetic with a
 *                          rounding test, the double-double and exact integer tiers of
 *                          Sec. II.B behind it.  (The plain form of the binary64 pair is
 *                          the double-double main path of Sec. II.B.)
 *   CRM_FORM_AUTO       -- the fastest form available for the function (DF32 where it
 *                          exists).
 * Every form returns the same, correctly rounded, bits: the form changes speed only.
 * Lanes whose fast-path rounding test fails are compacted into a device queue and
 * finished by a slow-path kernel (Sec. II.B: only the failing lanes take the slow path).
 *
 * Special values (the paper does not fix them; this library's convention):
 *   NaN input            -> the input, quieted (sign and payload kept);
 *   invalid operation    -> +qNaN (0x7FC00000 / 0x7FF8000000000000);
 *   odd functions keep the sign of zero; log-family(+-0) = -inf; log1p(-1) = -inf;
 *   rsqrt(+-0) = +-inf; expm1(-inf) = -1; tanh(+-inf) = +-1; atan(+-inf) = +-RN(pi/2).
 *
 * Memory and streams.  Pointers named "device" must be device memory (or memory the
 * device can access) allocated by the caller; the caller owns them.  Calls are
 * asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 * stream).  The library owns a per-(device, stream) workspace (hard-case queue and
 * counters) allocated on first use or by crm_reserve() and freed by crm_shutdown().
 * Calls on different streams may overlap; calls on one stream are ordered.
 * in == out (in place) is allowed; any other overlap returns CRM_ERR_OVERLAP.
 * Any alignment is accepted (unaligned heads and tails take a scalar loop).
 * n == 0 returns CRM_OK without launching anything.
 */
#ifndef CRM_H
#define CRM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CRM_EXPF = 0, CRM_EXP2F, CRM_EXP10F, CRM_EXPM1F, CRM_LOGF, CRM_LOG2F, CRM_LOG10F,
  CRM_LOG1PF, CRM_SINF, CRM_COSF, CRM_SINCOSF, CRM_TANF, CRM_ASINF, CRM_ACOSF,
  CRM_ATANF, CRM_SINHF, CRM_COSHF, CRM_TANHF, CRM_RSQRTF, /* binary32 in and out */
  CRM_EXP2 = 19, CRM_LOG = 20,                             /* binary64 in and out */
  /* more binary64 functions (the formulas of expf, log2f, log10f, exp10f in binary64; one
     form, the FP64-free one; not in crm_eval_batch) */
  CRM_EXP = 21, CRM_LOG2 = 22, CRM_LOG10 = 23, CRM_EXP10 = 24,
  CRM_NUM_FUNCS = 25
} crm_func_t;

/* Element formats: binary32, binary64, and the 16-bit formats of crm_eval_rm (IEEE
   binary16; bfloat16: binary32's exponent range with 8 significant bits). */
typedef enum { CRM_F32 = 0, CRM_F64 = 1, CRM_F16 = 2, CRM_BF16 = 3 } crm_dtype_t;
/* Rounding directions (IEEE 754 Sec. 4.3): to nearest with ties to even, toward -inf,
   toward +inf, toward zero. */
typedef enum { CRM_RN = 0, CRM_RD = 1, CRM_RU = 2, CRM_RZ = 3 } crm_rmode_t;
typedef enum { CRM_FORM_AUTO = 0, CRM_FORM_PLAIN_FP64 = 1, CRM_FORM_DF32 = 2 } crm_form_t;

typedef enum {
  CRM_OK = 0,
  CRM_ERR_FUNC = 1,     /* unknown function id */
  CRM_ERR_DTYPE = 2,    /* dtype does not match the function (e.g. CRM_EXPF with F64) */
  CRM_ERR_NULL = 3,     /* null in/out with n > 0, or null descriptor array */
  CRM_ERR_OVERLAP = 4,  /* in and out overlap partially */
  CRM_ERR_CUDA = 5,     /* a CUDA runtime call failed (see crm_last_cuda_error) */
  CRM_ERR_NOMEM = 6,    /* workspace allocation failed */
  CRM_ERR_FORM = 7,     /* unknown or unavailable form */
  CRM_ERR_CAPTURE = 8,  /* workspace must grow while the stream is being captured */
  CRM_ERR_ARG = 9,      /* other invalid argument (negative count, size too large) */
  CRM_ERR_NODEV = 10,   /* no CUDA device */
  CRM_ERR_SIZE = 11     /* n exceeds CRM_NOALLOC_MAX_ELEMS (crm_eval_noalloc only) */
} crm_status_t;

/* One array of a batch (crm_eval_batch).  in/out are device pointers; out holds 2n
   elements for CRM_SINCOSF (sin in [0,n), cos in [n,2n)). */
typedef struct {
  int32_t func_id;
  int32_t dtype;
  const void *in;
  void *out;
  uint64_t n;
} crm_desc_t;

/* Counters of the (device, stream) workspace; crm_stats synchronises the stream. */
typedef struct {
  uint64_t hard_total;       /* lanes that failed a fast-path rounding test */
  uint64_t unresolved_total; /* lanes no tier could decide (0 unless something is wrong) */
  uint64_t inline_total;     /* hard lanes finished inline because the queue was full */
  uint64_t last_count;       /* hard lanes of the last call on this stream */
  uint64_t timeouts;         /* bounded device waits that gave up (0 unless something is wrong) */
  uint64_t fp64_total;       /* queued lanes whose slow path ran an FP64 tier: for binary32 the
                                double-double tier behind the FP64-free one, for binary64 every
                                queued lane (its slow path starts in double-double) */
} crm_stats_t;

/* Evaluate func_id on n elements: out[i] = RN(f(in[i])) (sincosf: out[i] = sin,
   out[n+i] = cos).  in/out: device pointers of dtype elements.  Uses the process-wide
   default form (crm_set_form, env CRM_FORM = auto|plain|df).  Asynchronous.
   Errors: CRM_ERR_FUNC, CRM_ERR_DTYPE, CRM_ERR_NULL, CRM_ERR_OVERLAP, CRM_ERR_NOMEM,
   CRM_ERR_CAPTURE, CRM_ERR_CUDA; nothing is launched on error. */
int crm_eval(int func_id, int dtype, const void *in, void *out, uint64_t n, void *stream);

/* Same with an explicit form (crm_form_t). */
int crm_eval_form(int func_id, int dtype, int form, const void *in, void *out, uint64_t n,
                  void *stream);

/* Correct rounding in any direction and in the 16-bit formats: out[i] = rmode(f(in[i])),
   f evaluated exactly and rounded once in direction rmode (crm_rmode_t) to the element
   format dtype.  The paper's CPU design ends its evaluation by rounding toward zero with a
   sticky bit and converting in the caller's rounding mode (Sec. II.A); its GPU runs, and
   crm_eval, use round-to-nearest only.  Here every fast-tier result carries the sign of
   f(x) minus a nearby binary32 (binary64) number, which fixes the rounding in every
   direction and format; lanes where that sign is undecided (f(x) on or within the error
   bound of such a number) go to the slow path, which settles exact results explicitly.
     dtype CRM_F32, CRM_F64: the function's own format (binary64 for exp2 and log); rmode
       CRM_RN is crm_eval_form with CRM_FORM_AUTO;
     dtype CRM_F16, CRM_BF16: the 19 binary32 functions on 16-bit inputs and outputs (the
       formula of the binary32 function; in and out hold uint16 bit patterns, sincosf's out
       2n of them), in all four directions.
   Special values follow the binary32 conventions in each direction (overflow gives the
   largest finite number when rounding toward zero or away from the infinity, underflow
   the smallest subnormal when rounding away from zero).  in/out: device pointers, element
   aligned; in == out allowed, other overlap CRM_ERR_OVERLAP.  Asynchronous on `stream`;
   uses the stream's workspace as crm_eval does.  Errors: CRM_ERR_FUNC, CRM_ERR_DTYPE (a
   16-bit format with exp2 or log, or a mismatched dtype), CRM_ERR_ARG (rmode, alignment),
   CRM_ERR_NULL, CRM_ERR_OVERLAP, CRM_ERR_NOMEM, CRM_ERR_CAPTURE, CRM_ERR_CUDA. */
int crm_eval_rm(int func_id, int dtype, int rmode, const void *in, void *out, uint64_t n, void *stream);

/* ---- workloads built on the library: the paper's applications (Sec. III.A) ---- */
/* Complex functions to within 2 ulp per component (the paper's "2-ulp complex expf, logf,
   sinf"): cexp(x + iy) = e^x cos y + i e^x sin y; clog(z) = log|z| + i atan2(y, x);
   csin(x + iy) = sin x cosh y + i cos x sinh y.  Each component is formed from the
   library's double-float evaluations and rounded once: within 1/2 + 2^-12 ulp of the exact
   value (the correctly rounded result or a neighbour).  in/out: device arrays of n complex
   binary32 numbers (re, im interleaved, 8-byte aligned); in == out allowed.  Valid inputs:
   finite with |re|, |im| <= 40 for cexpf and csinf (the paper's test range; beyond it a
   component may overflow), finite with 2^-60 <= max(|re|, |im|) < 2^61 for clogf; others
   give unspecified values.
   Asynchronous on `stream`; no workspace.  Errors: CRM_ERR_FUNC, CRM_ERR_NULL, CRM_ERR_ARG,
   CRM_ERR_OVERLAP, CRM_ERR_CUDA. */
#define CRM_CEXPF 0
#define CRM_CLOGF 1
#define CRM_CSINF 2
int crm_eval_complex(int cfunc, const void *in, void *out, uint64_t n, void *stream);

/* Spectral interpolation by a brute-force discrete Fourier transform on the time samples
   (the paper's first application): for each frequency freq[m] (bins, 0 or in [2^-10, N)),
     out[2m] + i out[2m+1] = sum_{n<N} x[n] (cos t_n - i sin t_n),  t_n = 2 pi frac(freq[m] n / N),
   with t_n = RN(RN(frac) RN(2 pi)) (the fraction exact in integers), sin t_n and cos t_n
   correctly rounded (sincosf), the products exact and the sum in double-float per thread,
   then binary64 (error below 2^-40 of sum |x[n]|).  x: N binary32 samples, N a power of two
   up to 2^24; freq: M binary32 values; out: 2M binary64 values (NaN for a frequency outside
   the range).  Device pointers; asynchronous on `stream`; no workspace.  Errors:
   CRM_ERR_NULL, CRM_ERR_ARG (N, alignment), CRM_ERR_CUDA. */
int crm_spectral_dft(const float *x, uint64_t N, const float *freq, uint64_t M, double *out, void *stream);

/* Host-buffer variant: in/out are host pointers.  When both are page-locked memory that
   the device addresses directly (cudaHostAlloc / cudaHostRegister on a system with
   unified addressing, as on GB300), the kernels read and write them in place over the
   host link, with no staging copies.  Otherwise (pageable memory) the library copies
   chunks to a library-owned device staging area, evaluates and copies back, overlapping
   the transfers with compute.  Either way the call returns after the results are in
   `out` (synchronous), with the same bits as crm_eval_form on device copies.  The paper
   has no counterpart (its arrays live in the CPU's memory). */
int crm_eval_host(int func_id, int dtype, int form, const void *in, void *out, uint64_t n,
                  void *stream);

/* Evaluate `count` arrays of mixed functions and uneven lengths with one
   persistent kernel (the batching form) and one slow-path kernel.  descs is host memory,
   read before return (the library keeps a page-locked copy for the upload; a CUDA graph
   that captured the call re-reads that copy at every replay).  Arrays are cut into tiles
   of 2^k elements (crm_set_batch_tile, default 2^14); each block of the persistent grid
   owns a contiguous range of tiles.  Asynchronous.  Capturable after crm_reserve(.., count).
   Binary64 arrays (exp2, log) may be mixed in; a batch that holds any runs in the grouped
   mode (crm_set_batch_mode).  A captured call owns the descriptor buffers it staged: later
   batch calls on the stream (captured or not) use new ones, so every captured graph keeps
   evaluating the arrays it captured.  A second capture on the stream needs a batch call
   outside capture, or crm_reserve, in between (else CRM_ERR_CAPTURE).  Errors: as
   crm_eval for any descriptor. */
int crm_eval_batch(const crm_desc_t *descs, int count, int form, void *stream);
/* Tile size of the batching form, 2^log2_elems elements (8 <= log2_elems <= 24). */
int crm_set_batch_tile(int log2_elems);
/* Batch mode.  CRM_BATCH_MIXED: one persistent kernel over all arrays, a block-uniform
   switch on each tile's function (2 launches per batch).  CRM_BATCH_GROUPED (default): the
   arrays are ordered by function and each function present gets one persistent kernel
   specialised for it, then one slow-path kernel for the whole batch (at most 22
   launches, one CUDA graph when captured); a function whose chosen launch shape packs
   (crm_variant_info easy, e.g. picked by crm_autotune) has its arrays packed the same way.
   Both compute the same bits. */
#define CRM_BATCH_MIXED 0
#define CRM_BATCH_GROUPED 1
int crm_set_batch_mode(int mode);

/* ---- launch shapes and the autotuner (the paper has no counterpart: its SIMD kernels
   have one shape; on the GPU the best elements-per-thread, block size and load schedule
   depend on the function and the form).  A variant is one launch shape of the main
   kernel: vectors per thread per iteration (unroll), the vector width (vec_bytes 16 or 32:
   4 or 8 binary32 elements, 2 or 4 binary64 ones per access; a 32-byte shape falls back to
   the default shape when in and out are not 32-byte congruent), threads per block,
   register prefetch of the next iteration, a minimum of resident blocks per SM (a
   register cap), or the shared-memory pipelined kernel (bulk asynchronous copies).
   reg_table: the evaluator keeps a table of at most 16 entries in registers and reads it
   with warp shuffles instead of a larger table in shared memory (the paper's small tables
   read by permutes, Sec. II.A; exp family only: other functions do not provide it).
   easy: the shape packs, across the warp, the elements whose result is not known in
   advance (tiny arguments, where f rounds to x, 1 or RN(pi/2), are resolved without the
   evaluator) and evaluates only those; functions without such arguments (log, log2, log10,
   rsqrt, the binary64 ones) do not provide it.  The autotuner times these shapes beside the
   others: they win on data whose magnitudes span many binades, and lose a little elsewhere.
   crm_eval_host on mapped host buffers runs the same shape without packing (the packed
   results are stored one by one, which the host link serves slowly).
   Every variant computes the same bits.  Output pointers may be NULL. */
#define CRM_NUM_VARIANTS 13
int crm_variant_info(int variant, int *unroll, int *block, int *prefetch, int *pipelined, int *min_blocks,
                     int *vec_bytes, int *reg_table, int *easy);
/* Choose the variant of (func_id, form) for all later calls.  CRM_ERR_ARG if the form does
   not provide it (the plain FP64 form provides only the default shape). */
int crm_set_variant(int func_id, int form, int variant);
int crm_get_variant(int func_id, int form, int *variant);
/* Time every variant of (func_id, form) on the caller's arrays (in, out: device memory,
   n elements; `reps` timed calls each after one untimed call, CUDA events on `stream`),
   keep the fastest for later calls, and return it in *best; ms (host, CRM_NUM_VARIANTS
   floats, may be NULL) receives each variant's time per call, -1 where unavailable.
   Overwrites out.  Synchronizes `stream`; CRM_ERR_CAPTURE while the stream is captured.
   The choice is process-wide (all threads, all devices). */
int crm_autotune(int func_id, int dtype, int form, const void *in, void *out, uint64_t n, int reps,
                 void *stream, int *best, float *ms);
/* Same for the batching form: times both batch modes (crm_set_batch_mode) with tile sizes
   2^CRM_BATCH_TILE_MIN .. 2^CRM_BATCH_TILE_MAX on the given batch and keeps the fastest pair
   (ms: host, 2 x 7 floats indexed [mode][log2 tile - CRM_BATCH_TILE_MIN], may be NULL).
   While it runs, the process-wide batch mode and tile size take the candidate values, so
   batches launched meanwhile from other threads use them too (every mode and tile size
   computes the same bits). */
#define CRM_BATCH_TILE_MIN 10
#define CRM_BATCH_TILE_MAX 16
int crm_autotune_batch(const crm_desc_t *descs, int count, int form, int reps, void *stream, int *best_mode,
                       int *best_shift, float *ms);

/* No-allocation variant of crm_eval_form.  The paper has no counterpart: this entry
   point exists for callers that cannot allocate device memory when they call the
   library -- work recorded under stream capture (cudaMalloc is not permitted while a
   stream is being captured), serving processes that budget every device byte at
   start-up and forbid later allocation, and code running inside another component's
   memory manager.  It computes exactly what crm_eval_form computes and allocates
   nothing: its scratch (the hard-case queue and counters) is a statically reserved
   device array of 256 + 16 * CRM_NOALLOC_MAX_ELEMS bytes (16 MiB) that every GPU which
   loads the library holds until the process exits.
   in/out: device pointers owned by the caller, as for crm_eval (out holds 2n elements
   for CRM_SINCOSF).  n must not exceed CRM_NOALLOC_MAX_ELEMS (else CRM_ERR_SIZE, nothing
   launched).  The first call on each device looks up the array's device address with
   that device current; make that first call before any stream capture.  Every call on
   a device shares the one array (each call clears the queue count it needs), so calls
   whose work overlaps on the GPU (different streams, no ordering) race and must not be
   issued.  Asynchronous on `stream`.  Other errors as crm_eval_form. */
#define CRM_NOALLOC_MAX_ELEMS (1ull << 20)
int crm_eval_noalloc(int func_id, int dtype, int form, const void *in, void *out, uint64_t n,
                     void *stream);
/* Counters of crm_eval_noalloc on the current device (the static array's header, shared by
   every call on the device; same fields as crm_stats: unresolved_total and timeouts stay 0
   unless something is wrong).  Copies them into *out after synchronising `stream`; calls
   on other streams must have completed.  Allocates nothing.  The _reset form zeroes
   them. */
int crm_noalloc_stats(void *stream, crm_stats_t *out);
int crm_noalloc_stats_reset(void *stream);

/* Process-wide default form for crm_eval (initially from env CRM_FORM, else AUTO). */
int crm_set_form(int form);

/* Pre-allocate the workspace of (current device, stream) so that later calls allocate
   nothing (required before capturing calls into a CUDA graph): the hard-case queue gets
   one entry per 64 elements of max_elems (room for a hard-case rate of 1/64 in one call;
   at least 2^21 and at most 2^26 entries of 16 bytes; lanes beyond it are finished inline,
   never dropped), and the batch descriptors room for max_arrays arrays.  A queue never
   shrinks; a replaced queue stays allocated until crm_shutdown, because a graph captured
   earlier may address it. */
int crm_reserve(uint64_t max_elems, int max_arrays, void *stream);

/* Read (and synchronise) the counters of (current device, stream). */
int crm_stats(void *stream, crm_stats_t *out);
int crm_stats_reset(void *stream);
/* The number of lanes the last call on (current device, stream) queued for the slow path
   (crm_stats' last_count): synchronises the stream and writes it to *host_out. */
int crm_hard_case_count(void *stream, uint64_t *host_out);

/* Test hook: when nonzero, every lane fails its fast-path rounding test, so the queue
   and the slow path carry the whole array (results must not change).  on = 1 also makes
   every tier of the slow path run (the last one decides); on = 2 keeps the slow path's
   early exits, so that its first tier (the FP64-free middle tier where there is one)
   decides every lane it can. */
int crm_set_force_slow(int on);

const char *crm_status_str(int status);
/* The cudaError_t of the last CRM_ERR_CUDA on this thread. */
int crm_last_cuda_error(void);
/* Release every workspace (all devices).  Not to be called while work is in flight. */
void crm_shutdown(void);
/* Library version string. */
const char *crm_version(void);

#ifdef __cplusplus
}
#endif
#endif
