// k_complex.cu -- workloads built on the library's evaluators (the paper's applications,
// Sec. III.A): complex expf, logf and sinf to within 2 ulp, and spectral interpolation by
// a brute-force discrete Fourier transform whose sines and cosines are correctly rounded.
//
// Complex functions: each component is formed from the double-float pairs of the real
// evaluators (fast tiers, relative error below 2^-37 each) and rounded once:
//   cexp(x + iy) = e^x cos y + i e^x sin y,   csin(x + iy) = sin x cosh y + i cos x sinh y,
//   clog(z) = log|z| + i atan2(y, x),  log|z| = log(x^2 + y^2)/2 from the exact pair x^2 + y^2.
// A product of two pairs is good to 2^-36 of itself, so every component is within
// 1/2 + 2^-12 ulp of the exact value (faithful: the correctly rounded value or a neighbour),
// inside the paper's 2-ulp target.  The paper composes its correctly rounded real functions
// instead (a product of two rounded results is only within about 2.5 ulp in the worst case).
//
// Spectral interpolation: for each frequency f (0 <= f < N, N = 2^k samples x[n]),
//   X(f) = sum_n x[n] (cos theta_n - i sin theta_n),  theta_n = 2 pi frac(f n / N),
// with the phase formed exactly in integers (f n / N is a dyadic rational) and rounded once
// to binary32, theta_n = RN(RN(phase) * RN(2 pi)); sin and cos of theta_n correctly rounded
// (the library's sincosf, slow path inline for its rare hard lanes); x[n] cos and x[n] sin
// as exact products summed in double-float per thread, then in double across the block.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/crm.h"
#include "crm_fns.cuh"
#include "crm_internal.h"

namespace crm {

enum { CX_EXPF = 0, CX_LOGF = 1, CX_SINF = 2 };

// shared-memory tables: exp (64 x float4), trig (2/pi words, (sin, cos)(j pi/64), window
// entries), atan (17 pairs), ln (193 x float4)
constexpr int CXT_EXP = 0, CXT_TRIG = CXT_EXP + 64 * 16;
constexpr int CXT_ATAN = CXT_TRIG + FnTrig<TRIG_SINCOS>::tab_bytes<2>();
constexpr int CXT_LOG = CXT_ATAN + 18 * 8;
constexpr int CXT_BYTES = CXT_LOG + 193 * 16;

// sin and cos of y as pairs (trig_df_core's rotation by the quadrant)
CRM_DEV void sincos_pairs(float y, const unsigned char *sm, Pair<float> &sn, Pair<float> &cs) {
  const unsigned char *b = sm + CXT_TRIG;
  const TrigF R = trig_df_core<TRIG_SINCOS>(y, (const uint4 *)(b + FnTrig<TRIG_SINCOS>::OFF_PW),
                                            (const float4 *)(b + 64));
  const bool odd = (R.q & 1) != 0;
  sn = odd ? R.B : R.A;
  cs = odd ? R.A : R.B;
  if (trig_sin_sign(R.q, y)) sn = -sn;
  if (trig_cos_sign(R.q)) cs = -cs;
}

// a 2^k (k in [-126, 127]) rounded once from the unnormalised pair
CRM_DEV float pair_scaled(Pair<float> p, int k) {
  if (k > 63) {  // two steps keep every power of two representable
    p.hi *= 0x1p63f;
    p.lo *= 0x1p63f;
    k -= 63;
  } else if (k < -63) {
    p.hi *= 0x1p-63f;
    p.lo *= 0x1p-63f;
    k += 63;
  }
  const float s = bitsf((uint32_t)(k + 127) << 23);
  return fma_(p.hi, s, p.lo * s);
}

template <int W> CRM_DEV float2 cx_eval(float x, float y, const unsigned char *sm) {
  float2 out;
  if (W == CX_EXPF) {
    float s, r;
    uint32_t sb;
    exp_df_core<0>(x, (const float4 *)(sm + CXT_EXP), s, r, sb);
    int k = (int)(sb - fbits(CRM_SHIFTER_F)) >> 6;
    if (k > 0) {  // scale e^x first (exactly): a tiny sin y then multiplies a large factor
      const float p = bitsf((uint32_t)(k + 127) << 23);
      s *= p;
      r *= p;
      k = 0;
    }
    Pair<float> sn, cs;
    sincos_pairs(y, sm, sn, cs);
    out.x = pair_scaled(df_mul_raw({s, r}, cs), k);
    out.y = pair_scaled(df_mul_raw({s, r}, sn), k);
  } else if (W == CX_SINF) {
    Pair<float> sn, cs;
    sincos_pairs(x, sm, sn, cs);
    const float ay = fabsf(y);
    Pair<float> ch = {1.0f, 0.0f}, sh = {ay, 0.0f};  // |y| < 2^-25: cosh = 1, sinh = |y| to 2^-51
    int kc = 0, ks = 0;
    if (ay >= 0x1p-25f) {
      ch = hyp_df_core<HYP_COSH>(ay, (const float4 *)(sm + CXT_EXP), kc);
      sh = hyp_df_core<HYP_SINH>(ay, (const float4 *)(sm + CXT_EXP), ks);
    }
    if (y < 0.0f) sh = -sh;
    out.x = pair_scaled(df_mul_raw(sn, ch), kc);
    out.y = pair_scaled(df_mul_raw(cs, sh), ks);
  } else {
    // log|z|: s = x^2 + y^2 as a pair of exact squares, scaled by 2^(2m) so that the larger
    // part is in [1, 2) (|m| <= 60 for the valid inputs, so the core's exponent e of s stays
    // below 2^7 and e ln2_hi is exact), log s by the log1p-form core on the pair (us, ul)
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay);
    int m = 127 - (int)(fbits(mx) >> 23);  // mx 2^m in [1, 2)
    m = m > 60 ? 60 : (m < -60 ? -60 : m);
    const float sc = bitsf((uint32_t)(m + 127) << 23);
    const float a = mx * sc, b = fminf(ax, ay) * sc;  // a >= b; exact (b may lose bits below 2^-126)
    // the four words of a^2 + b^2 summed with error-free steps: near |z| = 1 the sum lies
    // within 2^-24 of a power of two and its low part is the whole result
    const Pair<float> a2 = two_prod(a, a), b2 = two_prod(b, b);
    const Pair<float> hh = fast_two_sum(a2.hi, b2.hi);  // a2 >= b2
    const Pair<float> ll = two_sum(a2.lo, b2.lo);
    const Pair<float> m2 = two_sum(hh.lo, ll.hi);
    Pair<float> s = fast_two_sum(hh.hi, m2.hi);
    s.lo = s.lo + (m2.lo + ll.lo);
    s = fast_two_sum(s.hi, s.lo);
    const Pair<float> L = log_df_core<3, true>(fbits(s.hi) + ((uint32_t)(-2 * m) << 23), s.hi, s.lo, false, 0.0f,
                                               (const float4 *)(sm + CXT_LOG));
    out.x = 0.5f * (L.hi + L.lo);
    // atan2(y, x): the atan(a/b) core on (|y|, |x|), pi minus it for x < 0, the sign of y
    Pair<float> t = atan_ratio_df({ay, 0.0f}, {ax, 0.0f}, (const float2 *)(sm + CXT_ATAN));
    if (fbits(x) >> 31) t = df_add_ordered_raw({CRM_PI_F_HI, CRM_PI_F_LO}, -t);
    const float th = t.hi + t.lo;
    out.y = (fbits(y) >> 31) ? -th : th;
  }
  return out;
}

template <int W> __global__ void __launch_bounds__(KBLOCK) k_complex(const float2 *in, float2 *out, uint64_t n) {
  __shared__ __align__(16) unsigned char sm[CXT_BYTES];
  FnExp<0>::load<2>(sm + CXT_EXP);
  FnTrig<TRIG_SINCOS>::load<2>(sm + CXT_TRIG);
  FnAtrig<AT_ATAN>::load<2>(sm + CXT_ATAN);
  FnLog<0>::load<2>(sm + CXT_LOG);
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * KBLOCK + threadIdx.x; i < n; i += (uint64_t)gridDim.x * KBLOCK) {
    const float2 z = in[i];
    out[i] = cx_eval<W>(z.x, z.y, sm);
  }
}

// ------------------------------------------------------------------ spectral interpolation
// theta = RN(RN(u) 2^-w RN(2 pi)) with u 2^-w = frac(f n / N) exactly: f = Mf 2^ef, N = 2^lg,
// f n / N = Mf n 2^(ef - lg), so the fraction is (Mf n mod 2^w) 2^-w with w = lg - ef (0 when
// w <= 0; Mf n < 2^48 when w >= 48).  f must lie in [2^-10, N) (or be 0): then w <= lg + 33.
CRM_DEV float dft_phase(float f, uint32_t n, int lg) {
  const uint32_t fb = fbits(f);
  if ((fb & 0x7FFFFFFFu) == 0) return 0.0f;
  const uint64_t Mf = (fb & 0x007FFFFFu) | 0x00800000u;
  const int w = lg - ((int)(fb >> 23) - 150);
  if (w <= 0) return 0.0f;
  uint64_t u = Mf * (uint64_t)n;
  if (w < 64) u &= (1ull << w) - 1ull;
  const float p = __ull2float_rn(u) * bitsf((uint32_t)(127 - w) << 23);  // exact scaling (w <= 126)
  return p * 0x1.921fb6p+2f;                                             // RN(2 pi)
}

__global__ void __launch_bounds__(KBLOCK) k_spectral(const float *x, uint64_t N, int lg, const float *freq,
                                                      uint64_t M, double *out) {
  __shared__ __align__(16) unsigned char sm[FnTrig<TRIG_SINCOS>::tab_bytes<2>()];
  __shared__ double red[2][KBLOCK / 32];
  FnTrig<TRIG_SINCOS>::load<2>(sm);
  __syncthreads();
  for (uint64_t m = blockIdx.x; m < M; m += gridDim.x) {
    const float f = freq[m];
    const bool ok = f == 0.0f || (f >= 0x1p-10f && f < (float)N);
    // per-thread double-float sums of x cos (re) and -x sin (im)
    float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
    for (uint64_t n = threadIdx.x; n < N; n += KBLOCK) {
      const float th = dft_phase(f, (uint32_t)n, lg);
      float y[2];
      bool h;
      FnTrig<TRIG_SINCOS>::eval<2>(th, sm, y, h);
      if (h) {  // the correctly rounded values from the slow path (rare lanes)
        int st;
        FnTrig<TRIG_SINCOS>::slow(th, y, st, false);
      }
      const float xn = x[n];
      const Pair<float> pc = two_prod(xn, y[1]), ps = two_prod(xn, -y[0]);
      Pair<float> a = two_sum(rh, pc.hi);
      rl = rl + (a.lo + pc.lo);
      rh = a.hi;
      a = two_sum(ih, ps.hi);
      il = il + (a.lo + ps.lo);
      ih = a.hi;
    }
    double re = (double)rh + (double)rl, im = (double)ih + (double)il;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xFFFFFFFFu, re, o);
      im += __shfl_down_sync(0xFFFFFFFFu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = re;
      red[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int wv = 0; wv < KBLOCK / 32; wv++) {
        sr += red[0][wv];
        si += red[1][wv];
      }
      out[2 * m] = ok ? sr : CRM_QNAN_D;
      out[2 * m + 1] = ok ? si : CRM_QNAN_D;
    }
    __syncthreads();
  }
}

}  // namespace crm

using namespace crm;

extern "C" int crm_eval_complex(int cfunc, const void *in, void *out, uint64_t n, void *stream) {
  ensure_init();
  if (cfunc < CRM_CEXPF || cfunc > CRM_CSINF) return CRM_ERR_FUNC;
  if (n == 0) return CRM_OK;
  if (!in || !out) return CRM_ERR_NULL;
  if (((uintptr_t)in % 8) || ((uintptr_t)out % 8) || n > (1ull << 40)) return CRM_ERR_ARG;
  const uintptr_t a0 = (uintptr_t)in, a1 = a0 + 8 * n, b0 = (uintptr_t)out, b1 = b0 + 8 * n;
  if (a0 != b0 && a0 < b1 && b0 < a1) return CRM_ERR_OVERLAP;
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *sym = cfunc == CRM_CEXPF ? (const void *)k_complex<CX_EXPF>
                                       : (cfunc == CRM_CLOGF ? (const void *)k_complex<CX_LOGF> : (const void *)k_complex<CX_SINF>);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sym, KBLOCK, 0);
  if (e != cudaSuccess) return cuda_fail_code(e);
  const uint64_t want = (n + KBLOCK - 1) / KBLOCK, cap = (uint64_t)sms * (bps > 0 ? bps : 1);
  const int grid = (int)(want < cap ? want : cap);
  cudaStream_t s = (cudaStream_t)stream;
  const float2 *zi = (const float2 *)in;
  float2 *zo = (float2 *)out;
  if (cfunc == CRM_CEXPF) k_complex<CX_EXPF><<<grid, KBLOCK, 0, s>>>(zi, zo, n);
  else if (cfunc == CRM_CLOGF) k_complex<CX_LOGF><<<grid, KBLOCK, 0, s>>>(zi, zo, n);
  else k_complex<CX_SINF><<<grid, KBLOCK, 0, s>>>(zi, zo, n);
  e = cudaGetLastError();
  return e == cudaSuccess ? CRM_OK : cuda_fail_code(e);
}

extern "C" int crm_spectral_dft(const float *x, uint64_t N, const float *freq, uint64_t M, double *out,
                                void *stream) {
  ensure_init();
  if (M == 0) return CRM_OK;
  if (!x || !freq || !out) return CRM_ERR_NULL;
  if (N == 0 || (N & (N - 1)) || N > (1ull << 24)) return CRM_ERR_ARG;
  if (((uintptr_t)x % 4) || ((uintptr_t)freq % 4) || ((uintptr_t)out % 8)) return CRM_ERR_ARG;
  int lg = 0;
  while ((1ull << lg) < N) lg++;
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)k_spectral, KBLOCK, 0);
  if (e != cudaSuccess) return cuda_fail_code(e);
  const uint64_t cap = (uint64_t)sms * (bps > 0 ? bps : 1);
  const int grid = (int)(M < cap ? M : cap);
  k_spectral<<<grid, KBLOCK, 0, (cudaStream_t)stream>>>(x, N, lg, freq, M, out);
  e = cudaGetLastError();
  return e == cudaSuccess ? CRM_OK : cuda_fail_code(e);
}
