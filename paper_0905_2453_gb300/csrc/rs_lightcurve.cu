// Light curves of magnification maps (Section 1): the profile-weighted mean of a map around each
// sample of a straight source track, and its magnitude change -2.5 log10 mu.
//
// One thread per sample; the 32 samples of a warp are consecutive samples of (mostly) one track,
// so the warp's loads of neighbouring pixels fall in the same L1 lines and every per-sample
// float64 step (position, box, quotient) is paid once per thread, not once per pixel.  A thread
// walks the rows of the box that bounds its profile's support and, per row, the chord of the
// support (a margin of ~2^-10 pixel each side).  With E = (di)^2 a0 + (dj)^2 a1 the float32 exponent of
// the pixel offset (di, dj) in pixel units, the chord's interior (E below the cut by more than a
// guard band, same margin) is summed without tests; at the rim membership is decided from
// E, and pixels whose E lies within the guard band repeat the float64 test
// ((lo + (i + 0.5) pix) - y)^2 + (...)^2 <= cut^2 (no fused multiply-add), so the covered pixel set
// is exactly that of a float64 evaluation.
// Gaussian weights are 2^-E with the exponent pre-scaled by log2(e) (one MUFU ex2).  Each row's
// partial sums are plain float32 (at most 2 R / pix + 3 terms); the rows are folded into compensated
// (TwoSum) float32 pairs and the mean is their float-float quotient.
#include "rs_internal.h"

namespace {

using rsint::LcTrack;

__device__ __forceinline__ void acc_two_sum(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
  s = t;
}

// sqrt(x) for x >= 0 from the hardware reciprocal square root (a few ulp; used for chord bounds
// that carry a margin of 2^-10 + 2^-16 h pixels, h the half-chord)
__device__ __forceinline__ float sqrt_approx(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

__device__ __forceinline__ float ex2_neg(float e) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-e));
  return r;
}

// The float64 membership test, written as the definition states it.
__device__ __noinline__ bool inside_f64(const LcTrack& T, int64_t k, int i, int j, double cut2) {
  const double yx = __dadd_rn(T.y00, __dmul_rn((double)k, T.st0));
  const double yy = __dadd_rn(T.y01, __dmul_rn((double)k, T.st1));
  const double cx = __dadd_rn(T.lo0, __dmul_rn((double)i + 0.5, T.pix0));
  const double cy = __dadd_rn(T.lo1, __dmul_rn((double)j + 0.5, T.pix1));
  const double dx = __dsub_rn(cx, yx);
  const double dy = __dsub_rn(cy, yy);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= cut2;
}

// A pixel near the rim of the support: decided by the float32 exponent, or by the float64 test of
// the definition when the exponent lies within the guard band of the cut.
template <int PROFILE>
__device__ __forceinline__ void rim_pixel(const LcTrack& T, int64_t k, int i, int j, int it, float fx, float a0,
                                          float ey, float ecut, float band, double cut2,
                                          const float* __restrict__ row, float& rw, float& rm) {
  const float dxp = __fsub_rn((float)(i - it), fx);
  const float e = fmaf(__fmul_rn(dxp, dxp), a0, ey);
  bool in = e <= ecut;
  if (fabsf(e - ecut) <= band) in = inside_f64(T, k, i, j, cut2);
  if (in) {
    const float w = PROFILE == 0 ? ex2_neg(e) : 1.f;
    rw = __fadd_rn(rw, w);
    rm = fmaf(w, __ldg(row + i), rm);
  }
}

// Gaussian weights are separable: 2^-(ex + ey) = 2^-ex 2^-ey.  A thread whose support box spans at most
// kLcCols columns keeps the column factors 2^-ex of its sample in shared memory (thread-private slots,
// conflict-free: slot c of thread t at c * 256 + t) and the untested chord interiors cost a load and a
// fused multiply-add per pixel; each row's interior sums are scaled by 2^-ey once.
constexpr int kLcThreads = 256;
constexpr int kLcCols = 32;

template <int PROFILE>
__global__ void __launch_bounds__(kLcThreads) light_curve_kernel(const LcTrack* __restrict__ tracks, int n_tracks,
                                                                 int64_t n_samples, double cut2, float ecut,
                                                                 double* __restrict__ mu_out,
                                                                 double* __restrict__ dm_out) {
  __shared__ float s_wx[PROFILE == 0 ? kLcCols * kLcThreads : 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_samples; g += stride) {
    // the track holding sample g: the last one whose first output position is <= g
    int lo = 0, hi = n_tracks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tracks[mid].out_off <= g) lo = mid; else hi = mid - 1;
    }
    const LcTrack& T = tracks[lo];
    const int64_t k = g - T.out_off;
    // sample position in pixel-index units (pixel i has its centre at t = i)
    const double t0 = fma((double)k, T.d0, T.t00);
    const double t1 = fma((double)k, T.d1, T.t01);
    float sw = 0.f, cw = 0.f, sm = 0.f, cm = 0.f;
    if (t0 > -T.rp0 - 2.0 && t0 < (double)T.np0 + T.rp0 + 1.0 && t1 > -T.rp1 - 2.0 &&
        t1 < (double)T.np1 + T.rp1 + 1.0) {
      const double ti = floor(t0), tj = floor(t1);
      const int it = (int)ti, jt = (int)tj;
      const float fx = (float)(t0 - ti), fy = (float)(t1 - tj);
      const float rpx = (float)T.rp0, rpy = (float)T.rp1;
      const int i_lo = max(it + (int)ceilf(fx - rpx) - 1, 0), i_hi = min(it + (int)floorf(fx + rpx) + 1, T.np0 - 1);
      const int j_lo = max(jt + (int)ceilf(fy - rpy) - 1, 0), j_hi = min(jt + (int)floorf(fy + rpy) + 1, T.np1 - 1);
      const float a0 = T.a0, a1 = T.a1, band = T.band;
      const float lim_hi = ecut + band, lim_lo = ecut - band;
      const bool sep = PROFILE == 0 && i_hi - i_lo < kLcCols;
      if (sep) {
        for (int i = i_lo; i <= i_hi; ++i) {
          const float dxp = __fsub_rn((float)(i - it), fx);
          s_wx[(i - i_lo) * kLcThreads + threadIdx.x] = ex2_neg(__fmul_rn(__fmul_rn(dxp, dxp), a0));
        }
      }
      for (int j = j_lo; j <= j_hi; ++j) {
        const float dyp = __fsub_rn((float)(j - jt), fy);
        const float ey = __fmul_rn(__fmul_rn(dyp, dyp), a1);
        const float rem_hi = lim_hi - ey;
        if (!(rem_hi >= 0.f)) continue;
        // chord of the support on this row (E <= cut + band) with a margin of 2^-10 + 2^-16 h pixels each
        // side: the float32 half-chord h is within a few 2^-24 h of its exact value (the guard band of the
        // exponent already covers the rounding of ey, a0 and the pixel offsets)
        const float hq_out = sqrt_approx(rem_hi * T.inv_a0);
        const float h_out = hq_out + fmaf(hq_out, 0x1p-16f, 0x1p-10f);
        const int c_lo = max(it + (int)ceilf(fx - h_out), i_lo);
        const int c_hi = min(it + (int)floorf(fx + h_out), i_hi);
        // interior of the chord (E <= cut - band, same margin): inside for certain, no test
        int n_lo = c_hi + 1, n_hi = c_hi;
        const float rem_lo = lim_lo - ey;
        if (rem_lo > 0.f) {
          const float hq_in = sqrt_approx(rem_lo * T.inv_a0);
          const float h_in = hq_in - fmaf(hq_in, 0x1p-16f, 0x1p-10f);
          if (h_in >= 0.f) {
            n_lo = max(it + (int)ceilf(fx - h_in), c_lo);
            n_hi = min(it + (int)floorf(fx + h_in), c_hi);
            if (n_lo > n_hi) {
              n_lo = c_hi + 1;
              n_hi = c_hi;
            }
          }
        }
        const float* __restrict__ row = T.mu + (int64_t)j * T.np0;
        float rw = 0.f, rm = 0.f;  // this row's partial sums (at most 2 R / pix + 3 terms)
        // rim pixels on the low side: float32 test, float64 test inside the guard band
        for (int i = c_lo; i < n_lo; ++i) rim_pixel<PROFILE>(T, k, i, j, it, fx, a0, ey, ecut, band, cut2, row, rw, rm);
        if (PROFILE == 0 && sep) {
          float iw = 0.f, im = 0.f;
          const float* wx = s_wx + threadIdx.x - i_lo * kLcThreads;
#pragma unroll 4
          for (int i = n_lo; i <= n_hi; ++i) {
            const float w = wx[i * kLcThreads];
            iw = __fadd_rn(iw, w);
            im = fmaf(w, __ldg(row + i), im);
          }
          if (n_lo <= n_hi) {
            const float wy = ex2_neg(ey);
            rw = fmaf(wy, iw, rw);
            rm = fmaf(wy, im, rm);
          }
        } else if (PROFILE == 0) {
          float kx = (float)(n_lo - it);
#pragma unroll 4
          for (int i = n_lo; i <= n_hi; ++i) {
            const float dxp = __fsub_rn(kx, fx);
            const float w = ex2_neg(fmaf(__fmul_rn(dxp, dxp), a0, ey));
            rw = __fadd_rn(rw, w);
            rm = fmaf(w, __ldg(row + i), rm);
            kx = __fadd_rn(kx, 1.f);
          }
        } else {
          float acc = 0.f;
#pragma unroll 4
          for (int i = n_lo; i <= n_hi; ++i) acc = __fadd_rn(acc, __ldg(row + i));
          rw = __fadd_rn(rw, (float)(n_hi - n_lo + 1));
          rm = __fadd_rn(rm, acc);
        }
        // rim pixels on the high side
        for (int i = n_hi + 1; i <= c_hi; ++i) rim_pixel<PROFILE>(T, k, i, j, it, fx, a0, ey, ecut, band, cut2, row, rw, rm);
        acc_two_sum(sw, cw, rw);
        acc_two_sum(sm, cm, rm);
      }
    }
    double m;
    if (sw > 0.f) {
      // float-float quotient (sm + cm) / (sw + cw): the residual of q sw is exact under fma
      const float q = __fdiv_rn(sm, sw);
      const float r = __fadd_rn(fmaf(-q, sw, sm), fmaf(-q, cw, cm));
      m = (double)q + (double)__fdiv_rn(r, sw);
    } else {
      m = __longlong_as_double(0x7ff8000000000000LL);
    }
    mu_out[g] = m;
    if (dm_out) dm_out[g] = (double)(-2.5f * log10f((float)m));
  }
}

}  // namespace

namespace rsint {

cudaError_t launch_light_curves(int profile, const LcTrack* tracks, int n_tracks, int64_t n_samples, double cut2,
                                float ecut, double* mu_out, double* dm_out, int grid, cudaStream_t s) {
  if (profile == 0)
    light_curve_kernel<0><<<grid, kLcThreads, 0, s>>>(tracks, n_tracks, n_samples, cut2, ecut, mu_out, dm_out);
  else
    light_curve_kernel<1><<<grid, kLcThreads, 0, s>>>(tracks, n_tracks, n_samples, cut2, ecut, mu_out, dm_out);
  return cudaGetLastError();
}

}  // namespace rsint
