// Float-float ("double-float") helpers shared by the certified re-evaluation kernels: error-free
// additions and one lens term of Eq. 2 evaluated to ~2^-44 relative on the FP32 pipe.
#pragma once

#include "rs_device.cuh"

namespace rsdev {

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah, al) += (bh, bl)
__device__ __forceinline__ void ff_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, ah, al);
}

// One lens term of Eq. 2 for ray (x1, x2) in float-float, added to (A1h, A1l), (A2h, A2l); the lens
// L = {x1, x1, x2, x2} with mass m (read only with MASS).
template <bool MASS>
__device__ __forceinline__ void lens_term_ff_at(const float4 L, float m, float x1, float x2, float& A1h, float& A1l,
                                                float& A2h, float& A2l) {
  // exact differences x - x_l as float pairs
  float ah, al, bh, bl;
  two_sum(x1, -L.x, ah, al);
  two_sum(x2, -L.z, bh, bl);
  // r^2 = (ah + al)^2 + (bh + bl)^2 to ~2^-46 relative (al^2, bl^2 dropped)
  const float p = __fmul_rn(ah, ah);
  float pe = __fmaf_rn(ah, ah, -p);
  pe = __fmaf_rn(__fmul_rn(2.f, ah), al, pe);
  const float q = __fmul_rn(bh, bh);
  float qe = __fmaf_rn(bh, bh, -q);
  qe = __fmaf_rn(__fmul_rn(2.f, bh), bl, qe);
  float s, se;
  two_sum(p, q, s, se);
  se = __fadd_rn(se, __fadd_rn(pe, qe));
  float rh, rl;
  fast_two_sum(s, se, rh, rl);
  // w = 1 / r^2: approximate reciprocal plus one Newton correction from the exact residual
  const float w0 = rcp_approx(rh);
  float e = __fmaf_rn(-rh, w0, 1.f);
  e = __fmaf_rn(-rl, w0, e);
  float wh, wl;
  fast_two_sum(w0, __fmul_rn(w0, e), wh, wl);
  if (MASS) {
    const float mh = __fmul_rn(wh, m);
    float ml = __fmaf_rn(wh, m, -mh);
    ml = __fmaf_rn(wl, m, ml);
    fast_two_sum(mh, ml, wh, wl);
  }
  // terms w * d, accumulated in float-float
  const float t1h = __fmul_rn(wh, ah);
  float t1l = __fmaf_rn(wh, ah, -t1h);
  t1l = __fmaf_rn(wh, al, t1l);
  t1l = __fmaf_rn(wl, ah, t1l);
  const float t2h = __fmul_rn(wh, bh);
  float t2l = __fmaf_rn(wh, bh, -t2h);
  t2l = __fmaf_rn(wh, bl, t2l);
  t2l = __fmaf_rn(wl, bh, t2l);
  ff_add(A1h, A1l, t1h, t1l);
  ff_add(A2h, A2l, t2h, t2l);
}

// Lens l of field f (see lens_term_ff_at).
template <bool MASS>
__device__ __forceinline__ void lens_term_ff(const FieldDev& f, int l, float x1, float x2, float& A1h, float& A1l,
                                             float& A2h, float& A2l) {
  lens_term_ff_at<MASS>(__ldg(f.lens4 + l), MASS ? __ldg(f.mass2 + l).x : 0.f, x1, x2, A1h, A1l, A2h, A2l);
}

// Lenses l0, l0 + stride, ... (< n) of field f in that order, four loads in flight at a time (the terms
// are still added one after the other, in lens order).
template <bool MASS>
__device__ __forceinline__ void lens_terms_ff_strided(const FieldDev& f, int l0, int stride, int n, float x1, float x2,
                                                      float& A1h, float& A1l, float& A2h, float& A2l) {
  int l = l0;
  for (; l + 3 * stride < n; l += 4 * stride) {
    float4 L[4];
    float m[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      L[k] = __ldg(f.lens4 + l + k * stride);
      m[k] = MASS ? __ldg(f.mass2 + l + k * stride).x : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) lens_term_ff_at<MASS>(L[k], m[k], x1, x2, A1h, A1l, A2h, A2l);
  }
  for (; l < n; l += stride) lens_term_ff<MASS>(f, l, x1, x2, A1h, A1l, A2h, A2l);
}

// Lanes per listed ray of the float-float evaluation: one warp for fields of up to kFfSmallField
// lenses, kFfWarps warps above (a single warp over 1e8 lenses is latency-bound for a fraction of a
// second per ray).  The lens split and the reduction order depend only on the lens count, so every
// kernel that evaluates a ray in float-float gets the same value.
constexpr int kFfSmallField = 1 << 16;
constexpr int kFfWarps = 16;
__host__ __device__ __forceinline__ int ff_warps(int n_lens) { return n_lens > kFfSmallField ? kFfWarps : 1; }

// Float-float deflection of one ray by lenses [0, f.n_lens) of a field, summed by the W warps of a
// group: lane lam = w * 32 + lane sums lenses lam, lam + 32 W, ... in order; each warp's 32 partials
// are combined by a fixed shuffle tree (16, 8, 4, 2, 1) and warp 0 adds warps 1 .. W-1 in order
// through red (W entries of shared memory).  Every thread of the group must call it with the same
// ray; W > 1 needs the whole CTA (a __syncthreads inside).  Thread 0 of the group returns alpha as
// float pairs {a1 hi, a1 lo, a2 hi, a2 lo}.
template <bool MASS>
__device__ __forceinline__ float4 deflect_ff_group(const FieldDev& f, float x1, float x2, int W, int w, float4* red) {
  const int lane = threadIdx.x & 31;
  float A1h = 0.f, A1l = 0.f, A2h = 0.f, A2l = 0.f;
  lens_terms_ff_strided<MASS>(f, w * 32 + lane, 32 * W, f.n_lens, x1, x2, A1h, A1l, A2h, A2l);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float b1h = __shfl_down_sync(0xffffffffu, A1h, off);
    const float b1l = __shfl_down_sync(0xffffffffu, A1l, off);
    const float b2h = __shfl_down_sync(0xffffffffu, A2h, off);
    const float b2l = __shfl_down_sync(0xffffffffu, A2l, off);
    ff_add(A1h, A1l, b1h, b1l);
    ff_add(A2h, A2l, b2h, b2l);
  }
  if (W > 1) {
    if (lane == 0) red[w] = make_float4(A1h, A1l, A2h, A2l);
    __syncthreads();
    if (w == 0 && lane == 0)
      for (int k = 1; k < W; ++k) {
        const float4 o = red[k];
        ff_add(A1h, A1l, o.x, o.y);
        ff_add(A2h, A2l, o.z, o.w);
      }
    __syncthreads();  // red is free again
  }
  return make_float4(A1h, A1l, A2h, A2l);
}

// deflect_ff_group for R rays of one field in one pass over the lenses: every lens a lane loads serves
// all R rays, and each ray's terms, shuffle tree and warp order are those of deflect_ff_group, so each
// ray gets the same bits as alone.  red: W * R entries of shared memory.  Thread 0 of the group
// returns the R results in out.
template <bool MASS, int R>
__device__ __forceinline__ void deflect_ff_group_rays(const FieldDev& f, const float (&x1)[R], const float (&x2)[R],
                                                      int W, int w, float4* red, float4 (&out)[R]) {
  const int lane = threadIdx.x & 31;
  const int stride = 32 * W, n = f.n_lens;
  float A1h[R], A1l[R], A2h[R], A2l[R];
#pragma unroll
  for (int r = 0; r < R; ++r) A1h[r] = A1l[r] = A2h[r] = A2l[r] = 0.f;
  int l = w * 32 + lane;
  for (; l + stride < n; l += 2 * stride) {  // two lenses in flight; each ray still adds them in lens order
    const float4 L0 = __ldg(f.lens4 + l), L1 = __ldg(f.lens4 + l + stride);
    const float m0 = MASS ? __ldg(f.mass2 + l).x : 0.f, m1 = MASS ? __ldg(f.mass2 + l + stride).x : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) lens_term_ff_at<MASS>(L0, m0, x1[r], x2[r], A1h[r], A1l[r], A2h[r], A2l[r]);
#pragma unroll
    for (int r = 0; r < R; ++r) lens_term_ff_at<MASS>(L1, m1, x1[r], x2[r], A1h[r], A1l[r], A2h[r], A2l[r]);
  }
  if (l < n) {
    const float4 L0 = __ldg(f.lens4 + l);
    const float m0 = MASS ? __ldg(f.mass2 + l).x : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) lens_term_ff_at<MASS>(L0, m0, x1[r], x2[r], A1h[r], A1l[r], A2h[r], A2l[r]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float b1h = __shfl_down_sync(0xffffffffu, A1h[r], off);
      const float b1l = __shfl_down_sync(0xffffffffu, A1l[r], off);
      const float b2h = __shfl_down_sync(0xffffffffu, A2h[r], off);
      const float b2l = __shfl_down_sync(0xffffffffu, A2l[r], off);
      ff_add(A1h[r], A1l[r], b1h, b1l);
      ff_add(A2h[r], A2l[r], b2h, b2l);
    }
  }
  if (W > 1) {
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < R; ++r) red[w * R + r] = make_float4(A1h[r], A1l[r], A2h[r], A2l[r]);
    __syncthreads();
    if (w == 0 && lane == 0)
      for (int k = 1; k < W; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 o = red[k * R + r];
          ff_add(A1h[r], A1l[r], o.x, o.y);
          ff_add(A2h[r], A2l[r], o.z, o.w);
        }
    __syncthreads();  // red is free again
  }
#pragma unroll
  for (int r = 0; r < R; ++r) out[r] = make_float4(A1h[r], A1l[r], A2h[r], A2l[r]);
}

// Eq. 6 and the pixel of a re-evaluated ray in float64: y = lam x - alpha with alpha1 = a.x + a.y,
// alpha2 = a.z + a.w (float pairs, exact in float64), u = (y - lo) * sc.  True with pix = p2 * np0 + p1
// (p = floor(u)) inside the window; false outside it (or for a ray on a lens: NaN compares false).
__device__ __forceinline__ bool ff_map_bin(const ShootDesc& d, float x1, float x2, float4 a, size_t& pix) {
  const double a1 = (double)a.x + (double)a.y, a2 = (double)a.z + (double)a.w;
  const double y1 = __dsub_rn(__dmul_rn(d.f.lam1, (double)x1), a1);
  const double y2 = __dsub_rn(__dmul_rn(d.f.lam2, (double)x2), a2);
  const double u1 = __dmul_rn(__dsub_rn(y1, d.lo0), d.sc0);
  const double u2 = __dmul_rn(__dsub_rn(y2, d.lo1), d.sc1);
  if (!((u1 >= 0.0) && (u1 < (double)d.np0) && (u2 >= 0.0) && (u2 < (double)d.np1))) return false;
  pix = (size_t)(int)floor(u2) * (size_t)d.np0 + (size_t)(int)floor(u1);
  return true;
}

}  // namespace rsdev
