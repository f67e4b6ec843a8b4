// Certified binning: float-float re-evaluation of the rays the float32 shoot could not bin with
// certainty (source position within its error band of a pixel or window edge).
//
// Each listed ray's deflection (Eq. 2) is summed again over all lenses of its field in
// float-float ("double-float") arithmetic on the FP32 pipe -- about 2^-44 relative per term,
// far cheaper on GB300 than float64 -- then mapped (Eq. 6) and binned with the float64 arithmetic of
// the definition.  One warp per listed ray: the lanes split the lens loop (coalesced lens loads) and a
// fixed reduction tree combines them, so the result is deterministic.
#include "rs_ff.cuh"
#include "rs_internal.h"

namespace {

using namespace rsdev;

// Deflection of one ray by all lenses of the field in float-float, spread over the 32 lanes of
// a warp: lane k sums lenses k, k + 32, ... in order; the 32 partial sums are combined by a fixed
// tree (shuffle-down by 16, 8, 4, 2, 1).  Every lane must call it with the same ray; lane 0
// returns alpha (the other lanes' values are partial).
template <bool MASS>
__device__ void deflect_ff_warp(const FieldDev& f, float x1, float x2, double& a1, double& a2) {
  const int lane = threadIdx.x & 31;
  float A1h = 0.f, A1l = 0.f, A2h = 0.f, A2l = 0.f;
  const int n = f.n_lens;
  for (int l = lane; l < n; l += 32) lens_term_ff<MASS>(f, l, x1, x2, A1h, A1l, A2h, A2l);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float b1h = __shfl_down_sync(0xffffffffu, A1h, off);
    const float b1l = __shfl_down_sync(0xffffffffu, A1l, off);
    const float b2h = __shfl_down_sync(0xffffffffu, A2h, off);
    const float b2l = __shfl_down_sync(0xffffffffu, A2l, off);
    ff_add(A1h, A1l, b1h, b1l);
    ff_add(A2h, A2l, b2h, b2l);
  }
  a1 = (double)A1h + (double)A1l;
  a2 = (double)A2h + (double)A2l;
}

// One warp per listed ray.
template <bool SINGLE>
__global__ void __launch_bounds__(128) recheck_kernel(const ShootDesc one, const ShootDesc* __restrict__ descs,
                                                      const uint2* __restrict__ list,
                                                      const unsigned int* __restrict__ count, unsigned int cap) {
  const unsigned int n = min(*count, cap);
  const unsigned int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned int e = warp; e < n; e += nwarps) {
    const uint2 it = list[e];
    const ShootDesc& d = SINGLE ? one : descs[it.x];
    const int64_t r = (int64_t)it.y;
    const int64_t jrel = r / d.n0;
    const int64_t i = r - jrel * d.n0;
    const float x1 = ray_coord(i, d.sp0, d.or0);
    const float x2 = ray_coord(d.j_begin + jrel, d.sp1, d.or1);
    double a1, a2;
    if (d.f.has_mass)
      deflect_ff_warp<true>(d.f, x1, x2, a1, a2);
    else
      deflect_ff_warp<false>(d.f, x1, x2, a1, a2);
    if ((threadIdx.x & 31) != 0) continue;
    const double y1 = __dsub_rn(__dmul_rn(d.f.lam1, (double)x1), a1);
    const double y2 = __dsub_rn(__dmul_rn(d.f.lam2, (double)x2), a2);
    const double u1 = __dmul_rn(__dsub_rn(y1, d.lo0), d.sc0);
    const double u2 = __dmul_rn(__dsub_rn(y2, d.lo1), d.sc1);
    const bool inwin = (u1 >= 0.0) && (u1 < (double)d.np0) && (u2 >= 0.0) && (u2 < (double)d.np1);
    if (inwin) {
      const int p1 = (int)floor(u1);
      const int p2 = (int)floor(u2);
      atomicAdd(d.counts + (size_t)p2 * (size_t)d.np0 + (size_t)p1, 1u);
    } else if (d.oow != nullptr) {
      atomicAdd(d.oow, 1ull);
    }
  }
}

// One warp per listed ray, same evaluation as the re-evaluation above.
__global__ void __launch_bounds__(128) trace_ff_kernel(const FieldDev f, double or0, double or1, double sp0,
                                                       double sp1, const int64_t* __restrict__ ij, int64_t k,
                                                       double* __restrict__ y, double* __restrict__ alpha) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= k) return;  // whole warps leave together
  const float x1 = ray_coord(ij[2 * r], sp0, or0);
  const float x2 = ray_coord(ij[2 * r + 1], sp1, or1);
  double a1, a2;
  if (f.has_mass)
    deflect_ff_warp<true>(f, x1, x2, a1, a2);
  else
    deflect_ff_warp<false>(f, x1, x2, a1, a2);
  if ((threadIdx.x & 31) != 0) return;
  y[2 * r] = __dsub_rn(__dmul_rn(f.lam1, (double)x1), a1);
  y[2 * r + 1] = __dsub_rn(__dmul_rn(f.lam2, (double)x2), a2);
  if (alpha != nullptr) {
    alpha[2 * r] = a1;
    alpha[2 * r + 1] = a2;
  }
}

}  // namespace

namespace rsint {

cudaError_t launch_recheck(const rsdev::ShootDesc* single, const rsdev::ShootDesc* descs, const uint2* list,
                           const unsigned int* count, unsigned int cap, int grid, cudaStream_t s) {
  if (cap == 0) return cudaSuccess;
  if (single != nullptr)
    recheck_kernel<true><<<grid, 128, 0, s>>>(*single, nullptr, list, count, cap);
  else
    recheck_kernel<false><<<grid, 128, 0, s>>>(rsdev::ShootDesc{}, descs, list, count, cap);
  return cudaGetLastError();
}

cudaError_t launch_trace_ff(const rsdev::FieldDev& f, double or0, double or1, double sp0, double sp1,
                            const int64_t* ij, int64_t k, double* y, double* alpha, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const int64_t grid = (k + 3) / 4;  // four warps (rays) per 128-thread CTA
  trace_ff_kernel<<<(unsigned)grid, 128, 0, s>>>(f, or0, or1, sp0, sp1, ij, k, y, alpha);
  return cudaGetLastError();
}

}  // namespace rsint
