// Certified binning: float-float re-evaluation of the rays the float32 shoot could not bin with
// certainty (source position within its error band of a pixel or window edge).
//
// Each listed ray's deflection (Eq. 2) is summed again over all lenses of its field in
// float-float ("double-float") arithmetic on the FP32 pipe -- about 2^-44 relative per term,
// far cheaper on GB300 than float64 -- then mapped (Eq. 6) and binned with the float64 arithmetic of
// the definition.  One warp per listed ray (sixteen for fields of more than 2^16 lenses): the lanes
// split the lens loop (coalesced lens loads) and a fixed reduction order combines them, so the result
// is deterministic.
#include <algorithm>

#include "rs_ff.cuh"
#include "rs_internal.h"

namespace {

using namespace rsdev;

// Warps of a CTA of the re-evaluation kernels with W warps per listed ray: W = 1, four rays per CTA;
// W = kFfWarps, one ray per CTA.
template <int W>
__host__ __device__ constexpr int ff_cta_warps() {
  return W == 1 ? 4 : W;
}

// Float-float deflection of ray (x1, x2) of field f by the calling group (all W warps of it).
template <int W>
__device__ __forceinline__ float4 ff_alpha(const FieldDev& f, float x1, float x2, float4* red) {
  const int w = (int)(threadIdx.x >> 5) % W;
  return f.has_mass ? deflect_ff_group<true>(f, x1, x2, W, w, red) : deflect_ff_group<false>(f, x1, x2, W, w, red);
}

// Listed rays whose field takes W warps per ray (the others are left to the kernel of their W): each
// group of W warps evaluates one ray at a time, then its first thread maps (Eq. 6) and bins with the
// float64 arithmetic of the definition.
template <int W, bool SINGLE>
__global__ void __launch_bounds__(32 * ff_cta_warps<W>()) recheck_kernel(const ShootDesc one,
                                                                         const ShootDesc* __restrict__ descs,
                                                                         const uint2* __restrict__ list,
                                                                         const unsigned int* __restrict__ count,
                                                                         unsigned int cap) {
  __shared__ float4 red[W];
  constexpr int G = ff_cta_warps<W>() / W;  // groups per CTA
  const unsigned int n = min(*count, cap);
  const unsigned int g = threadIdx.x / (32 * W);
  for (unsigned int e0 = blockIdx.x * G; e0 < n; e0 += gridDim.x * G) {  // CTA-uniform
    const unsigned int e = e0 + g;
    if (e >= n) continue;  // only when G > 1, where no barrier is used
    const uint2 it = list[e];
    const ShootDesc& d = SINGLE ? one : descs[it.x];
    if (ff_warps(d.f.n_lens) != W) continue;  // uniform over the group
    const int64_t r = (int64_t)it.y;
    const int64_t jrel = r / d.n0;
    const int64_t i = r - jrel * d.n0;
    const float x1 = ray_coord(i, d.sp0, d.or0);
    const float x2 = ray_coord(d.j_begin + jrel, d.sp1, d.or1);
    const float4 a = ff_alpha<W>(d.f, x1, x2, red);
    if ((threadIdx.x & (32 * W - 1)) != 0) continue;
    size_t pix = 0;
    if (ff_map_bin(d, x1, x2, a, pix)) {
      atomicAdd(d.counts + pix, 1u);
    } else if (d.oow != nullptr) {
      atomicAdd(d.oow, 1ull);
    }
  }
}

// Listed rays of one field with W > 1 warps per ray, up to kRaysPerPass at a time: each ray of a
// field this large streams the whole lens array, so one pass serves several (one field's lenses from
// DRAM once per pass instead of once per ray).  CTA b takes entries [n b / grid, n (b + 1) / grid)
// of the list; the per-ray arithmetic is recheck_kernel's, so the counts are the same bits.
constexpr int kRaysPerPass = 4;

template <int W, int R>
__device__ __forceinline__ void recheck_rays(const ShootDesc& d, const uint2* __restrict__ list, unsigned int e,
                                             float4* red) {
  float x1[R], x2[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t ray = (int64_t)list[e + r].y;
    const int64_t jrel = ray / d.n0;
    x1[r] = ray_coord(ray - jrel * d.n0, d.sp0, d.or0);
    x2[r] = ray_coord(d.j_begin + jrel, d.sp1, d.or1);
  }
  float4 a[R];
  const int w = (int)(threadIdx.x >> 5);
  if (d.f.has_mass)
    deflect_ff_group_rays<true, R>(d.f, x1, x2, W, w, red, a);
  else
    deflect_ff_group_rays<false, R>(d.f, x1, x2, W, w, red, a);
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    size_t pix = 0;
    if (ff_map_bin(d, x1[r], x2[r], a[r], pix))
      atomicAdd(d.counts + pix, 1u);
    else if (d.oow != nullptr)
      atomicAdd(d.oow, 1ull);
  }
}

template <int W>
__global__ void __launch_bounds__(32 * W) recheck_field_kernel(const ShootDesc d, const uint2* __restrict__ list,
                                                               const unsigned int* __restrict__ count,
                                                               unsigned int cap) {
  __shared__ float4 red[W * kRaysPerPass];
  const uint64_t n = min(*count, cap);
  const unsigned int lo = (unsigned int)(n * blockIdx.x / gridDim.x);
  const unsigned int hi = (unsigned int)(n * (blockIdx.x + 1) / gridDim.x);
  for (unsigned int e = lo; e < hi;) {  // CTA-uniform
    const unsigned int k = min(hi - e, (unsigned int)kRaysPerPass);
    if (k == 4)
      recheck_rays<W, 4>(d, list, e, red);
    else if (k == 3)
      recheck_rays<W, 3>(d, list, e, red);
    else if (k == 2)
      recheck_rays<W, 2>(d, list, e, red);
    else
      recheck_rays<W, 1>(d, list, e, red);
    e += k;
  }
}

// Listed rays of rs_trace_certified: the same evaluation as the re-evaluation above.
template <int W>
__global__ void __launch_bounds__(32 * ff_cta_warps<W>()) trace_ff_kernel(const FieldDev f, double or0, double or1,
                                                                          double sp0, double sp1,
                                                                          const int64_t* __restrict__ ij, int64_t k,
                                                                          double* __restrict__ y,
                                                                          double* __restrict__ alpha) {
  __shared__ float4 red[W];
  constexpr int G = ff_cta_warps<W>() / W;
  const int64_t r = (int64_t)blockIdx.x * G + threadIdx.x / (32 * W);
  if (r >= k) return;  // whole groups leave together (W > 1: one group per CTA)
  const float x1 = ray_coord(ij[2 * r], sp0, or0);
  const float x2 = ray_coord(ij[2 * r + 1], sp1, or1);
  const float4 a = ff_alpha<W>(f, x1, x2, red);
  if ((threadIdx.x & (32 * W - 1)) != 0) return;
  const double a1 = (double)a.x + (double)a.y, a2 = (double)a.z + (double)a.w;
  y[2 * r] = __dsub_rn(__dmul_rn(f.lam1, (double)x1), a1);
  y[2 * r + 1] = __dsub_rn(__dmul_rn(f.lam2, (double)x2), a2);
  if (alpha != nullptr) {
    alpha[2 * r] = a1;
    alpha[2 * r + 1] = a2;
  }
}

template <int W>
cudaError_t launch_recheck_w(const ShootDesc* single, const ShootDesc* descs, const uint2* list,
                             const unsigned int* count, unsigned int cap, int grid, cudaStream_t s) {
  constexpr int T = 32 * ff_cta_warps<W>();
  if (single != nullptr)
    recheck_kernel<W, true><<<grid, T, 0, s>>>(*single, nullptr, list, count, cap);
  else
    recheck_kernel<W, false><<<grid, T, 0, s>>>(ShootDesc{}, descs, list, count, cap);
  return cudaGetLastError();
}

}  // namespace

namespace rsint {

cudaError_t launch_recheck(const rsdev::ShootDesc* single, const rsdev::ShootDesc* descs, const uint2* list,
                           const unsigned int* count, unsigned int cap, int grid, cudaStream_t s) {
  if (cap == 0) return cudaSuccess;
  // grid: CTAs of the one-warp kernel (eight per SM); the 16-warp kernel runs two per SM
  const bool small = single == nullptr || rsdev::ff_warps(single->f.n_lens) == 1;
  const bool large = single == nullptr || rsdev::ff_warps(single->f.n_lens) > 1;
  cudaError_t e = cudaSuccess;
  if (small) e = launch_recheck_w<1>(single, descs, list, count, cap, grid, s);
  if (e == cudaSuccess && large) {
    if (single != nullptr) {  // one field: several listed rays per pass over its lenses
      recheck_field_kernel<rsdev::kFfWarps><<<std::max(1, grid / 4), 32 * rsdev::kFfWarps, 0, s>>>(*single, list,
                                                                                                 count, cap);
      e = cudaGetLastError();
    } else {
      e = launch_recheck_w<rsdev::kFfWarps>(single, descs, list, count, cap, std::max(1, grid / 4), s);
    }
  }
  return e;
}

cudaError_t launch_trace_ff(const rsdev::FieldDev& f, double or0, double or1, double sp0, double sp1,
                            const int64_t* ij, int64_t k, double* y, double* alpha, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if (rsdev::ff_warps(f.n_lens) == 1) {
    const int64_t grid = (k + 3) / 4;  // four warps (rays) per 128-thread CTA
    trace_ff_kernel<1><<<(unsigned)grid, 128, 0, s>>>(f, or0, or1, sp0, sp1, ij, k, y, alpha);
  } else {
    trace_ff_kernel<rsdev::kFfWarps><<<(unsigned)k, 32 * rsdev::kFfWarps, 0, s>>>(f, or0, or1, sp0, sp1, ij, k, y,
                                                                                  alpha);
  }
  return cudaGetLastError();
}

}  // namespace rsint
