// Lens-partitioned ("staged") shooting, the billion-lens scheme of Section 3.3: the deflection of
// every ray is summed over the lenses of one partition at a time, the partially deflected rays
// carried between passes, and the rays are mapped and binned after the last partition.  The carried
// state is the shoot kernel's own per-ray accumulators (two-float alpha sums and error-band sums)
// and the ray's largest-term bound so far (a maximum over partitions), so with partitions of
// multiples of 256 lenses the final sums and bands are bitwise those of one pass over all lenses.
// Certified binning re-evaluates the listed rays in float-float, again partition by partition.
#include <algorithm>

#include "rs_ff.cuh"
#include "rs_internal.h"

namespace {

using namespace rsdev;

constexpr int kWarps = 4, kRpt = 8, kNp = kRpt / 2, kBlock = kWarps * 32;
constexpr int kStateWords = 7;  // per ray pair: H1, L1, H2, L2, SS, AB (packed pairs), T (a float pair)

// State layout: word k (0 .. kStateWords * kNp - 1) of thread t of tile T at
// state[(T * kStateWords * kNp + k) * kBlock + t], coalesced across the threads of a CTA.
__device__ __forceinline__ void state_io(uint64_t* __restrict__ st, DeflectAcc<kNp>& a, uint64_t (&tn)[kNp],
                                         bool store) {
  uint64_t* w[kStateWords] = {a.H1, a.L1, a.H2, a.L2, a.SS, a.AB, tn};
#pragma unroll
  for (int k = 0; k < kStateWords; ++k)
#pragma unroll
    for (int q = 0; q < kNp; ++q) {
      uint64_t* p = st + (size_t)(k * kNp + q) * kBlock;
      if (store)
        p[0] = w[k][q];
      else
        w[k][q] = p[0];
    }
}

using StagedSmem = ShootSmem<kWarps, kRpt, rsint::kTile>;

template <bool MASS>
__global__ void __launch_bounds__(kBlock, 2) staged_kernel(const ShootDesc d, uint64_t* __restrict__ state, int first,
                                                           int last) {
  extern __shared__ __align__(128) unsigned char rs_smem[];
  auto& ss = *reinterpret_cast<StagedSmem*>(rs_smem);
  LensSmem<rsint::kTile, kWarps>& sm = ss.lens;
  PipeState ps;
  pipe_init(sm.bar, ps);
  constexpr int SEG = 32 * kRpt;
  const int64_t tile = blockIdx.x;
  const int64_t ncol = (d.n0 + SEG - 1) / SEG;
  const int64_t trow = tile / ncol;
  const int64_t tcol = tile - trow * ncol;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t jrel = trow * kWarps + warp;
  const bool row_ok = jrel < d.n_rows;
  const int64_t j = d.j_begin + (row_ok ? jrel : d.n_rows - 1);
  const float x2r = ray_coord(j, d.sp1, d.or1);
  float x1[kRpt], x2[kRpt];
  bool valid[kRpt];
#pragma unroll
  for (int k = 0; k < kRpt; ++k) {
    int64_t i = tcol * SEG + lane + 32 * k;
    valid[k] = row_ok && i < d.n0;
    if (i >= d.n0) i = d.n0 - 1;
    x1[k] = ray_coord(i, d.sp0, d.or0);
    x2[k] = x2r;
  }
  if (lane == 0) sm.x2row[warp] = x2r;
  if (threadIdx.x == 0) {
    const int64_t ia = tcol * SEG, ib = min(ia + SEG, d.n0) - 1;
    const int64_t ja = trow * kWarps, jb = min(ja + kWarps, d.n_rows) - 1;
    near_set_box(ss.near, 0, ray_coord(ia, d.sp0, d.or0), ray_coord(ib, d.sp0, d.or0),
                 ray_coord(d.j_begin + ja, d.sp1, d.or1), ray_coord(d.j_begin + jb, d.sp1, d.or1));
  }
  uint64_t X1[kNp], X2[kNp];
  pack_rays<kRpt>(x1, x2, X1, X2);
  DeflectAcc<kNp> acc;
  uint64_t tp[kNp];  // largest-term bound of each ray pair over the partitions so far
  uint64_t* st = state + (size_t)tile * kStateWords * kNp * kBlock + threadIdx.x;
  if (first) {
#pragma unroll
    for (int q = 0; q < kNp; ++q) acc.H1[q] = acc.L1[q] = acc.H2[q] = acc.L2[q] = acc.SS[q] = acc.AB[q] = tp[q] = 0ull;
  } else {
    state_io(st, acc, tp, false);
  }
#pragma unroll
  for (int k = 0; k < kRpt; ++k) ss.near.t[k * kBlock + threadIdx.x] = 0.f;
  __syncthreads();  // the box and the row coordinates are set
  if (!deflect_accumulate<kRpt, rsint::kTile, MASS, true, kWarps>(d.f, X1, X2, acc, sm, ps, &ss.near)) return;
  float tn[kRpt];
#pragma unroll
  for (int q = 0; q < kNp; ++q) {
    f2_unpack(tp[q], tn[2 * q], tn[2 * q + 1]);
    tn[2 * q] = fmaxf(tn[2 * q], fmaxf(ss.near.t[(2 * q) * kBlock + threadIdx.x], d.f.mcap));
    tn[2 * q + 1] = fmaxf(tn[2 * q + 1], fmaxf(ss.near.t[(2 * q + 1) * kBlock + threadIdx.x], d.f.mcap));
    tp[q] = f2_pack(tn[2 * q], tn[2 * q + 1]);
  }
  if (!last) {
    state_io(st, acc, tp, true);
    return;
  }
  float a1h[kRpt], a1l[kRpt], a2h[kRpt], a2l[kRpt], sig[kRpt];
  deflect_finish<kRpt>(acc, a1h, a1l, a2h, a2l, sig);
  bin_rays<kRpt, 32>(d, x1, x2, a1h, a1l, a2h, a2l, sig, tn, valid, jrel, tcol * SEG + lane, lane);
}

// ---- float-float re-evaluation of the listed rays, partition by partition ----------------------

// Partial float-float deflection of each listed ray by one partition, added to ff[e] = {A1h, A1l,
// A2h, A2l} (set on the first partition).  W warps per listed ray (see ff_warps), lanes split the
// partition's lenses, fixed reduction order.
template <int W, bool MASS>
__global__ void __launch_bounds__(W == 1 ? 128 : 32 * W) recheck_part_kernel(const ShootDesc d,
                                                                               const uint2* __restrict__ list,
                                                                               const unsigned int* __restrict__ count,
                                                                               unsigned int cap,
                                                                               float4* __restrict__ ff, int first) {
  __shared__ float4 red[W];
  constexpr int G = W == 1 ? 4 : 1;  // groups (rays in flight) per CTA
  const unsigned int n = min(*count, cap);
  const unsigned int g = threadIdx.x / (32 * W);
  for (unsigned int e0 = blockIdx.x * G; e0 < n; e0 += gridDim.x * G) {  // CTA-uniform
    const unsigned int e = e0 + g;
    if (e >= n) continue;  // only when G > 1, where no barrier is used
    const int64_t r = (int64_t)list[e].y;
    const int64_t jrel = r / d.n0;
    const int64_t i = r - jrel * d.n0;
    const float x1 = ray_coord(i, d.sp0, d.or0);
    const float x2 = ray_coord(d.j_begin + jrel, d.sp1, d.or1);
    float4 a = deflect_ff_group<MASS>(d.f, x1, x2, W, (int)(threadIdx.x >> 5) % W, red);
    if ((threadIdx.x & (32 * W - 1)) != 0) continue;
    if (!first) {
      const float4 o = ff[e];
      ff_add(a.x, a.y, o.x, o.y);
      ff_add(a.z, a.w, o.z, o.w);
    }
    ff[e] = a;
  }
}

// Map and bin the listed rays from their float-float deflections (as the single-pass re-evaluation).
__global__ void __launch_bounds__(128) recheck_bin_kernel(const ShootDesc d, const uint2* __restrict__ list,
                                                          const unsigned int* __restrict__ count, unsigned int cap,
                                                          const float4* __restrict__ ff) {
  const unsigned int n = min(*count, cap);
  for (unsigned int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int64_t r = (int64_t)list[e].y;
    const int64_t jrel = r / d.n0;
    const int64_t i = r - jrel * d.n0;
    const float x1 = ray_coord(i, d.sp0, d.or0);
    const float x2 = ray_coord(d.j_begin + jrel, d.sp1, d.or1);
    size_t pix = 0;
    if (ff_map_bin(d, x1, x2, ff[e], pix)) {
      atomicAdd(d.counts + pix, 1u);
    } else if (d.oow != nullptr) {
      atomicAdd(d.oow, 1ull);
    }
  }
}

}  // namespace

namespace rsint {

int64_t staged_tiles(int64_t n_rows, int64_t n0) { return shoot_tiles<kWarps, kRpt>(n_rows, n0); }

size_t staged_state_bytes(int64_t n_rows, int64_t n0) {
  return (size_t)staged_tiles(n_rows, n0) * kStateWords * kNp * kBlock * sizeof(uint64_t);
}

template <bool MASS>
cudaError_t launch_staged_m(const rsdev::ShootDesc& d, uint64_t* state, bool first, bool last, int64_t grid,
                            cudaStream_t s) {
  constexpr size_t smem = sizeof(StagedSmem);
  cudaError_t e = smem_opt_in<staged_kernel<MASS>>(smem);
  if (e != cudaSuccess) return e;
  staged_kernel<MASS><<<(unsigned)grid, kBlock, smem, s>>>(d, state, first ? 1 : 0, last ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_staged(const rsdev::ShootDesc& d, uint64_t* state, bool first, bool last, cudaStream_t s) {
  const int64_t grid = staged_tiles(d.n_rows, d.n0);
  if (grid <= 0) return cudaSuccess;
  if (grid >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  return d.f.has_mass ? launch_staged_m<true>(d, state, first, last, grid, s)
                      : launch_staged_m<false>(d, state, first, last, grid, s);
}

cudaError_t launch_recheck_part(const rsdev::ShootDesc& d, const uint2* list, const unsigned int* count,
                                unsigned int cap, float4* ff, bool first, int grid, cudaStream_t s) {
  if (cap == 0) return cudaSuccess;
  const int f = first ? 1 : 0;
  if (ff_warps(d.f.n_lens) == 1) {
    if (d.f.has_mass)
      recheck_part_kernel<1, true><<<grid, 128, 0, s>>>(d, list, count, cap, ff, f);
    else
      recheck_part_kernel<1, false><<<grid, 128, 0, s>>>(d, list, count, cap, ff, f);
  } else {
    const int g = std::max(1, grid / 4), t = 32 * kFfWarps;
    if (d.f.has_mass)
      recheck_part_kernel<kFfWarps, true><<<g, t, 0, s>>>(d, list, count, cap, ff, f);
    else
      recheck_part_kernel<kFfWarps, false><<<g, t, 0, s>>>(d, list, count, cap, ff, f);
  }
  return cudaGetLastError();
}

cudaError_t launch_recheck_bin(const rsdev::ShootDesc& d, const uint2* list, const unsigned int* count,
                               unsigned int cap, const float4* ff, int grid, cudaStream_t s) {
  if (cap == 0) return cudaSuccess;
  recheck_bin_kernel<<<grid, 128, 0, s>>>(d, list, count, cap, ff);
  return cudaGetLastError();
}

}  // namespace rsint
