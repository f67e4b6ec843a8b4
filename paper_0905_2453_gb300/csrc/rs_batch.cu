// Persistent batched shoot kernel: many independent lens fields in one launch.
//
// Work items are (field, ray tile) pairs ordered on the host by decreasing cost
// (longest-processing-time first).  Resident CTAs pull the next item from a
// global counter; each item runs the same per-ray arithmetic as the plain
// kernel, so a field's counts are bitwise those of its own rs_shoot.
#include "rs_internal.h"

namespace {

using namespace rsdev;

// MINB resident CTAs per SM as the occupancy floor, as for the plain kernel, except three: the
// launch shapes compiled for three CTAs per SM (168 registers) run here as their two-CTA twins.
// Inside the item loop the 168-register build of the tile body ran 1.6-3 % slower than the plain
// kernel's (one-field batches of 1e3-1e5 lenses), whatever held the descriptor (shared memory,
// kernel parameter, constant bank, global) and with the tile body out of line; at two CTAs per SM
// (up to 255 registers) the batch kernel matches the plain one.  The four-CTA shape (4 rays per
// thread, 128 registers) is for small fields, whose batches it speeds up by a third.  Counts do not
// depend on the shape.
template <int MINB>
constexpr int batch_minb() {
  return MINB == 3 ? 2 : MINB;
}
template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    batch_kernel(const ShootDesc* __restrict__ descs, const int2* __restrict__ items, int n_items, int* counter) {
  extern __shared__ __align__(128) unsigned char rs_smem[];
  auto& ss = *reinterpret_cast<ShootSmem<WARPS, RPT, TILE>*>(rs_smem);
  __shared__ int s_item;
  // the current item's field descriptor, staged in shared memory once per item so that the tile
  // code reads it as cheaply as the plain kernel reads its kernel-parameter descriptor
  __shared__ __align__(16) ShootDesc s_desc;
  static_assert(sizeof(ShootDesc) % 4 == 0, "descriptor copied as 32-bit words");
  PipeState ps;
  pipe_init(ss.lens.bar, ps);
  int cur_field = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const int2 w = items[it];
    if (w.x != cur_field) {  // CTA-uniform
      const uint32_t* src = reinterpret_cast<const uint32_t*>(descs + w.x);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_desc);
      for (int k = threadIdx.x; k < (int)(sizeof(ShootDesc) / 4); k += WARPS * 32) dst[k] = src[k];
      cur_field = w.x;
    }
    __syncthreads();  // s_desc ready; every thread has read s_item
    const bool ok = shoot_tile<WARPS, RPT, TILE, MASS>(s_desc, (int64_t)w.y, ss, ps);
    if (!ok) break;
  }
}

template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
cudaError_t launch_batch_m(const ShootDesc* descs, const int2* items, int n_items, int* counter, int grid,
                           cudaStream_t s) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<batch_kernel<WARPS, RPT, TILE, MASS, MINB>>(smem);
  if (e != cudaSuccess) return e;
  batch_kernel<WARPS, RPT, TILE, MASS, MINB><<<grid, WARPS * 32, smem, s>>>(descs, items, n_items, counter);
  return cudaGetLastError();
}

template <int WARPS, int RPT, int TILE, int MINB>
cudaError_t launch_batch_t(bool mass, const ShootDesc* descs, const int2* items, int n_items, int* counter, int grid,
                           cudaStream_t s) {
  return mass ? launch_batch_m<WARPS, RPT, TILE, true, MINB>(descs, items, n_items, counter, grid, s)
              : launch_batch_m<WARPS, RPT, TILE, false, MINB>(descs, items, n_items, counter, grid, s);
}

template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
cudaError_t occ_m(int* blocks) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<batch_kernel<WARPS, RPT, TILE, MASS, MINB>>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<WARPS, RPT, TILE, MASS, MINB>,
                                                       WARPS * 32, smem);
}

template <int WARPS, int RPT, int TILE, int MINB>
cudaError_t occ_t(bool mass, int* blocks) {
  return mass ? occ_m<WARPS, RPT, TILE, true, MINB>(blocks) : occ_m<WARPS, RPT, TILE, false, MINB>(blocks);
}

}  // namespace

namespace rsint {

cudaError_t launch_batch(int cfg, bool mass, const rsdev::ShootDesc* descs, const int2* items, int n_items,
                         int* counter, int grid, cudaStream_t s) {
  switch (cfg) {
#define RS_CASE(i, w, r, t, m) \
  case i:                       \
    return launch_batch_t<w, r, t, batch_minb<m>()>(mass, descs, items, n_items, counter, grid, s);
    RS_LAUNCH_SHAPES(RS_CASE)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_blocks_per_sm(int cfg, bool mass, int* blocks) {
  switch (cfg) {
#define RS_CASE(i, w, r, t, m) \
  case i:                       \
    return occ_t<w, r, t, batch_minb<m>()>(mass, blocks);
    RS_LAUNCH_SHAPES(RS_CASE)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsint
