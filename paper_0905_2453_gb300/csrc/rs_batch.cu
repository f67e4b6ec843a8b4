// Persistent batched shoot kernel: many independent lens fields in one launch.
//
// Work items are (field, ray tile) pairs ordered on the host by decreasing cost
// (longest-processing-time first).  Resident CTAs pull the next item from a
// global counter; each item runs the same per-ray arithmetic as the plain
// kernel, so a field's counts are bitwise those of its own rs_shoot.
#include "rs_internal.h"

namespace {

using namespace rsdev;

// Two CTAs per SM as the occupancy floor for small CTAs (more registers, as for the plain kernel);
// eight-warp CTAs keep the default allocation (a two-CTA floor would force spills there).
template <int WARPS, int RPT, int TILE, bool MASS>
__global__ void __launch_bounds__(WARPS * 32, WARPS <= 4 ? 2 : 1)
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

template <int WARPS, int RPT, int TILE, bool MASS>
cudaError_t launch_batch_m(const ShootDesc* descs, const int2* items, int n_items, int* counter, int grid,
                           cudaStream_t s) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<batch_kernel<WARPS, RPT, TILE, MASS>>(smem);
  if (e != cudaSuccess) return e;
  batch_kernel<WARPS, RPT, TILE, MASS><<<grid, WARPS * 32, smem, s>>>(descs, items, n_items, counter);
  return cudaGetLastError();
}

template <int WARPS, int RPT, int TILE>
cudaError_t launch_batch_t(bool mass, const ShootDesc* descs, const int2* items, int n_items, int* counter, int grid,
                           cudaStream_t s) {
  return mass ? launch_batch_m<WARPS, RPT, TILE, true>(descs, items, n_items, counter, grid, s)
              : launch_batch_m<WARPS, RPT, TILE, false>(descs, items, n_items, counter, grid, s);
}

template <int WARPS, int RPT, int TILE, bool MASS>
cudaError_t occ_m(int* blocks) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<batch_kernel<WARPS, RPT, TILE, MASS>>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_kernel<WARPS, RPT, TILE, MASS>, WARPS * 32,
                                                       smem);
}

template <int WARPS, int RPT, int TILE>
cudaError_t occ_t(bool mass, int* blocks) {
  return mass ? occ_m<WARPS, RPT, TILE, true>(blocks) : occ_m<WARPS, RPT, TILE, false>(blocks);
}

}  // namespace

namespace rsint {

cudaError_t launch_batch(int cfg, bool mass, const rsdev::ShootDesc* descs, const int2* items, int n_items,
                         int* counter, int grid, cudaStream_t s) {
  switch (cfg) {
    case 0: return launch_batch_t<2, 8, 256>(mass, descs, items, n_items, counter, grid, s);
    case 1: return launch_batch_t<4, 4, 256>(mass, descs, items, n_items, counter, grid, s);
    case 2: return launch_batch_t<4, 8, 256>(mass, descs, items, n_items, counter, grid, s);
    case 3: return launch_batch_t<8, 4, 256>(mass, descs, items, n_items, counter, grid, s);
    case 4: return launch_batch_t<8, 8, 256>(mass, descs, items, n_items, counter, grid, s);
    case 5: return launch_batch_t<8, 6, 256>(mass, descs, items, n_items, counter, grid, s);
    case 6: return launch_batch_t<2, 8, 512>(mass, descs, items, n_items, counter, grid, s);
    case 7: return launch_batch_t<4, 4, 512>(mass, descs, items, n_items, counter, grid, s);
    case 8: return launch_batch_t<4, 8, 512>(mass, descs, items, n_items, counter, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_blocks_per_sm(int cfg, bool mass, int* blocks) {
  switch (cfg) {
    case 0: return occ_t<2, 8, 256>(mass, blocks);
    case 1: return occ_t<4, 4, 256>(mass, blocks);
    case 2: return occ_t<4, 8, 256>(mass, blocks);
    case 3: return occ_t<8, 4, 256>(mass, blocks);
    case 4: return occ_t<8, 8, 256>(mass, blocks);
    case 5: return occ_t<8, 6, 256>(mass, blocks);
    case 6: return occ_t<2, 8, 512>(mass, blocks);
    case 7: return occ_t<4, 4, 512>(mass, blocks);
    case 8: return occ_t<4, 8, 512>(mass, blocks);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsint
