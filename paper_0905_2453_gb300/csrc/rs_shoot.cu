// Plain (one field per launch) shoot kernel and the listed-ray trace kernel.
#include "rs_internal.h"

namespace {

using namespace rsdev;

// MINB resident CTAs per SM as the occupancy floor: two let the compiler keep a small CTA's eight rays
// per thread, their two-float accumulators and a deep instruction window in up to 255 registers;
// three (168 registers) hide more latency with twelve warps per SM; eight-warp CTAs take one.
template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) shoot_kernel(const ShootDesc d) {
  extern __shared__ __align__(128) unsigned char rs_smem[];
  auto& ss = *reinterpret_cast<ShootSmem<WARPS, RPT, TILE>*>(rs_smem);
  PipeState ps;
  pipe_init(ss.lens.bar, ps);
  (void)shoot_tile<WARPS, RPT, TILE, MASS>(d, (int64_t)blockIdx.x, ss, ps);
}

template <int BLOCK, int RPT, int TILE, bool MASS>
__global__ void __launch_bounds__(BLOCK)
    trace_kernel(const FieldDev f, double or0, double or1, double sp0, double sp1, const int64_t* __restrict__ ij,
                 int64_t k, double* __restrict__ y, double* __restrict__ alpha, double* __restrict__ err) {
  __shared__ LensSmem<TILE> sm;
  PipeState ps;
  pipe_init(sm.bar, ps);
  const int64_t base = (int64_t)blockIdx.x * (BLOCK * RPT);
  float x1[RPT], x2[RPT];
  bool valid[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int64_t r = base + (int64_t)q * BLOCK + threadIdx.x;
    valid[q] = r < k;
    if (!valid[q]) r = k - 1;
    x1[q] = ray_coord(ij[2 * r], sp0, or0);
    x2[q] = ray_coord(ij[2 * r + 1], sp1, or1);
  }
  double a1[RPT], a2[RPT];
  float sig[RPT];
  if (!deflect<RPT, TILE, MASS, false, 1>(f, x1, x2, a1, a2, sig, sm, ps)) return;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    if (!valid[q]) continue;
    const int64_t r = base + (int64_t)q * BLOCK + threadIdx.x;
    const double y1 = __dsub_rn(__dmul_rn(f.lam1, (double)x1[q]), a1[q]);
    const double y2 = __dsub_rn(__dmul_rn(f.lam2, (double)x2[q]), a2[q]);
    y[2 * r] = y1;
    y[2 * r + 1] = y2;
    if (alpha != nullptr) {
      alpha[2 * r] = a1[q];
      alpha[2 * r + 1] = a2[q];
    }
    if (err != nullptr) {
      // the ray's largest-term bound over every lens: the value the shoot kernels reach through
      // their near-lens search
      const float tn = near_term_all<MASS>(f, x1[q], x2[q]);
      const double b = (double)band_halfwidth(sig[q], tn, f.lamabs, x1[q], x2[q]);
      err[2 * r] = b;
      err[2 * r + 1] = b;
    }
  }
}

template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
cudaError_t launch_shoot_m(const ShootDesc& d, int64_t grid, cudaStream_t s) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<shoot_kernel<WARPS, RPT, TILE, MASS, MINB>>(smem);
  if (e != cudaSuccess) return e;
  shoot_kernel<WARPS, RPT, TILE, MASS, MINB><<<(unsigned)grid, WARPS * 32, smem, s>>>(d);
  return cudaGetLastError();
}

template <int WARPS, int RPT, int TILE, int MINB>
cudaError_t launch_shoot_t(const ShootDesc& d, cudaStream_t s) {
  const int64_t grid = shoot_tiles<WARPS, RPT>(d.n_rows, d.n0);
  if (grid <= 0) return cudaSuccess;
  if (grid >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  return d.f.has_mass ? launch_shoot_m<WARPS, RPT, TILE, true, MINB>(d, grid, s)
                      : launch_shoot_m<WARPS, RPT, TILE, false, MINB>(d, grid, s);
}

template <int WARPS, int RPT, int TILE, bool MASS, int MINB>
cudaError_t occupancy_m(int* blocks) {
  constexpr size_t smem = sizeof(ShootSmem<WARPS, RPT, TILE>);
  cudaError_t e = rsint::smem_opt_in<shoot_kernel<WARPS, RPT, TILE, MASS, MINB>>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, shoot_kernel<WARPS, RPT, TILE, MASS, MINB>,
                                                       WARPS * 32, smem);
}

template <int WARPS, int RPT, int TILE, int MINB>
cudaError_t occupancy_t(bool mass, int* blocks) {
  return mass ? occupancy_m<WARPS, RPT, TILE, true, MINB>(blocks) : occupancy_m<WARPS, RPT, TILE, false, MINB>(blocks);
}

}  // namespace

namespace rsint {

cudaError_t shoot_blocks_per_sm(int cfg, bool mass, int* blocks) {
  switch (cfg) {
#define RS_CASE(i, w, r, t, m) \
  case i:                       \
    return occupancy_t<w, r, t, m>(mass, blocks);
    RS_LAUNCH_SHAPES(RS_CASE)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_shoot(int cfg, const rsdev::ShootDesc& d, cudaStream_t s) {
  switch (cfg) {
#define RS_CASE(i, w, r, t, m) \
  case i:                       \
    return launch_shoot_t<w, r, t, m>(d, s);
    RS_LAUNCH_SHAPES(RS_CASE)
#undef RS_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_trace(const rsdev::FieldDev& f, double or0, double or1, double sp0, double sp1,
                         const int64_t* ij, int64_t k, double* y, double* alpha, double* err, cudaStream_t s) {
  constexpr int B = 128, R = 4;
  if (k <= 0) return cudaSuccess;
  const int64_t grid = (k + B * R - 1) / (B * R);
  if (f.has_mass)
    trace_kernel<B, R, kTile, true><<<(unsigned)grid, B, 0, s>>>(f, or0, or1, sp0, sp1, ij, k, y, alpha, err);
  else
    trace_kernel<B, R, kTile, false><<<(unsigned)grid, B, 0, s>>>(f, or0, or1, sp0, sp1, ij, k, y, alpha, err);
  return cudaGetLastError();
}

}  // namespace rsint
