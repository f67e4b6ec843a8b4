// Internal host-side interface between the C-ABI layer (rs_api.cu) and the kernel
// translation units (rs_shoot.cu, rs_batch.cu).  Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_device.cuh"

namespace rsint {

// Lenses per shared-memory stage of the kernels without a tile choice (listed rays, culled cells,
// staged partitions); a multiple of rsdev::kGroup.
constexpr int kTile = 256;

// Launch shapes compiled into the library; the per-ray arithmetic is identical for all (the lens
// tile is a multiple of the 256-lens summation period, so the group and renormalisation schedule
// does not depend on it).  A CTA of block / 32 warps covers block / 32 grid rows by 32 * rpt columns,
// stages tile lenses per step, and is compiled for at least min_ctas resident CTAs per SM (the
// register budget per thread follows: 2 -> up to 255 registers, 3 -> 168 for 128-thread CTAs).
// X(index, warps, rays per thread, lens tile, min_ctas)
#define RS_LAUNCH_SHAPES(X)                                                                           \
  X(0, 2, 8, 256, 2) X(1, 4, 4, 256, 2) X(2, 4, 8, 256, 2) X(3, 8, 4, 256, 1) X(4, 8, 8, 256, 1)   \
  X(5, 8, 6, 256, 1) X(6, 2, 8, 512, 2) X(7, 4, 4, 512, 2) X(8, 4, 8, 512, 2) X(9, 4, 8, 256, 3)   \
  X(10, 4, 8, 512, 3) X(11, 4, 4, 256, 4)

struct KernelCfg {
  int block;     // threads per CTA (a multiple of 32)
  int rpt;       // rays per thread (even: packed pairs)
  int tile;      // lenses per shared-memory stage (256 or 512)
  int min_ctas;  // resident CTAs per SM the kernel is compiled for
};
#define RS_CFG_ENTRY(i, w, r, t, m) {32 * (w), r, t, m},
constexpr KernelCfg kCfgs[] = {RS_LAUNCH_SHAPES(RS_CFG_ENTRY)};
#undef RS_CFG_ENTRY
constexpr int kNumCfg = (int)(sizeof(kCfgs) / sizeof(kCfgs[0]));
constexpr int kDefaultCfg = 8;  // 128 threads x 8 rays x 512-lens tiles, two CTAs per SM

// Dynamic shared memory beyond 48 KiB per CTA needs a one-time opt-in per kernel and device.
template <auto Kernel>
cudaError_t smem_opt_in(size_t bytes) {
  if (bytes <= ((size_t)48 << 10)) return cudaSuccess;
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

inline int find_cfg(int block, int rpt, int tile, int min_ctas) {
  for (int i = 0; i < kNumCfg; ++i)
    if (kCfgs[i].block == block && kCfgs[i].rpt == rpt && kCfgs[i].tile == tile && kCfgs[i].min_ctas == min_ctas)
      return i;
  return -1;
}

// The shape a batch runs for launch shape cfg: the batch kernel is not built for three resident CTAs
// per SM (rs_batch.cu), so a three-CTA shape runs as its two-CTA twin, in the twin's group.
inline int batch_cfg(int cfg) {
  if (kCfgs[cfg].min_ctas != 3) return cfg;
  const int twin = find_cfg(kCfgs[cfg].block, kCfgs[cfg].rpt, kCfgs[cfg].tile, 2);
  return twin >= 0 ? twin : cfg;
}

// Plain launch: one CTA per ray tile of block * rpt rays.
cudaError_t launch_shoot(int cfg, const rsdev::ShootDesc& d, cudaStream_t s);
// Resident CTAs per SM of the plain shoot kernel of launch shape cfg.
cudaError_t shoot_blocks_per_sm(int cfg, bool mass, int* blocks);

// Listed rays -> source positions (and deflections, and band half-widths), float32 path.
cudaError_t launch_trace(const rsdev::FieldDev& f, double or0, double or1, double sp0, double sp1,
                         const int64_t* ij, int64_t k, double* y, double* alpha, double* err, cudaStream_t s);

// Listed rays -> source positions in float-float (the certified re-evaluation).
cudaError_t launch_trace_ff(const rsdev::FieldDev& f, double or0, double or1, double sp0, double sp1,
                            const int64_t* ij, int64_t k, double* y, double* alpha, cudaStream_t s);

// Re-evaluate and bin the listed rays (single: one field, descriptor by value; else descs[field]).
cudaError_t launch_recheck(const rsdev::ShootDesc* single, const rsdev::ShootDesc* descs, const uint2* list,
                           const unsigned int* count, unsigned int cap, int grid, cudaStream_t s);

// Capacity of the re-evaluation list for a call of n_rays rays.
inline unsigned int recheck_capacity(int64_t n_rays) {
  int64_t c = n_rays / 32;
  if (c < 4096) c = n_rays < 4096 ? n_rays : 4096;
  if (c > ((int64_t)1 << 24)) c = (int64_t)1 << 24;
  return (unsigned int)c;
}

// Persistent batched launch over LPT-ordered (field, ray tile) items.
// mass: the items all belong to fields with (true) or without (false) per-lens masses.
cudaError_t launch_batch(int cfg, bool mass, const rsdev::ShootDesc* descs, const int2* items, int n_items,
                         int* counter, int grid, cudaStream_t s);
cudaError_t batch_blocks_per_sm(int cfg, bool mass, int* blocks);

// Culled shooting (rs_cull.cu): cells of 16 x 16 rays, bounded first in groups of 4 x 4 cells.
// cull_cells returns the number of 16 x 16 cells of a call (and the cells per row), cull_coarse_cells
// the number of 64 x 64 cells; launch_cull appends the 64 x 64 cells that may reach the window to
// `coarse` (count *n_coarse) and then the 16 x 16 cells of those that may to `list` (count *n_kept,
// rays in *n_shot if not null), counting the rays of all others out of window; launch_shoot_cells
// shoots the listed cells (grid: persistent CTAs of 128 threads).  Counters start at zero.
int64_t cull_cells(int64_t n_rows, int64_t n0, int64_t* n_cx);
int64_t cull_coarse_cells(int64_t n_rows, int64_t n0);
cudaError_t launch_cull(const rsdev::ShootDesc& d, double hi0, double hi1, unsigned* coarse, unsigned* n_coarse,
                        unsigned* list, unsigned* n_kept, unsigned long long* n_shot, cudaStream_t s);
cudaError_t launch_shoot_cells(const rsdev::ShootDesc& d, int64_t n_cx, const unsigned* list, const unsigned* n_kept,
                               int grid, cudaStream_t s);

// Lens-partitioned shooting (rs_staged.cu), default launch shape (4 warps x 8 rays): the per-ray
// accumulator state of a call of n_rows x n0 rays takes staged_state_bytes; launch_staged adds the
// partition d.f to it (first: start from zero; last: map and bin instead of storing).  The listed
// rays of certified binning are re-evaluated partition by partition into ff (16 bytes per entry)
// and binned by launch_recheck_bin.
int64_t staged_tiles(int64_t n_rows, int64_t n0);
size_t staged_state_bytes(int64_t n_rows, int64_t n0);
cudaError_t launch_staged(const rsdev::ShootDesc& d, uint64_t* state, bool first, bool last, cudaStream_t s);
cudaError_t launch_recheck_part(const rsdev::ShootDesc& d, const uint2* list, const unsigned int* count,
                                unsigned int cap, float4* ff, bool first, int grid, cudaStream_t s);
cudaError_t launch_recheck_bin(const rsdev::ShootDesc& d, const uint2* list, const unsigned int* count,
                               unsigned int cap, const float4* ff, int grid, cudaStream_t s);

// Light curves (rs_lightcurve.cu): one descriptor per track with samples, in output order.
struct LcTrack {
  const float* mu;          // map, float[np1][np0]
  int np0, np1;
  double lo0, lo1;          // window lower edges
  double pix0, pix1;        // pixel sizes (hi - lo) / npix
  double y00, y01;          // first sample
  double st0, st1;          // sample step
  double t00, t01;          // first sample in pixel-index units: (y0 - lo) / pix - 0.5
  double d0, d1;            // step in pixel-index units: step / pix
  double rp0, rp1;          // support radius in pixels per axis (R / pix)
  float a0, a1;             // exponent per squared pixel offset (Gaussian: log2(e) pix^2 / (2 s^2); disc: pix^2 / s^2)
  float inv_a0;             // 1 / a0
  float band;               // guard band of the float32 exponent around the cut
  int64_t n;                // samples (> 0)
  int64_t out_off;          // first output position
};

// profile: 0 Gaussian, 1 disc.  cut2: the float64 squared support radius; ecut: the cut in exponent units.
cudaError_t launch_light_curves(int profile, const LcTrack* tracks, int n_tracks, int64_t n_samples, double cut2,
                                float ecut, double* mu_out, double* dm_out, int grid, cudaStream_t s);

}  // namespace rsint
