// Culled shooting (the interactive zoom of Section 4: a sub-window of the source plane re-shot at
// higher resolution): rays are grouped in cells of 16 x 16; a cell is skipped when a rigorous bound
// shows that none of its rays can land in the window, and the others are shot with the same per-ray
// arithmetic as rs_shoot, so the counts and the out-of-window count equal those of rs_shoot.
//
// Bound for a cell with ray box centre c and circumradius rho (every ray x of the cell has
// |x - c| <= rho), lenses at distance d_i = |c - x_i| > rho:
//   |alpha(x) - alpha(c)| <= sum_i m_i |x - c| / (|x - x_i| |c - x_i|) <= rho sum_i m_i / (d_i (d_i - rho)) = B
// (from |a/|a|^2 - b/|b|^2| = |a - b| / (|a| |b|)), and sum_i m_i / |x - x_i| <= sum_i m_i / (d_i - rho) = S,
// which bounds the float32 error band of every ray of the cell (a small multiple of 2^-24 S).  So
// y_k(x) = lam_k x_k - alpha_k(x) lies within [min, max](lam_k x_k) - alpha_k(c) +- (B + margins); a cell
// whose box misses the window on some axis is skipped and its rays are counted out of window.  A
// cell with a lens within 1.02 rho of c has no finite bound and is always shot.  The bound is applied
// to cells of 64 x 64 rays first and then to the 16 x 16 cells of the kept ones.
#include "rs_internal.h"

namespace {

using namespace rsdev;

constexpr int kCell = 16;        // rays per cell side
constexpr int kCullBlock = 256;  // cells per CTA of the bound kernel

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void fold(float& hi, float& lo, float p) {
  const float t = __fadd_rn(hi, p);
  const float bp = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
  hi = t;
}

// One thread per cell: the bound sums over all lenses (tiles staged in shared memory), then the
// cell's source-plane box against the window.  Kept cells are appended to `out`; skipped cells add
// their rays to the out-of-window count.  Two levels: cells of 64 x 64 rays over the whole call
// (parent == nullptr), then the 16 cells of 16 x 16 rays of every kept 64 x 64 cell.
template <bool MASS>
__global__ void __launch_bounds__(kCullBlock)
    cull_kernel(const ShootDesc d, int cell_rays, int64_t n_cx, int64_t n_cells, const unsigned* __restrict__ parent,
                const unsigned* __restrict__ parent_count, int64_t n_px, double hi0, double hi1,
                unsigned* __restrict__ out, unsigned* __restrict__ out_count, unsigned long long* __restrict__ n_shot) {
  __shared__ float4 s_lens[kCullBlock];
  __shared__ float s_mass[kCullBlock];
  const int64_t n_cy = (d.n_rows + cell_rays - 1) / cell_rays;
  int64_t cx, cy;
  bool ok;
  if (parent != nullptr) {
    const int64_t pc = *parent_count;
    if ((int64_t)blockIdx.x * kCullBlock >= pc * 16) return;  // CTA-uniform: no parent cells left
    const int64_t t = (int64_t)blockIdx.x * kCullBlock + threadIdx.x;
    const int64_t slot = t >> 4;
    const int sub = (int)(t & 15);
    ok = slot < pc;
    const int64_t p = parent[ok ? slot : 0];
    const int64_t py = p / n_px, px = p - py * n_px;
    cx = px * 4 + (sub & 3);
    cy = py * 4 + (sub >> 2);
    ok = ok && cx < n_cx && cy < n_cy;
  } else {
    const int64_t c = (int64_t)blockIdx.x * kCullBlock + threadIdx.x;
    ok = c < n_cells;
    cy = c / n_cx;
    cx = c - cy * n_cx;
  }
  if (!ok) cx = cy = 0;
  const int64_t i0 = cx * cell_rays, i1 = min(i0 + cell_rays, d.n0) - 1;
  const int64_t r0 = cy * cell_rays, r1 = min(r0 + cell_rays, d.n_rows) - 1;
  const float xa1 = ray_coord(i0, d.sp0, d.or0), xb1 = ray_coord(i1, d.sp0, d.or0);
  const float xa2 = ray_coord(d.j_begin + r0, d.sp1, d.or1), xb2 = ray_coord(d.j_begin + r1, d.sp1, d.or1);
  const float c1 = 0.5f * (xa1 + xb1), c2 = 0.5f * (xa2 + xb2);
  const double h1 = fmax((double)c1 - (double)xa1, (double)xb1 - (double)c1);
  const double h2 = fmax((double)c2 - (double)xa2, (double)xb2 - (double)c2);
  const float rho = (float)(sqrt(h1 * h1 + h2 * h2) * (1.0 + 0x1p-20)) + 1e-30f;
  const float rho_near = 1.02f * rho;  // d <= 1.02 rho: no usable bound
  float a1h = 0.f, a1l = 0.f, a2h = 0.f, a2l = 0.f, bh = 0.f, bl = 0.f, sh = 0.f, sl = 0.f;
  bool near = false;
  const int n = d.f.n_lens;
  for (int t0 = 0; t0 < n; t0 += kCullBlock) {
    __syncthreads();
    const int l = t0 + threadIdx.x;
    if (l < n) {
      s_lens[threadIdx.x] = d.f.lens4[l];
      s_mass[threadIdx.x] = MASS ? d.f.mass2[l].x : 1.f;
    }
    __syncthreads();
    const int cnt = min(kCullBlock, n - t0);
    for (int g = 0; g < cnt; g += 32) {
      float pa1 = 0.f, pa2 = 0.f, pb = 0.f, ps = 0.f;
      const int ge = min(g + 32, cnt);
      for (int q = g; q < ge; ++q) {
        const float4 L = s_lens[q];
        const float m = s_mass[q];
        const float dx = c1 - L.x, dy = c2 - L.z;
        const float d2 = fmaf(dx, dx, dy * dy);
        const float rs = rsqrt_approx(d2);
        const float dist = d2 * rs;
        near |= !(dist > rho_near);  // NaN (a lens on the centre) counts as near
        const float mi = m * rs * rs;
        pa1 = fmaf(mi, dx, pa1);
        pa2 = fmaf(mi, dy, pa2);
        const float mg = m * rcp_approx(dist - rho);
        ps += mg;
        pb = fmaf(mg, rs, pb);
      }
      fold(a1h, a1l, pa1);
      fold(a2h, a2l, pa2);
      fold(bh, bl, pb);
      fold(sh, sl, ps);
    }
  }
  if (!ok) return;
  const int64_t rays = (i1 - i0 + 1) * (r1 - r0 + 1);
  bool keep = true;
  if (!near) {
    // terms carry a few 2^-22 relative (approximate reciprocal square root and reciprocal, the gap's
    // cancellation when d is near 1.02 rho: <= 2^-16), sums of 32 float terms ~2^-19 of their
    // absolute sum: inflate B and S by 2^-8
    const double S = ((double)sh + (double)sl) * (1.0 + 0x1p-8);
    const double B = (double)rho * ((double)bh + (double)bl) * (1.0 + 0x1p-8);
    const double A1 = (double)a1h + (double)a1l, A2 = (double)a2h + (double)a2l;
    // alpha(c) error <= ~2^-18 S; the float32 band of a ray <= ~59 u S(x) <= 2^-18 S; float64 roundings
    const double x1m = fmax(fabs((double)xa1), fabs((double)xb1)), x2m = fmax(fabs((double)xa2), fabs((double)xb2));
    const double M = B + 0x1p-11 * S +
                     0x1p-40 * (fabs(d.f.lam1) * x1m + fabs(d.f.lam2) * x2m + fabs(A1) + fabs(A2) + B + 1.0 +
                                fabs(d.lo0) + fabs(d.lo1) + fabs(hi0) + fabs(hi1));
    const double p1 = d.f.lam1 * (double)xa1, q1 = d.f.lam1 * (double)xb1;
    const double p2 = d.f.lam2 * (double)xa2, q2 = d.f.lam2 * (double)xb2;
    const double y1min = fmin(p1, q1) - A1 - M, y1max = fmax(p1, q1) - A1 + M;
    const double y2min = fmin(p2, q2) - A2 - M, y2max = fmax(p2, q2) - A2 + M;
    const bool finite = isfinite(M) && isfinite(A1) && isfinite(A2);
    keep = !finite || !(y1max < d.lo0 || y1min > hi0 || y2max < d.lo1 || y2min > hi1);
  }
  if (keep) {
    const unsigned slot = atomicAdd(out_count, 1u);
    out[slot] = (unsigned)(cy * n_cx + cx);
    if (n_shot) atomicAdd(n_shot, (unsigned long long)rays);
  } else if (d.oow) {
    atomicAdd(d.oow, (unsigned long long)rays);
  }
}

// Kept cells: a CTA of four warps shoots four cells per pass (one per warp); lane l holds row l / 2
// of its cell and columns 8 (l % 2) .. 8 (l % 2) + 7.  The per-ray arithmetic is rs_shoot's (per-ray
// squared distances instead of the shared row table give bitwise the same values).
template <bool MASS>
__global__ void __launch_bounds__(128, 2) shoot_cells_kernel(const ShootDesc d, int64_t n_cx,
                                                             const unsigned* __restrict__ list,
                                                             const unsigned* __restrict__ n_kept) {
  constexpr int RPT = 8;
  __shared__ LensSmem<rsint::kTile, 1> sm;
  __shared__ NearSmem<rsint::kTile, 4, 128, RPT> ns;  // one near-lens box per warp (its cell)
  PipeState ps;
  pipe_init(sm.bar, ps);
  const unsigned count = *n_kept;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (unsigned base = blockIdx.x * 4u; base < count; base += gridDim.x * 4u) {  // CTA-uniform
    const unsigned slot = base + (unsigned)warp;
    const bool cell_ok = slot < count;
    const int64_t cell = (int64_t)list[cell_ok ? slot : count - 1];
    const int64_t cy = cell / n_cx, cx = cell - cy * n_cx;
    const int64_t jrel = cy * kCell + (lane >> 1);
    const bool row_ok = cell_ok && jrel < d.n_rows;
    const int64_t j = d.j_begin + (jrel < d.n_rows ? jrel : d.n_rows - 1);
    const float x2r = ray_coord(j, d.sp1, d.or1);
    const int64_t i_base = cx * kCell + (lane & 1) * RPT;
    float x1[RPT], x2[RPT];
    bool valid[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      int64_t i = i_base + k;
      valid[k] = row_ok && i < d.n0;
      if (i >= d.n0) i = d.n0 - 1;
      x1[k] = ray_coord(i, d.sp0, d.or0);
      x2[k] = x2r;
    }
    if (lane == 0) {
      // the cell's ray box (coordinates grow with the grid index)
      const int64_t ia = cx * kCell, ib = min(ia + kCell, d.n0) - 1;
      const int64_t ja = cy * kCell, jb = min(ja + kCell, d.n_rows) - 1;
      near_set_box(ns, warp, ray_coord(ia, d.sp0, d.or0), ray_coord(ib, d.sp0, d.or0),
                   ray_coord(d.j_begin + ja, d.sp1, d.or1), ray_coord(d.j_begin + jb, d.sp1, d.or1));
    }
    __syncthreads();  // every box is set before the first lens tile is searched
    float a1h[RPT], a1l[RPT], a2h[RPT], a2l[RPT], sig[RPT], tn[RPT];
    if (!deflect_pairs<RPT, rsint::kTile, MASS, false, 1>(d.f, x1, x2, a1h, a1l, a2h, a2l, sig, tn, sm, ps, &ns))
      return;
    bin_rays<RPT, 1>(d, x1, x2, a1h, a1l, a2h, a2l, sig, tn, valid, jrel, i_base, lane);
  }
}

}  // namespace

namespace rsint {

int64_t cull_cells(int64_t n_rows, int64_t n0, int64_t* n_cx) {
  *n_cx = (n0 + kCell - 1) / kCell;
  return ((n_rows + kCell - 1) / kCell) * *n_cx;
}

int64_t cull_coarse_cells(int64_t n_rows, int64_t n0) {
  constexpr int64_t C = 4 * kCell;
  return ((n_rows + C - 1) / C) * ((n0 + C - 1) / C);
}

cudaError_t launch_cull(const rsdev::ShootDesc& d, double hi0, double hi1, unsigned* coarse, unsigned* n_coarse,
                        unsigned* list, unsigned* n_kept, unsigned long long* n_shot, cudaStream_t s) {
  constexpr int64_t C = 4 * kCell;
  const int64_t n_px = (d.n0 + C - 1) / C;
  const int64_t n_coarse_cells = cull_coarse_cells(d.n_rows, d.n0);
  if (n_coarse_cells <= 0) return cudaSuccess;
  const int64_t n_cx = (d.n0 + kCell - 1) / kCell;
  const int64_t g1 = (n_coarse_cells + kCullBlock - 1) / kCullBlock;
  const int64_t g2 = (n_coarse_cells * 16 + kCullBlock - 1) / kCullBlock;
  if (d.f.has_mass) {
    cull_kernel<true><<<(unsigned)g1, kCullBlock, 0, s>>>(d, (int)C, n_px, n_coarse_cells, nullptr, nullptr, 0, hi0,
                                                          hi1, coarse, n_coarse, nullptr);
    cull_kernel<true><<<(unsigned)g2, kCullBlock, 0, s>>>(d, kCell, n_cx, 0, coarse, n_coarse, n_px, hi0, hi1, list,
                                                          n_kept, n_shot);
  } else {
    cull_kernel<false><<<(unsigned)g1, kCullBlock, 0, s>>>(d, (int)C, n_px, n_coarse_cells, nullptr, nullptr, 0, hi0,
                                                           hi1, coarse, n_coarse, nullptr);
    cull_kernel<false><<<(unsigned)g2, kCullBlock, 0, s>>>(d, kCell, n_cx, 0, coarse, n_coarse, n_px, hi0, hi1, list,
                                                           n_kept, n_shot);
  }
  return cudaGetLastError();
}

cudaError_t launch_shoot_cells(const rsdev::ShootDesc& d, int64_t n_cx, const unsigned* list, const unsigned* n_kept,
                               int grid, cudaStream_t s) {
  if (d.f.has_mass)
    shoot_cells_kernel<true><<<grid, 128, 0, s>>>(d, n_cx, list, n_kept);
  else
    shoot_cells_kernel<false><<<grid, 128, 0, s>>>(d, n_cx, list, n_kept);
  return cudaGetLastError();
}

}  // namespace rsint
