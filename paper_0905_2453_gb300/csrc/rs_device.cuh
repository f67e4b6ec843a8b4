// Device side of the inverse ray-shooting path (sm_103a).
//
// What one CTA computes: a tile of BLOCK x RPT rays of a regular image-plane
// grid (one grid row per warp), deflected by all lenses of a field (Eq. 2, a
// direct sum; the paper's ray x lens decomposition of Eq. 5 with lens tiles
// staged through shared memory, Section 2.2), mapped to the source plane with
// the macro-model of Eq. 6 and binned into a uint32 count map (Eq. 4 counts).
//
// GB300 mapping
//   * Lens tiles of TILE lenses are copied global -> shared by the bulk-copy
//     (TMA) engine, double-buffered, completion tracked by an mbarrier.  Each
//     CTA fetches its own tiles; there is no multicast.
//   * Lenses are stored duplicated, {x1, x1, x2, x2} (and {m, m}), so one
//     shared-memory load yields the 64-bit operand pairs of the packed
//     f32x2 instructions: every packed op advances two rays against one lens.
//   * The rays of a warp share one grid row, so (x2 - x2_lens) and its square
//     come from a per-row table built in shared memory once per lens tile.
//   * Per lens and ray pair: sub.f32x2, fma.f32x2 (|d|^2), the reciprocal,
//     [mul.f32x2 by the mass], fma.f32x2 x2 -- the ten flops per interaction of
//     the paper's Appendix A.  For three of every four lens pairs (unit masses;
//     one of two with masses) one rcp.approx of the product of the two squared
//     distances serves both lenses (Montgomery's simultaneous inversion), which
//     balances the MUFU pipe (16 reciprocals/clk/SM) against the FMA pipe.
//   * Per ray, each group of kGroup = 64 consecutive lenses is summed from zero
//     in float32, then folded into a two-float (hi, lo) accumulator with an
//     error-free TwoSum, so the deflection keeps its low-order bits over 1e8
//     lenses.  alpha = hi + lo, Eq. 6 and the pixel coordinate are evaluated
//     in float-float once per ray (Section 4's remark on using extra precision
//     only where it is needed; float64 only for the ray coordinates and for
//     rays re-evaluated by certified binning).
//   * Binning: one global atomic add per in-window ray; out-of-window rays
//     are counted per warp with a ballot and one 64-bit atomic per warp.
//
// Every wait on an mbarrier is bounded (about one second of globaltimer); on
// timeout the CTA records RS_ETIMEOUT in the field's status word, waits
// (bounded) for its own copies still in flight and returns.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsdev {

constexpr int kGroup = 64;                 // lenses per float32 partial sum (fixed: part of the arithmetic)
constexpr int kRenorm = 256;               // (hi, lo) renormalised after every 256 lenses (fixed: arithmetic)
constexpr int kLensPad = 1024;             // device lens arrays are padded to a multiple of this
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // bounded mbarrier wait: 1 s
constexpr unsigned kStatusTimeout = 5u;    // == RS_ETIMEOUT (low byte of the status word)
constexpr unsigned kStatusListFull = 0x100u;  // a certified-binning list overflowed (bit 8)

// ----------------------------------------------------------------------------------------------
// Packed f32x2 arithmetic (sm_100+): a uint64_t holds {lo = ray A, hi = ray B}.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Exact-rounding add/sub without flush-to-zero, for the TwoSum.
__device__ __forceinline__ uint64_t f2_add_x(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub_x(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// |a| lane-wise (clears both sign bits).
__device__ __forceinline__ uint64_t f2_abs(uint64_t a) { return a & 0x7fffffff7fffffffull; }
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// (hi, lo) <- Fast2Sum(hi, lo): keeps |lo| <= ulp(hi)/2 so that the float32 sum of TwoSum residuals in
// lo does not itself lose accuracy over millions of groups (|hi| >= |lo| holds: lo is a sum of at most
// eight residuals, each <= ulp(hi)/2).
__device__ __forceinline__ void renormalise(uint64_t& hi, uint64_t& lo) {
  const uint64_t s = f2_add_x(hi, lo);
  lo = f2_sub_x(lo, f2_sub_x(s, hi));
  hi = s;
}

// Error-free transformation of hi + p into (s, e), s = fl(hi + p), s + e = hi + p exactly
// (Knuth's TwoSum), lane-wise on both rays; e is accumulated into lo.
__device__ __forceinline__ void twosum_accumulate(uint64_t& hi, uint64_t& lo, uint64_t p) {
  uint64_t s = f2_add_x(hi, p);
  uint64_t bp = f2_sub_x(s, hi);
  uint64_t ap = f2_sub_x(s, bp);
  uint64_t db = f2_sub_x(p, bp);
  uint64_t da = f2_sub_x(hi, ap);
  uint64_t e = f2_add_x(da, db);
  lo = f2_add_x(lo, e);
  hi = s;
}

// ----------------------------------------------------------------------------------------------
// Shared memory, mbarrier and bulk copy (TMA) helpers.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void lds_pair2(uint32_t addr, uint64_t& a, uint64_t& b) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
__device__ __forceinline__ uint64_t lds_pair(uint32_t addr) {
  uint64_t a;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(a) : "r"(addr));
  return a;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity to complete (limit in ns of globaltimer).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// ----------------------------------------------------------------------------------------------
// Descriptors.
// ----------------------------------------------------------------------------------------------
struct FieldDev {
  const float4* lens4;  // {x1, x1, x2, x2} per lens, padded to a multiple of kLensPad lenses
  const float2* mass2;  // {m, m} per lens (same padding), or nullptr for unit masses
  int32_t n_lens;
  int32_t has_mass;
  double lam1, lam2;    // (1 - kappa_c) - gamma, (1 - kappa_c) + gamma
  float lamabs;         // max(|lam1|, |lam2|), for the Eq. 6 rounding term of the error band
  float mcap;           // the largest mass / h: bounds every term of a lens farther than h from a ray (0: no lenses)
  unsigned int* status; // device status word (RS_OK / RS_ETIMEOUT)
};

struct ShootDesc {
  FieldDev f;
  double or0, or1, sp0, sp1;  // ray grid origin and spacing
  int64_t n0;                 // rays per grid row
  int64_t j_begin;            // first grid row of this call
  int64_t n_rows;             // grid rows in this call (rows x n0 < 2^32 rays)
  double lo0, lo1, sc0, sc1;  // window lower corner and npix / (hi - lo)
  float scf0, scf1;           // the scales as float (error-band arithmetic only)
  int32_t np0, np1;           // pixels per axis
  uint32_t* counts;           // [np1][np0]
  unsigned long long* oow;    // out-of-window counter or nullptr
  uint2* rc_list;             // certified binning: rays to re-evaluate {field_id, ray index}, or nullptr
  unsigned int* rc_count;     // entries requested so far (may exceed rc_cap)
  unsigned int rc_cap;        // capacity of rc_list
  int32_t field_id;           // index of this field in its batch (0 for a single-field call)
  // float-float splits (hi + lo) of lam1, lam2, lo0, lo1, sc0, sc1 for the float32 epilogue
  float lam1h, lam1l, lam2h, lam2l, lo0h, lo0l, lo1h, lo1l, sc0h, sc0l, sc1h, sc1l;
};

// Certified binning: a ray whose float32 source position lies within kSigmaSafety * sigma of a
// pixel edge (sigma: the per-ray error estimate below) is re-evaluated in float-float arithmetic
// before it is counted.
constexpr float kSigmaSafety = 10.0f;
// sigma = u sqrt(64 sum_g (P1_g^2 + P2_g^2)): the rounding of a 64-lens float32 group partial is a
// random walk of at most 64 steps of ~u |P_g|; u = 2^-24.
constexpr float kSigmaScale = 5.9604645e-08f * 8.0f * kSigmaSafety;
// Coherent errors: the rounding of d1 = x1 - x1_lens keeps the ray's x1 only to ulp(d1) for lenses
// much farther away than |x1| -- the same shift for every lens of a binade, i.e. a systematic
// displacement of the ray seen by the far field -- and a bias of the approximate reciprocal
// scales every term alike.  Both are bounded by a few u times sum_g (|P1_g| + |P2_g|), which
// upper-bounds |alpha| and tracks sum_i |t_i| for a far field of many lenses.
constexpr float kSystematicScale = 2.0f * 5.9604645e-08f;

constexpr int kMaxSeg = 256;  // grid columns of one CTA tile: 32 lanes x at most 8 rays per thread

// ----------------------------------------------------------------------------------------------
// Near-lens term of the error band.
//
// The band built from the group partials misses one kind of float32 error: where the terms of
// lenses near a ray cancel inside one 64-lens group, the partial is far smaller than those terms,
// whose own rounding (a few u of each) it does not show.  Every ray therefore also carries
//   T = max(mcap, max over lenses with r^2 <= h^2 of m_i / r_i),
// an upper bound on its largest single term (mcap = largest mass / h bounds the term of every
// lens farther than h), and its band grows by kNearScale T.  T depends only on the ray and the
// field (every kernel evaluates the same float32 expression, near_term, and a maximum does not
// depend on the order).  The shoot kernels find the lenses within h of a CTA's ray box while the
// lens tiles stream through shared memory, so only those few are evaluated per ray.
// ----------------------------------------------------------------------------------------------
constexpr float kNearH2 = 1.0f;          // h^2: h = 1, the Einstein radius of a unit mass
constexpr double kNearPad = 1.001;       // box widening: > h by a margin covering float32 rounding
constexpr float kNearScale = 0x1p-20f;   // 16 u

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// m / r of one lens for one ray when the lens lies within h (float32 r^2 <= h^2), else 0.  A ray on
// the lens gives +inf (its band is then infinite); a massless lens gives NaN, which fmaxf ignores.
__device__ __forceinline__ float near_term(float x1, float x2, float lx, float ly, float m) {
  const float d1 = __fsub_rn(x1, lx), d2 = __fsub_rn(x2, ly);
  const float r2 = __fmaf_rn(d1, d1, __fmul_rn(d2, d2));
  return r2 <= kNearH2 ? __fmul_rn(m, rsqrt_approx(r2)) : 0.f;
}

// No near-lens search (listed-ray kernels evaluate T over every lens themselves).
struct NoNear {
  static constexpr bool kOn = false;
  static constexpr int kGroups = 1;
};

// Near-lens search state of a CTA of BLOCK threads holding RPT rays each, whose rays form NG groups
// (NG = 1: one box around all rays of the CTA; NG = warps: one box per warp).  While a lens tile is
// being summed, each warp checks its share of the tile's lenses against the boxes and lists the hits
// (field lens indices) in the list of the tile's parity; the list is evaluated during the next tile,
// after the end-of-tile barrier that already separates the two, so the search adds no barrier and
// nothing to the serial part of a tile boundary.
template <int TILE, int NG, int BLOCK, int RPT>
struct __align__(16) NearSmem {
  static constexpr bool kOn = true;
  static constexpr int kGroups = NG;
  float box[NG][4];        // x1 lo, x1 hi, x2 lo, x2 hi of each group's rays, widened by h (rounded outwards)
  int n[2][NG];            // lenses listed per tile parity and group
  int idx[2][NG][TILE];    // their indices in the field
  float t[RPT * BLOCK];    // per ray: the largest near term so far (thread x's ray k at k * BLOCK + x)
};

// Box of the rays [x1a, x1b] x [x2a, x2b] widened by kNearPad: a lens outside it is farther than h
// from every ray inside, in float32 as well (its rounded d1 or d2 exceeds h).  Empties the group's lists.
template <class NS>
__device__ __forceinline__ void near_set_box(NS& ns, int g, float x1a, float x1b, float x2a, float x2b) {
  ns.box[g][0] = __double2float_rd(__dsub_rd((double)x1a, kNearPad));
  ns.box[g][1] = __double2float_ru(__dadd_ru((double)x1b, kNearPad));
  ns.box[g][2] = __double2float_rd(__dsub_rd((double)x2a, kNearPad));
  ns.box[g][3] = __double2float_ru(__dadd_ru((double)x2b, kNearPad));
  ns.n[0][g] = 0;
  ns.n[1][g] = 0;
}

// The calling warp's share of the current tile (cnt lenses at l4, field index of the first: base):
// lenses inside a group's box are appended to that group's list of parity par.  Whole warps call it.
template <int TILE, class NS>
__device__ __forceinline__ void near_gather(NS& ns, int par, const float4* l4, int cnt, int base, int nwarps) {
  constexpr int NG = NS::kGroups;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int share = (TILE + nwarps - 1) / nwarps;
  const int l0 = warp * share, l1 = min(l0 + share, cnt);
  for (int l = l0 + lane; l - lane < l1; l += 32) {  // warp-uniform trip count
    const bool ok = l < l1;
    const float4 L = l4[ok ? l : l0];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const bool in = ok && L.x >= ns.box[g][0] && L.x <= ns.box[g][1] && L.z >= ns.box[g][2] && L.z <= ns.box[g][3];
      const unsigned mask = __ballot_sync(0xffffffffu, in);
      if (mask != 0u) {
        const int leader = __ffs(mask) - 1;
        int slot = 0;
        if (lane == leader) slot = atomicAdd(&ns.n[par][g], __popc(mask));
        slot = __shfl_sync(0xffffffffu, slot, leader);
        if (in) ns.idx[par][g][slot + __popc(mask & ((1u << lane) - 1u))] = base + l;
      }
    }
  }
}

// Near terms of group g's lenses listed with parity par for the thread's rays (packed pairs X1, X2),
// folded into the thread's entries of ns.t; lens coordinates from the field's arrays.
template <int NP, bool MASS, class NS>
__device__ __forceinline__ void near_eval(NS& ns, int par, int g, const FieldDev& f, const uint64_t (&X1)[NP],
                                          const uint64_t (&X2)[NP], int nthreads) {
  const int n = ns.n[par][g];
  if (n == 0) return;
  float x1[2 * NP], x2[2 * NP], t[2 * NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    f2_unpack(X1[q], x1[2 * q], x1[2 * q + 1]);
    f2_unpack(X2[q], x2[2 * q], x2[2 * q + 1]);
  }
#pragma unroll
  for (int k = 0; k < 2 * NP; ++k) t[k] = ns.t[k * nthreads + threadIdx.x];
  for (int e = 0; e < n; ++e) {
    const int l = ns.idx[par][g][e];
    const float4 L = __ldg(f.lens4 + l);
    const float m = MASS ? __ldg(f.mass2 + l).x : 1.f;
#pragma unroll
    for (int k = 0; k < 2 * NP; ++k) t[k] = fmaxf(t[k], near_term(x1[k], x2[k], L.x, L.z, m));
  }
#pragma unroll
  for (int k = 0; k < 2 * NP; ++k) ns.t[k * nthreads + threadIdx.x] = t[k];
}

// T of one ray over every lens of a field (listed-ray kernels): the same value as the shoot's.
template <bool MASS>
__device__ __forceinline__ float near_term_all(const FieldDev& f, float x1, float x2) {
  float t = f.mcap;
  for (int l = 0; l < f.n_lens; ++l) {
    const float4 L = __ldg(f.lens4 + l);
    const float m = MASS ? __ldg(f.mass2 + l).x : 1.f;
    t = fmaxf(t, near_term(x1, x2, L.x, L.z, m));
  }
  return t;
}

template <int TILE, int ROWS = 1>
struct __align__(16) LensSmem {
  float4 lens4[2][TILE];     // double-buffered lens tiles {x1, x1, x2, x2}
  float2 mass2[2][TILE];     // {m, m}
  float4 rowtab[ROWS][TILE]; // per CTA row r and lens l of the current tile: {d2, d2, d2^2, d2^2}
  float x2row[ROWS];         // x2 of the CTA's rows
  float x1col[kMaxSeg];      // x1 of the CTA's columns (shoot_tile)
  uint64_t bar[2];
};

// Pipeline state carried across ray tiles by the persistent kernel (CTA-uniform).
struct PipeState {
  uint32_t parity[2];
};

__device__ __forceinline__ void pipe_init(uint64_t* bar, PipeState& ps) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  ps.parity[0] = 0;
  ps.parity[1] = 0;
  __syncthreads();
}

template <int TILE, bool MASS, int ROWS>
__device__ __forceinline__ void issue_lens_tile(const FieldDev& f, LensSmem<TILE, ROWS>& sm, int tile, int buf) {
  // called by one thread.  The tile's lenses rounded up to an even count (16-byte multiples for both
  // arrays): at most one lens past the field's last, which the padding of the device arrays (and of a
  // view's parent) always holds; lenses past the count are never read.
  const int cnt = min(TILE, f.n_lens - tile * TILE);
  const uint32_t n2 = (uint32_t)(cnt + (cnt & 1));
  const uint32_t b4 = n2 * (uint32_t)sizeof(float4);
  const uint32_t b2 = MASS ? n2 * (uint32_t)sizeof(float2) : 0u;
  fence_proxy_async_smem();
  mbar_expect_tx(&sm.bar[buf], b4 + b2);
  bulk_g2s(&sm.lens4[buf][0], f.lens4 + (size_t)tile * TILE, b4, &sm.bar[buf]);
  if (MASS) bulk_g2s(&sm.mass2[buf][0], f.mass2 + (size_t)tile * TILE, b2, &sm.bar[buf]);
}

// ----------------------------------------------------------------------------------------------
// Ray position (i, j) -> float, as the header defines it.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ float ray_coord(int64_t idx, double spacing, double origin) {
  return __double2float_rn(__fma_rn((double)idx, spacing, origin));
}

// ----------------------------------------------------------------------------------------------
// Lens-pair step.  Two consecutive lenses a, b against one ray pair (lanes A, B of each operand).
// d1 = x1 - x1_lens; r2 = d1^2 + d2^2 with d2^2 (S2) supplied; w = m / r2; P += w * (d1, d2).
//
// MONT: one reciprocal serves both lenses (Montgomery's simultaneous inversion):
//   inv = 1 / (r2a * r2b),  1/r2a = r2b * inv,  1/r2b = r2a * inv.
// Two MUFU operations per ray pair instead of four, for three extra packed multiplies on the
// FMA pipe.  With |coordinates| <= 1e9 the product stays below 6.4e37 (no overflow); it can
// only underflow when the ray is within ~3e-10 of one of the two lenses, a ray whose own
// deflection is then ~1e9 (out of any window), and only that ray is affected.
// ----------------------------------------------------------------------------------------------
template <bool MONT, bool MASS>
__device__ __forceinline__ void lens_pair_step(uint64_t X1, uint64_t Lxa, uint64_t Lxb, uint64_t D2a, uint64_t S2a,
                                               uint64_t D2b, uint64_t S2b, uint64_t Ma, uint64_t Mb, uint64_t& P1,
                                               uint64_t& P2) {
  const uint64_t d1a = f2_sub(X1, Lxa);
  const uint64_t d1b = f2_sub(X1, Lxb);
  const uint64_t r2a = f2_fma(d1a, d1a, S2a);
  const uint64_t r2b = f2_fma(d1b, d1b, S2b);
  uint64_t wa, wb;
  if (MONT) {
    const uint64_t pr = f2_mul(r2a, r2b);
    float p0, p1;
    f2_unpack(pr, p0, p1);
    const uint64_t inv = f2_pack(rcp_approx(p0), rcp_approx(p1));
    wa = f2_mul(r2b, inv);
    wb = f2_mul(r2a, inv);
  } else {
    float a0, a1, b0, b1;
    f2_unpack(r2a, a0, a1);
    f2_unpack(r2b, b0, b1);
    wa = f2_pack(rcp_approx(a0), rcp_approx(a1));
    wb = f2_pack(rcp_approx(b0), rcp_approx(b1));
  }
  if (MASS) {
    wa = f2_mul(wa, Ma);
    wb = f2_mul(wb, Mb);
  }
  P1 = f2_fma(wa, d1a, P1);
  P2 = f2_fma(wa, D2a, P2);
  P1 = f2_fma(wb, d1b, P1);
  P2 = f2_fma(wb, D2b, P2);
}

// A single lens (the odd last lens of a field), direct reciprocal.
template <bool MASS>
__device__ __forceinline__ void lens_single_step(uint64_t X1, uint64_t Lx, uint64_t D2, uint64_t S2, uint64_t M,
                                                 uint64_t& P1, uint64_t& P2) {
  const uint64_t d1 = f2_sub(X1, Lx);
  const uint64_t r2 = f2_fma(d1, d1, S2);
  float a0, a1;
  f2_unpack(r2, a0, a1);
  uint64_t w = f2_pack(rcp_approx(a0), rcp_approx(a1));
  if (MASS) w = f2_mul(w, M);
  P1 = f2_fma(w, d1, P1);
  P2 = f2_fma(w, D2, P2);
}

// Which lens pairs of a group use the shared reciprocal: pair index p within its group.
// Unit masses: three of every four pairs; per-lens masses (one more multiply per lens): every
// other pair.  These ratios balance the FMA and MUFU pipes; they are fixed, so every ray of a
// field always gets the same arithmetic.
template <bool MASS>
__device__ __forceinline__ constexpr bool mont_pair(int p) {
  return MASS ? ((p & 1) == 0) : ((p & 3) != 3);
}

// Loads lens l of the current shared-memory buffer: Lx = {x1, x1}, Ly = {x2, x2}, M = {m, m}.
template <bool MASS>
__device__ __forceinline__ void load_lens(uint32_t lbase, uint32_t mbase, int l, uint64_t& Lx, uint64_t& Ly,
                                          uint64_t& M) {
  lds_pair2(lbase + (uint32_t)l * 16u, Lx, Ly);
  M = MASS ? lds_pair(mbase + (uint32_t)l * 8u) : 0ull;
}

// One lens pair (lenses l, l + 1) against all ray pairs of the thread.
// ROW: all rays of the thread share x2 (one grid row); d2 and d2^2 of the row come from the
// shared-memory row table built once per lens tile (rt = that row's table).  Otherwise each ray
// pair forms them itself.  Either way every ray gets exactly the same operations.
template <int NP, bool MONT, bool MASS, bool ROW>
__device__ __forceinline__ void lens_pair_all(uint32_t lbase, uint32_t mbase, uint32_t rt, int l,
                                              const uint64_t (&X1)[NP], const uint64_t (&X2)[NP], uint64_t (&P1)[NP],
                                              uint64_t (&P2)[NP]) {
  uint64_t Lxa, Lya, Ma, Lxb, Lyb, Mb;
  if (ROW) {
    Lxa = lds_pair(lbase + (uint32_t)l * 16u);
    Lxb = lds_pair(lbase + (uint32_t)(l + 1) * 16u);
    Ma = MASS ? lds_pair(mbase + (uint32_t)l * 8u) : 0ull;
    Mb = MASS ? lds_pair(mbase + (uint32_t)(l + 1) * 8u) : 0ull;
    uint64_t D2a, S2a, D2b, S2b;
    lds_pair2(rt + (uint32_t)l * 16u, D2a, S2a);
    lds_pair2(rt + (uint32_t)(l + 1) * 16u, D2b, S2b);
#pragma unroll
    for (int q = 0; q < NP; ++q) lens_pair_step<MONT, MASS>(X1[q], Lxa, Lxb, D2a, S2a, D2b, S2b, Ma, Mb, P1[q], P2[q]);
  } else {
    load_lens<MASS>(lbase, mbase, l, Lxa, Lya, Ma);
    load_lens<MASS>(lbase, mbase, l + 1, Lxb, Lyb, Mb);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const uint64_t D2a = f2_sub(X2[q], Lya), D2b = f2_sub(X2[q], Lyb);
      const uint64_t S2a = f2_mul(D2a, D2a), S2b = f2_mul(D2b, D2b);
      lens_pair_step<MONT, MASS>(X1[q], Lxa, Lxb, D2a, S2a, D2b, S2b, Ma, Mb, P1[q], P2[q]);
    }
  }
}

// Row table for the current lens tile: entry (r, l) = {d2, d2, d2^2, d2^2} with d2 = x2(row r) - x2(lens l),
// the same float32 operations a thread would otherwise repeat for every lens.
// (Only the tile's cnt lenses: the last tile of a small field may hold far fewer than TILE.)
template <int TILE, int ROWS>
__device__ __forceinline__ void build_row_table(LensSmem<TILE, ROWS>& sm, int b, int cnt) {
  constexpr int BLOCK = ROWS * 32;
  for (int l = threadIdx.x; l < cnt; l += BLOCK) {
    const float y = sm.lens4[b][l].z;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const uint64_t D2 = f2_sub(f2_pack(sm.x2row[r], sm.x2row[r]), f2_pack(y, y));
      const uint64_t S2 = f2_mul(D2, D2);
      float d0, d1, s0, s1;
      f2_unpack(D2, d0, d1);
      f2_unpack(S2, s0, s1);
      sm.rowtab[r][l] = make_float4(d0, d1, s0, s1);
    }
  }
}

// ----------------------------------------------------------------------------------------------
// Deflection of RPT rays per thread by all lenses of the field (Eq. 2).
// x1/x2: ray coordinates (ROW: all rays of a warp share x2, recorded in sm.x2row[warp] by the
// caller).  alpha1/alpha2 (double) out.  Returns false if a bounded wait gave up (the CTA must
// then stop; the status word has been set).  The arithmetic per ray depends only on the ray and
// the field.
// ----------------------------------------------------------------------------------------------
// Per-ray accumulators of the deflection sum, packed two rays per 64-bit register: two-float
// (hi, lo) sums of alpha1 and alpha2, and the error-band sums of squared and absolute group partials.
template <int NP>
struct DeflectAcc {
  uint64_t H1[NP], L1[NP], H2[NP], L2[NP], SS[NP], AB[NP];
};

// Accumulate the field's lenses into acc (X1/X2: packed ray coordinates).  The arithmetic depends on
// a lens's index within the field only through the group (64) and renormalisation (256) schedule,
// so a field split into parts of multiples of 256 lenses, accumulated part after part, gives
// bitwise the sums of the whole field.  Returns false if a bounded wait gave up (the CTA must then
// stop; the status word has been set).
// With a near-lens search (NS::kOn), every tile's lenses inside the group boxes of ns are listed and
// their near terms folded into ns.t (the caller sets the boxes and the thread's ns.t entries).
template <int RPT, int TILE, bool MASS, bool ROW, int ROWS, class NS = NoNear>
__device__ __forceinline__ bool deflect_accumulate(const FieldDev& f, const uint64_t (&X1)[RPT / 2],
                                                   const uint64_t (&X2)[RPT / 2], DeflectAcc<RPT / 2>& acc,
                                                   LensSmem<TILE, ROWS>& sm, PipeState& ps, NS* ns = nullptr) {
  static_assert(TILE % kGroup == 0 && kGroup % 8 == 0, "lens tile must hold whole lens groups");
  static_assert(kRenorm % kGroup == 0, "renormalisation falls on group boundaries");
  constexpr int NP = RPT / 2;
  uint64_t (&H1)[NP] = acc.H1;
  uint64_t (&L1)[NP] = acc.L1;
  uint64_t (&H2)[NP] = acc.H2;
  uint64_t (&L2)[NP] = acc.L2;
  uint64_t (&SS)[NP] = acc.SS;
  uint64_t (&AB)[NP] = acc.AB;
  const int n = f.n_lens;
  const int ntiles = (n + TILE - 1) / TILE;
  const uint32_t rt = smem_u32(&sm.rowtab[ROW ? (threadIdx.x >> 5) : 0][0]);
  bool ok = true;
  if (threadIdx.x == 0) {
    if (ntiles > 0) issue_lens_tile<TILE, MASS>(f, sm, 0, 0);
    if (ntiles > 1) issue_lens_tile<TILE, MASS>(f, sm, 1, 1);
  }
  int t = 0;
  for (; t < ntiles; ++t) {
    const int b = t & 1;
    const bool got = mbar_wait_bounded(&sm.bar[b], ps.parity[b]);
    ps.parity[b] ^= 1u;
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    const int cnt = min(TILE, n - t * TILE);
    if (ROW) {
      build_row_table<TILE, ROWS>(sm, b, cnt);
      __syncthreads();
    }
    if constexpr (NS::kOn) {
      // the previous tile's list is complete (end-of-tile barrier); this tile's share goes to the other list
      if (t > 0) near_eval<NP, MASS>(*ns, (t - 1) & 1, NS::kGroups == 1 ? 0 : (int)(threadIdx.x >> 5), f, X1, X2,
                                     (int)blockDim.x);
      near_gather<TILE>(*ns, t & 1, &sm.lens4[b][0], cnt, t * TILE, (int)(blockDim.x >> 5));
    }
    const uint32_t lbase = smem_u32(&sm.lens4[b][0]);
    const uint32_t mbase = smem_u32(&sm.mass2[b][0]);
    int g = 0;
    for (; g + kGroup <= cnt; g += kGroup) {
      uint64_t P1[NP], P2[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) P1[q] = P2[q] = 0ull;
#pragma unroll
      for (int p4 = 0; p4 < kGroup / 8; ++p4) {  // blocks of four lens pairs: fixed reciprocal pattern
        const int l = g + p4 * 8;
        lens_pair_all<NP, mont_pair<MASS>(0), MASS, ROW>(lbase, mbase, rt, l + 0, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(1), MASS, ROW>(lbase, mbase, rt, l + 2, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(2), MASS, ROW>(lbase, mbase, rt, l + 4, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(3), MASS, ROW>(lbase, mbase, rt, l + 6, X1, X2, P1, P2);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        twosum_accumulate(H1[q], L1[q], P1[q]);
        twosum_accumulate(H2[q], L2[q], P2[q]);
        SS[q] = f2_fma(P1[q], P1[q], SS[q]);
        SS[q] = f2_fma(P2[q], P2[q], SS[q]);
        AB[q] = f2_add_x(AB[q], f2_add_x(f2_abs(P1[q]), f2_abs(P2[q])));
      }
      if ((t * TILE + g + kGroup) % kRenorm == 0) {  // CTA-uniform
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          renormalise(H1[q], L1[q]);
          renormalise(H2[q], L2[q]);
        }
      }
    }
    if (g < cnt) {  // last, partial group of the field: same pattern by pair index, odd lens direct
      uint64_t P1[NP], P2[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) P1[q] = P2[q] = 0ull;
      int p = 0;
      for (; g + 2 * p + 8 <= cnt; p += 4) {  // whole blocks of four pairs first (p = 0 mod 4 at each)
        lens_pair_all<NP, mont_pair<MASS>(0), MASS, ROW>(lbase, mbase, rt, g + 2 * p + 0, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(1), MASS, ROW>(lbase, mbase, rt, g + 2 * p + 2, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(2), MASS, ROW>(lbase, mbase, rt, g + 2 * p + 4, X1, X2, P1, P2);
        lens_pair_all<NP, mont_pair<MASS>(3), MASS, ROW>(lbase, mbase, rt, g + 2 * p + 6, X1, X2, P1, P2);
      }
      for (; g + 2 * p + 1 < cnt; ++p) {
        if (mont_pair<MASS>(p))
          lens_pair_all<NP, true, MASS, ROW>(lbase, mbase, rt, g + 2 * p, X1, X2, P1, P2);
        else
          lens_pair_all<NP, false, MASS, ROW>(lbase, mbase, rt, g + 2 * p, X1, X2, P1, P2);
      }
      if (g + 2 * p < cnt) {
        const int l = g + 2 * p;
        uint64_t Lx, Ly, M;
        load_lens<MASS>(lbase, mbase, l, Lx, Ly, M);
        if (ROW) {
          uint64_t D2, S2;
          lds_pair2(rt + (uint32_t)l * 16u, D2, S2);
#pragma unroll
          for (int q = 0; q < NP; ++q) lens_single_step<MASS>(X1[q], Lx, D2, S2, M, P1[q], P2[q]);
        } else {
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const uint64_t D2 = f2_sub(X2[q], Ly);
            lens_single_step<MASS>(X1[q], Lx, D2, f2_mul(D2, D2), M, P1[q], P2[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        twosum_accumulate(H1[q], L1[q], P1[q]);
        twosum_accumulate(H2[q], L2[q], P2[q]);
        SS[q] = f2_fma(P1[q], P1[q], SS[q]);
        SS[q] = f2_fma(P2[q], P2[q], SS[q]);
        AB[q] = f2_add_x(AB[q], f2_add_x(f2_abs(P1[q]), f2_abs(P2[q])));
      }
    }
    __syncthreads();  // every thread is done with buffer b, the row table and the previous tile's near list
    if (threadIdx.x == 0) {
      if constexpr (NS::kOn)
        for (int g = 0; g < NS::kGroups; ++g) ns->n[(t + 1) & 1][g] = 0;  // evaluated: free for tile t + 1
      if (t + 2 < ntiles) issue_lens_tile<TILE, MASS>(f, sm, t + 2, b);
    }
  }
  if constexpr (NS::kOn) {
    if (ok && ntiles > 0)  // the last tile's list (complete: end-of-tile barrier)
      near_eval<NP, MASS>(*ns, (ntiles - 1) & 1, NS::kGroups == 1 ? 0 : (int)(threadIdx.x >> 5), f, X1, X2,
                          (int)blockDim.x);
  }
  if (!ok) {
    // Record the timeout and drain this CTA's copies still in flight (bounded) before leaving:
    // tile t (its parity was already flipped above) and tile t + 1 if it was issued.
    if (threadIdx.x == 0) atomicOr(f.status, kStatusTimeout);
    (void)mbar_wait_bounded(&sm.bar[t & 1], ps.parity[t & 1] ^ 1u);
    if (t + 1 < ntiles) (void)mbar_wait_bounded(&sm.bar[(t + 1) & 1], ps.parity[(t + 1) & 1]);
    return false;
  }
  return true;
}

// alpha as float pairs (hi, lo: alpha = hi + lo exactly, |lo| <= ulp(hi) / 2) and the error-band
// estimate sig of each ray from its accumulators.
template <int RPT>
__device__ __forceinline__ void deflect_finish(const DeflectAcc<RPT / 2>& acc, float (&a1h)[RPT], float (&a1l)[RPT],
                                               float (&a2h)[RPT], float (&a2l)[RPT], float (&sig)[RPT]) {
  constexpr int NP = RPT / 2;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    f2_unpack(acc.H1[q], a1h[2 * q], a1h[2 * q + 1]);
    f2_unpack(acc.L1[q], a1l[2 * q], a1l[2 * q + 1]);
    f2_unpack(acc.H2[q], a2h[2 * q], a2h[2 * q + 1]);
    f2_unpack(acc.L2[q], a2l[2 * q], a2l[2 * q + 1]);
    float s, sB, b, bB;
    f2_unpack(acc.SS[q], s, sB);
    f2_unpack(acc.AB[q], b, bB);
    // |alpha| enters through the rounding of Eq. 6 (~1e-16 |alpha| in float64): 8e-15 (|hi1| + |hi2|)
    sig[2 * q] = kSigmaScale * sqrtf(s) + kSystematicScale * b + 8e-15f * (fabsf(a1h[2 * q]) + fabsf(a2h[2 * q]));
    sig[2 * q + 1] =
        kSigmaScale * sqrtf(sB) + kSystematicScale * bB + 8e-15f * (fabsf(a1h[2 * q + 1]) + fabsf(a2h[2 * q + 1]));
  }
}

template <int RPT>
__device__ __forceinline__ void pack_rays(const float (&x1)[RPT], const float (&x2)[RPT], uint64_t (&X1)[RPT / 2],
                                          uint64_t (&X2)[RPT / 2]) {
#pragma unroll
  for (int q = 0; q < RPT / 2; ++q) {
    X1[q] = f2_pack(x1[2 * q], x1[2 * q + 1]);
    X2[q] = f2_pack(x2[2 * q], x2[2 * q + 1]);
  }
}

// Deflection of the thread's rays and, with a near-lens search (the caller set the boxes), the
// largest-term bound T of every ray (tn); without one, tn = mcap (the caller adds the near terms).
template <int RPT, int TILE, bool MASS, bool ROW, int ROWS, class NS = NoNear>
__device__ __forceinline__ bool deflect_pairs(const FieldDev& f, const float (&x1)[RPT], const float (&x2)[RPT],
                                              float (&a1h)[RPT], float (&a1l)[RPT], float (&a2h)[RPT],
                                              float (&a2l)[RPT], float (&sig)[RPT], float (&tn)[RPT],
                                              LensSmem<TILE, ROWS>& sm, PipeState& ps, NS* ns = nullptr) {
  static_assert(RPT % 2 == 0, "rays per thread must be even (packed pairs)");
  constexpr int NP = RPT / 2;
  uint64_t X1[NP], X2[NP];
  pack_rays<RPT>(x1, x2, X1, X2);
  DeflectAcc<NP> acc;
#pragma unroll
  for (int q = 0; q < NP; ++q) acc.H1[q] = acc.L1[q] = acc.H2[q] = acc.L2[q] = acc.SS[q] = acc.AB[q] = 0ull;
  if constexpr (NS::kOn) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) ns->t[k * blockDim.x + threadIdx.x] = 0.f;
  }
  if (!deflect_accumulate<RPT, TILE, MASS, ROW, ROWS, NS>(f, X1, X2, acc, sm, ps, ns)) return false;
  deflect_finish<RPT>(acc, a1h, a1l, a2h, a2l, sig);
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    if constexpr (NS::kOn)
      tn[k] = fmaxf(ns->t[k * blockDim.x + threadIdx.x], f.mcap);
    else
      tn[k] = f.mcap;
  }
  return true;
}

// As deflect_pairs without a near-lens search, with alpha in float64 (hi + lo, exact).
template <int RPT, int TILE, bool MASS, bool ROW, int ROWS>
__device__ __forceinline__ bool deflect(const FieldDev& f, const float (&x1)[RPT], const float (&x2)[RPT],
                                        double (&a1)[RPT], double (&a2)[RPT], float (&sig)[RPT],
                                        LensSmem<TILE, ROWS>& sm, PipeState& ps) {
  float a1h[RPT], a1l[RPT], a2h[RPT], a2l[RPT], tn[RPT];
  if (!deflect_pairs<RPT, TILE, MASS, ROW, ROWS>(f, x1, x2, a1h, a1l, a2h, a2l, sig, tn, sm, ps)) return false;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    a1[k] = (double)a1h[k] + (double)a1l[k];
    a2[k] = (double)a2h[k] + (double)a2l[k];
  }
  return true;
}

// Half-width of the band around y within which the float32 path cannot decide the pixel: sig (the
// safety-scaled random-rounding estimate, the coherent term and the alpha part of a float64
// evaluation of Eq. 6), the near-lens term of the ray's largest-term bound tn, and the lam x part of
// the Eq. 6 rounding.  The shoot's float-float epilogue adds its own rounding bound on top (ff_pixel).
__device__ __forceinline__ float band_halfwidth(float sig, float tn, float lamabs, float x1, float x2) {
  return sig + kNearScale * tn + 4e-15f * lamabs * (fabsf(x1) + fabsf(x2));
}

// ----------------------------------------------------------------------------------------------
// One axis of Eq. 6 and of the pixel coordinate in float-float: y = lam x - alpha and
// u = (y - lo) * sc with lam, lo, sc given as float pairs (hi + lo) and alpha = ah + al.  Returns
// kUOk with p = floor(u) and f = u - p in [0, 1) (rounded to float); kUFar if |u| >= 2^22; kUNaN if
// u is not a number (a ray on a lens).  eu bounds the float-float rounding of u (2^-40 of the
// magnitudes involved; the arithmetic keeps ~2^-45).
// ----------------------------------------------------------------------------------------------
constexpr int kUOk = 0, kUFar = 1, kUNaN = 2;

__device__ __forceinline__ int ff_pixel(float x, float lh, float ll, float ah, float al, float loh, float lol,
                                        float sch, float scl, int& p, float& f, float& eu) {
  const float pr = __fmul_rn(lh, x);
  const float pe = __fmaf_rn(lh, x, -pr);                 // lh x = pr + pe exactly
  float s = __fadd_rn(pr, -ah);
  float bb = __fsub_rn(s, pr);
  float t = __fadd_rn(__fsub_rn(pr, __fsub_rn(s, bb)), __fsub_rn(-ah, bb));  // pr - ah = s + t exactly
  t = __fadd_rn(t, __fadd_rn(pe, __fmaf_rn(ll, x, -al)));   // y = s + t
  float v = __fadd_rn(s, -loh);
  bb = __fsub_rn(v, s);
  float w = __fadd_rn(__fsub_rn(s, __fsub_rn(v, bb)), __fsub_rn(-loh, bb));  // s - loh = v + w exactly
  w = __fadd_rn(w, __fsub_rn(t, lol));                    // y - lo = v + w
  const float uh = __fmul_rn(v, sch);
  const float ue = __fadd_rn(__fmaf_rn(v, sch, -uh), __fmaf_rn(w, sch, __fmul_rn(v, scl)));  // u = uh + ue
  eu = 0x1p-40f * ((fabsf(pr) + fabsf(ah) + fabsf(loh)) * sch + fabsf(uh) + 1.f);
  if (!(fabsf(uh) < 0x1p22f)) {
    p = -1;
    f = 0.f;
    return (uh == uh && ue == ue) ? kUFar : kUNaN;
  }
  float kf = floorf(uh);
  float fr = __fadd_rn(__fsub_rn(uh, kf), ue);            // uh - kf is exact
  if (fr < 0.f) {
    kf -= 1.f;
    fr = __fadd_rn(fr, 1.f);
  } else if (fr >= 1.f) {
    kf += 1.f;
    fr = __fsub_rn(fr, 1.f);
  }
  if (fr >= 1.f) fr = 0x1.fffffep-1f;                     // rounding of a fraction just below 1
  p = (int)kf;
  f = fr;
  return kUOk;
}

// ----------------------------------------------------------------------------------------------
// One axis of Eq. 6 and of the pixel coordinate in float32 only: uf = ((lh x - ah) - loh) * sch, and a bound E on
// |uf - u| for the exact u of (lam, alpha, lo, sc): the four roundings (<= u each of the magnitudes involved,
// A = |lh x| + |ah| + |loh| in pixel units) and the dropped low parts (|ll x| <= u |lh x|, |lol| <= u |loh|,
// |scl| <= u sch, and |al| itself) sum to <= 5u (A + |uf|) + |al| sch; E = 2^-21 (A + |uf|) + |al| sch is that
// with more than 1.5x to spare, which also covers the float32 rounding of E.
__device__ __forceinline__ float fast_pixel(float x, float lh, float ah, float al, float loh, float sch, float& e) {
  const float pr = __fmul_rn(lh, x);
  const float uf = __fmul_rn(__fsub_rn(__fsub_rn(pr, ah), loh), sch);
  e = __fmaf_rn(fabsf(al), sch, 0x1p-21f * __fmaf_rn(fabsf(pr) + fabsf(ah) + fabsf(loh), sch, fabsf(uf)));
  return uf;
}

// Certain decision of one axis from u = p + f (f in [0, 1)) known to within m (m < 1/2): inside pixel p of
// the np pixels, or outside the window on this axis.
__device__ __forceinline__ bool axis_inside(int p, float f, float m, int np) {
  return p >= 0 && p < np && f >= m && f <= 1.f - m;
}
__device__ __forceinline__ bool axis_outside(int p, float f, float m, int np) {
  // u + m < 0 iff p <= -2, or p = -1 and 1 - f > m; u - m >= np iff p > np, or p = np and f >= m
  return p <= -2 || (p == -1 && 1.f - f > m) || p > np || (p == np && f >= m);
}

// ----------------------------------------------------------------------------------------------
// Eq. 6 and binning of a thread's RPT rays (ray k at grid column i_base + STRIDE k of call row
// jrel): counts, the out-of-window count, and, with certified binning, the list of rays to
// re-evaluate in float-float.  Every lane of the warp must call it (warp-aggregated atomics).
//
// With certified binning most rays are decided from a float32 evaluation of u with a bound on its
// own rounding (fast_pixel): certain when u's band, widened by that bound, lies inside one pixel or
// outside the window.  The others take the float-float evaluation (ff_pixel) and its narrower margin,
// and those still uncertain are listed for the float-float re-evaluation over the lenses.
// ----------------------------------------------------------------------------------------------
template <int RPT, int STRIDE>
__device__ __forceinline__ void bin_rays(const ShootDesc& d, const float (&x1)[RPT], const float (&x2)[RPT],
                                         const float (&a1h)[RPT], const float (&a1l)[RPT], const float (&a2h)[RPT],
                                         const float (&a2l)[RPT], const float (&sig)[RPT], const float (&tn)[RPT],
                                         const bool (&valid)[RPT], int64_t jrel, int64_t i_base, int lane) {
  unsigned oow_lane = 0;
  const bool certify = d.rc_list != nullptr;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    int p1 = -1, p2 = -1;
    bool inwin = false, decided = false, need = false;
    float band = 0.f;
    if (certify) {
      band = band_halfwidth(sig[k], tn[k], d.f.lamabs, x1[k], x2[k]);
      float e1, e2;
      const float u1 = fast_pixel(x1[k], d.lam1h, a1h[k], a1l[k], d.lo0h, d.sc0h, e1);
      const float u2 = fast_pixel(x2[k], d.lam2h, a2h[k], a2l[k], d.lo1h, d.sc1h, e2);
      const float m1 = band * d.scf0 + e1 + 1e-7f, m2 = band * d.scf1 + e2 + 1e-7f;
      if (fabsf(u1) < 0x1p22f && fabsf(u2) < 0x1p22f && m1 < 0.5f && m2 < 0.5f) {  // NaN fails
        const float k1 = floorf(u1), k2 = floorf(u2);
        const int q1 = (int)k1, q2 = (int)k2;
        const float f1 = __fsub_rn(u1, k1), f2 = __fsub_rn(u2, k2);  // exact for |u| < 2^22
        const bool in_sure = axis_inside(q1, f1, m1, d.np0) && axis_inside(q2, f2, m2, d.np1);
        const bool out_sure = axis_outside(q1, f1, m1, d.np0) || axis_outside(q2, f2, m2, d.np1);
        decided = in_sure || out_sure;
        inwin = in_sure;
        p1 = q1;
        p2 = q2;
      }
    }
    if (!decided) {
      // Eq. 6 and u = (y - lo) * npix / (hi - lo) in float-float (~2^-44 relative): pixel index p and
      // fraction f of u, and the bound eu on the float-float rounding (pixel units)
      float f1, f2, eu1, eu2;
      const int st1 = ff_pixel(x1[k], d.lam1h, d.lam1l, a1h[k], a1l[k], d.lo0h, d.lo0l, d.sc0h, d.sc0l, p1, f1, eu1);
      const int st2 = ff_pixel(x2[k], d.lam2h, d.lam2l, a2h[k], a2l[k], d.lo1h, d.lo1l, d.sc1h, d.sc1l, p2, f2, eu2);
      inwin = st1 == kUOk && st2 == kUOk && (p1 >= 0) && (p1 < d.np0) && (p2 >= 0) && (p2 < d.np1);
      if (certify) {
        // Certain: the band [u - du, u + du] lies inside one pixel of the window, or outside the window
        // on some axis.  Margins: the band in pixel units, the float-float rounding, and 1e-7 for the
        // float rounding of the fraction (margins below 1/2; wider bands are never certain).
        const float m1 = band * d.scf0 + eu1 + 1e-7f, m2 = band * d.scf1 + eu2 + 1e-7f;
        const bool ok1 = st1 == kUOk && m1 < 0.5f, ok2 = st2 == kUOk && m2 < 0.5f;
        const bool out1 = ok1 && axis_outside(p1, f1, m1, d.np0);
        const bool out2 = ok2 && axis_outside(p2, f2, m2, d.np1);
        // a non-finite position is out of window by definition; |u| >= 2^22 is when the window is narrower
        const bool out_sure = st1 == kUNaN || st2 == kUNaN || (st1 == kUFar && d.np0 <= (1 << 21)) ||
                              (st2 == kUFar && d.np1 <= (1 << 21)) || out1 || out2;
        const bool in_sure = inwin && ok1 && ok2 && axis_inside(p1, f1, m1, d.np0) && axis_inside(p2, f2, m2, d.np1);
        need = valid[k] && !out_sure && !in_sure;
      }
    }
    bool bin_now = valid[k];
    if (certify) {
      const unsigned mask = __ballot_sync(0xffffffffu, need);
      if (mask != 0u) {
        const int leader = __ffs(mask) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(d.rc_count, (unsigned)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) {
          const unsigned slot = base + (unsigned)__popc(mask & ((1u << lane) - 1u));
          if (slot < d.rc_cap) {
            const int64_t i = i_base + STRIDE * k;
            d.rc_list[slot] = make_uint2((unsigned)d.field_id, (unsigned)(jrel * d.n0 + i));
            bin_now = false;  // counted by the float-float re-evaluation
          } else {
            atomicOr(d.f.status, kStatusListFull);  // list full: the ray keeps its float32 decision
          }
        }
      }
    }
    if (bin_now && inwin) atomicAdd(d.counts + (size_t)p2 * (size_t)d.np0 + (size_t)p1, 1u);
    const unsigned miss = __ballot_sync(0xffffffffu, bin_now && !inwin);
    oow_lane += __popc(miss);
  }
  if (d.oow != nullptr && lane == 0 && oow_lane != 0) atomicAdd(d.oow, (unsigned long long)oow_lane);
}

// ----------------------------------------------------------------------------------------------
// Ray tiles of a shoot call.  A CTA of WARPS warps covers WARPS consecutive grid rows (one per
// warp) by 32 * RPT consecutive columns; lane l of a warp holds columns c0 + l + 32 k, k < RPT.
// ----------------------------------------------------------------------------------------------
template <int WARPS, int RPT>
__host__ __device__ __forceinline__ int64_t shoot_tiles(int64_t n_rows, int64_t n0) {
  const int64_t seg = 32 * RPT;
  return ((n_rows + WARPS - 1) / WARPS) * ((n0 + seg - 1) / seg);
}

// Shared memory of the shoot kernels: lens tiles and row table, and the near-lens search of the
// CTA's ray box.
template <int WARPS, int RPT, int TILE>
struct ShootSmem {
  LensSmem<TILE, WARPS> lens;
  NearSmem<TILE, 1, WARPS * 32, RPT> near;
};

template <int WARPS, int RPT, int TILE, bool MASS>
__device__ __forceinline__ bool shoot_tile(const ShootDesc& d, int64_t tile, ShootSmem<WARPS, RPT, TILE>& ss,
                                           PipeState& ps) {
  LensSmem<TILE, WARPS>& sm = ss.lens;
  constexpr int SEG = 32 * RPT;
  static_assert(SEG <= kMaxSeg, "tile columns fit the shared coordinate row");
  const int64_t ncol = (d.n0 + SEG - 1) / SEG;
  const int64_t trow = tile / ncol;
  const int64_t tcol = tile - trow * ncol;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t jrel = trow * WARPS + warp;
  const bool row_ok = jrel < d.n_rows;
  // Ray coordinates (float64 fma rounded to float, as the header defines them) of the tile's SEG
  // columns and WARPS rows, each formed once per CTA rather than once per warp: the float64 pipe is
  // narrow, and on small fields these conversions would otherwise delay every tile's start.
  for (int c = threadIdx.x; c < SEG + WARPS; c += WARPS * 32) {
    if (c < SEG) {
      int64_t i = tcol * SEG + c;
      if (i >= d.n0) i = d.n0 - 1;
      sm.x1col[c] = ray_coord(i, d.sp0, d.or0);
    } else {
      int64_t jr = trow * WARPS + (c - SEG);
      if (jr >= d.n_rows) jr = d.n_rows - 1;
      sm.x2row[c - SEG] = ray_coord(d.j_begin + jr, d.sp1, d.or1);  // also read by build_row_table
    }
  }
  if (threadIdx.x == 0) {
    // the tile's ray box: coordinates grow with the grid index
    const int64_t ia = tcol * SEG, ib = min(ia + SEG, d.n0) - 1;
    const int64_t ja = trow * WARPS, jb = min(ja + WARPS, d.n_rows) - 1;
    near_set_box(ss.near, 0, ray_coord(ia, d.sp0, d.or0), ray_coord(ib, d.sp0, d.or0),
                 ray_coord(d.j_begin + ja, d.sp1, d.or1), ray_coord(d.j_begin + jb, d.sp1, d.or1));
  }
  __syncthreads();
  const float x2r = sm.x2row[warp];
  float x1[RPT], x2[RPT];
  bool valid[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t i = tcol * SEG + lane + 32 * k;
    valid[k] = row_ok && i < d.n0;
    x1[k] = sm.x1col[lane + 32 * k];
    x2[k] = x2r;
  }
  float a1h[RPT], a1l[RPT], a2h[RPT], a2l[RPT], sig[RPT], tn[RPT];
  if (!deflect_pairs<RPT, TILE, MASS, true, WARPS>(d.f, x1, x2, a1h, a1l, a2h, a2l, sig, tn, sm, ps, &ss.near))
    return false;
  bin_rays<RPT, 32>(d, x1, x2, a1h, a1l, a2h, a2l, sig, tn, valid, jrel, tcol * SEG + lane, lane);
  return true;
}

}  // namespace rsdev
