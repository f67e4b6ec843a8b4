// C-ABI layer of librs.so, core: error reporting, argument validation, fields (static and moving),
// launch shape selection, the plain, culled and listed-ray shoots, Eq. 4 normalisation, the
// bounded-wait self-test, and the small elementwise kernels (lens repacking, lens motion, Eq. 4).
// Batches, lens-partitioned shoots and light curves live in rs_api_batch.cu, rs_api_staged.cu and
// rs_api_lightcurve.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rs_host.h"

using rsdev::FieldDev;
using rsdev::ShootDesc;

namespace {

__global__ void pack_lenses_kernel(const float* __restrict__ xy, const float* __restrict__ m, int64_t n, int64_t n_pad,
                                   float4* __restrict__ lens4, float2* __restrict__ mass2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const float2 p = reinterpret_cast<const float2*>(xy)[i];
      lens4[i] = make_float4(p.x, p.x, p.y, p.y);
      if (mass2) {
        const float mi = m[i];
        mass2[i] = make_float2(mi, mi);
      }
    } else {
      lens4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mass2) mass2[i] = make_float2(0.f, 0.f);
    }
  }
}

// flag[0] |= 1 if some mass is not exactly 1 (NaN included): such a field needs the weighted kernels;
// flag[1] = max of the bit patterns of |m| (the largest |m|: non-negative floats order as their bits).
__global__ void mass_check_kernel(const float* __restrict__ m, int64_t n, unsigned int* __restrict__ flag) {
  bool weighted = false;
  unsigned int mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    weighted |= !(m[i] == 1.0f);
    mx = max(mx, __float_as_uint(fabsf(m[i])));
  }
  if (__syncthreads_or(weighted) && threadIdx.x == 0) atomicOr(flag, 1u);
  atomicMax(flag + 1, mx);
}

// Moving fields: {x1, x2, v1, v2} per lens at t = 0.
__global__ void motion_pack_kernel(const float* __restrict__ xy, const float* __restrict__ v, int64_t n,
                                   float4* __restrict__ motion) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 p = reinterpret_cast<const float2*>(xy)[i];
    const float2 q = reinterpret_cast<const float2*>(v)[i];
    motion[i] = make_float4(p.x, p.y, q.x, q.y);
  }
}

// Lens positions at time t: x + v t in double (product, then sum, no fma), rounded to float32; the
// packed layout of pack_lenses_kernel (padding lenses untouched).
__global__ void move_lenses_kernel(const float4* __restrict__ motion, int64_t n, double t, float4* __restrict__ lens4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 m = motion[i];
    const float x1 = __double2float_rn(__dadd_rn((double)m.x, __dmul_rn((double)m.z, t)));
    const float x2 = __double2float_rn(__dadd_rn((double)m.y, __dmul_rn((double)m.w, t)));
    lens4[i] = make_float4(x1, x1, x2, x2);
  }
}

// Eq. 4: mu = N * (1 / N_av), float32; uint4/float4 vectors when aligned.
__global__ void magnification_kernel(const uint32_t* __restrict__ c, float* __restrict__ mu, int64_t n, float inv_nav,
                                     int vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (vec) {
    const int64_t nv = n / 4;
    const uint4* c4 = reinterpret_cast<const uint4*>(c);
    float4* m4 = reinterpret_cast<float4*>(mu);
    for (int64_t i = t0; i < nv; i += stride) {
      const uint4 v = c4[i];
      m4[i] = make_float4((float)v.x * inv_nav, (float)v.y * inv_nav, (float)v.z * inv_nav, (float)v.w * inv_nav);
    }
    done = nv * 4;
  }
  for (int64_t i = done + t0; i < n; i += stride) mu[i] = (float)c[i] * inv_nav;
}

// Waits on an mbarrier phase that nothing completes, with the given limit: exercises the bounded
// wait and its error status without hanging or faulting the device.
__global__ void selftest_wait_kernel(uint64_t limit_ns, unsigned int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    rsdev::mbar_init(&bar, 1);
    rsdev::mbar_fence_init();
  }
  __syncthreads();
  const bool ok = rsdev::mbar_wait_bounded(&bar, 0u, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) *out = ok ? 0u : rsdev::kStatusTimeout;
}

}  // namespace

namespace rshost {

thread_local std::string g_err;
// Launch shape per mass mode (index 0: unit masses, 1: per-lens masses).
int g_cfg[2] = {rsint::kDefaultCfg, rsint::kDefaultCfg};
// Certified binning (float-float re-evaluation of rays inside their error band of a pixel edge).
int g_certify = 1;
// Device memory for the per-ray state of a staged (lens-partitioned) shoot; larger calls run in row blocks.
size_t g_staged_budget = (size_t)2 << 30;

// Allocation-failure injection (test support): when armed with n >= 0, the n-th following library
// allocation (0: the next one) reports cudaErrorMemoryAllocation instead of allocating.
std::atomic<int64_t> g_alloc_fail_in{-1};

bool inject_alloc_failure() {
  int64_t v = g_alloc_fail_in.load();
  while (v >= 0)
    if (g_alloc_fail_in.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

int recheck_grid(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v < 1) v = 1;
  return v * 8;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
              cudaGetErrorString(e));
}

int check_grid(const rs_ray_grid* g) {
  if (!g) return fail(RS_EINVAL, "ray grid is NULL");
  for (int k = 0; k < 2; ++k) {
    if (!finite_coord(g->origin[k])) return fail(RS_EINVAL, "grid origin[%d] not finite or beyond 1e9", k);
    if (!(std::isfinite(g->spacing[k]) && g->spacing[k] > 0.0))
      return fail(RS_EINVAL, "grid spacing[%d] must be finite and > 0", k);
    if (g->n[k] < 0) return fail(RS_EINVAL, "grid n[%d] < 0", k);
    const double far = g->origin[k] + (double)(g->n[k] > 0 ? g->n[k] - 1 : 0) * g->spacing[k];
    if (!finite_coord(far)) return fail(RS_EINVAL, "grid extent along axis %d beyond 1e9", k);
  }
  return RS_OK;
}

int check_window(const rs_window* w) {
  if (!w) return fail(RS_EINVAL, "window is NULL");
  for (int k = 0; k < 2; ++k) {
    if (!(std::isfinite(w->lo[k]) && std::isfinite(w->hi[k]) && w->hi[k] > w->lo[k]))
      return fail(RS_EINVAL, "window axis %d: need finite lo < hi", k);
    if (w->npix[k] < 1) return fail(RS_EINVAL, "window npix[%d] < 1", k);
    if (w->npix[k] > (1 << 22)) return fail(RS_EINVAL, "window npix[%d] > 2^22", k);
    const double sc = (double)w->npix[k] / (w->hi[k] - w->lo[k]);
    if (!(std::isfinite(sc) && sc > 0.0)) return fail(RS_EINVAL, "window axis %d: degenerate pixel scale", k);
  }
  if ((int64_t)w->npix[0] * (int64_t)w->npix[1] > (int64_t)1 << 40)
    return fail(RS_EOVERFLOW, "window has more than 2^40 pixels");
  return RS_OK;
}

// The arguments every shoot call shares: grid, row range, window and the counts buffer.
int check_call(const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w, const uint32_t* d_counts) {
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if ((rc = check_window(w)) != RS_OK) return rc;
  if (!d_counts) return fail(RS_EINVAL, "d_counts is NULL");
  if (row_begin < 0 || row_end < row_begin || row_end > g->n[1])
    return fail(RS_EINVAL, "row range [%lld, %lld) outside [0, %lld]", (long long)row_begin, (long long)row_end,
                (long long)g->n[1]);
  return RS_OK;
}

int check_field_device(const rs_field* f) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != f->device) return fail(RS_EINVAL, "field lives on device %d but device %d is current", f->device, cur);
  return RS_OK;
}

int num_sms(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
  return v > 0 ? v : 1;
}

int fill_desc(const rs_field* f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w,
              uint32_t* d_counts, uint64_t* d_oow, ShootDesc* d) {
  const int64_t rows = row_end - row_begin;
  const int64_t n_rays = rows * g->n[0];
  if (g->n[0] > 0 && rows > 0 && (rows > ((int64_t)1 << 32) / g->n[0] || n_rays >= ((int64_t)1 << 32)))
    return fail(RS_EOVERFLOW, "a call shoots at most 2^32 - 1 rays (got %lld rows x %lld)", (long long)rows,
                (long long)g->n[0]);
  memset(d, 0, sizeof(*d));
  d->f = f->dev;
  d->or0 = g->origin[0];
  d->or1 = g->origin[1];
  d->sp0 = g->spacing[0];
  d->sp1 = g->spacing[1];
  d->n0 = g->n[0];
  d->j_begin = row_begin;
  d->n_rows = rows;
  d->lo0 = w->lo[0];
  d->lo1 = w->lo[1];
  d->sc0 = (double)w->npix[0] / (w->hi[0] - w->lo[0]);
  d->sc1 = (double)w->npix[1] / (w->hi[1] - w->lo[1]);
  // rounded up so that the float band in pixel units is never narrower than in float64
  d->scf0 = std::nextafter((float)d->sc0, INFINITY);
  d->scf1 = std::nextafter((float)d->sc1, INFINITY);
  d->np0 = w->npix[0];
  d->np1 = w->npix[1];
  d->counts = d_counts;
  d->oow = reinterpret_cast<unsigned long long*>(d_oow);
  // float-float splits for the float32 epilogue (hi = nearest float, lo = nearest float of the rest)
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  split(d->f.lam1, d->lam1h, d->lam1l);
  split(d->f.lam2, d->lam2h, d->lam2l);
  split(d->lo0, d->lo0h, d->lo0l);
  split(d->lo1, d->lo1h, d->lo1l);
  split(d->sc0, d->sc0h, d->sc0l);
  split(d->sc1, d->sc1h, d->sc1l);
  return RS_OK;
}

float near_cap(int64_t n_lens, float m_max) {
  // the near radius h is 1: the cap on every term of a lens farther than h is the largest mass itself
  return n_lens > 0 ? m_max : 0.f;
}

cudaError_t launch_pack_lenses(const float* xy, const float* m, int64_t n, int64_t n_pad, float4* lens4,
                               float2* mass2, int blocks, cudaStream_t s) {
  pack_lenses_kernel<<<blocks, 256, 0, s>>>(xy, m, n, n_pad, lens4, mass2);
  return cudaGetLastError();
}

}  // namespace rshost

using namespace rshost;

extern "C" {

const char* rs_last_error(void) { return g_err.c_str(); }

const char* rs_version(void) { return "rs-gb300 0.4 (sm_103a)"; }

int rs_device_code_version(int* binary_version) {
  if (!binary_version) return fail(RS_EINVAL, "binary_version is NULL");
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, magnification_kernel);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
  *binary_version = a.binaryVersion;
  return RS_OK;
}

int rs_set_launch_config(int has_masses, int block, int rays_per_thread, int lens_tile, int min_ctas) {
  const int c = rsint::find_cfg(block, rays_per_thread, lens_tile, min_ctas);
  if (c < 0)
    return fail(RS_EINVAL, "no compiled launch shape (%d threads, %d rays/thread, %d-lens tiles, %d CTAs/SM)", block,
                rays_per_thread, lens_tile, min_ctas);
  g_cfg[has_masses ? 1 : 0] = c;
  return RS_OK;
}

int rs_get_launch_config(int has_masses, int* block, int* rays_per_thread, int* lens_tile, int* min_ctas) {
  const int c = g_cfg[has_masses ? 1 : 0];
  if (block) *block = rsint::kCfgs[c].block;
  if (rays_per_thread) *rays_per_thread = rsint::kCfgs[c].rpt;
  if (lens_tile) *lens_tile = rsint::kCfgs[c].tile;
  if (min_ctas) *min_ctas = rsint::kCfgs[c].min_ctas;
  return RS_OK;
}

int rs_launch_occupancy(int has_masses, int block, int rays_per_thread, int lens_tile, int min_ctas,
                        int* ctas_per_sm) {
  if (!ctas_per_sm) return fail(RS_EINVAL, "ctas_per_sm is NULL");
  const int c = rsint::find_cfg(block, rays_per_thread, lens_tile, min_ctas);
  if (c < 0)
    return fail(RS_EINVAL, "no compiled launch shape (%d threads, %d rays/thread, %d-lens tiles, %d CTAs/SM)", block,
                rays_per_thread, lens_tile, min_ctas);
  cudaError_t e = rsint::shoot_blocks_per_sm(c, has_masses != 0, ctas_per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  return RS_OK;
}

int rs_launch_configs(int* shapes, int cap, int* count) {
  if (count) *count = rsint::kNumCfg;
  for (int i = 0; i < rsint::kNumCfg && i < cap && shapes; ++i) {
    shapes[4 * i] = rsint::kCfgs[i].block;
    shapes[4 * i + 1] = rsint::kCfgs[i].rpt;
    shapes[4 * i + 2] = rsint::kCfgs[i].tile;
    shapes[4 * i + 3] = rsint::kCfgs[i].min_ctas;
  }
  return RS_OK;
}

int rs_create_field(const float* lens_xy, const float* masses, int64_t n_lens, double kappa_c, double gamma,
                    int inputs_on_device, void* stream, rs_field_t* out) {
  if (!out) return fail(RS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_lens < 0) return fail(RS_EINVAL, "n_lens < 0");
  if (n_lens >= ((int64_t)1 << 31) - rsdev::kLensPad) return fail(RS_EOVERFLOW, "n_lens must be < 2^31 - 1024");
  if (n_lens > 0 && !lens_xy) return fail(RS_EINVAL, "lens_xy is NULL");
  if (!std::isfinite(kappa_c) || !std::isfinite(gamma)) return fail(RS_EINVAL, "kappa_c and gamma must be finite");
  // masses that are all exactly 1 select the unit-mass kernels, as NULL does (the masses are still
  // stored, so such a field can be a lens partition next to weighted ones)
  bool unit_masses = true;
  float m_max = n_lens > 0 ? 1.f : 0.f;  // largest mass (the near-lens band term's cap)
  if (!inputs_on_device) {
    for (int64_t i = 0; i < 2 * n_lens; ++i)
      if (!finite_coord((double)lens_xy[i])) return fail(RS_EINVAL, "lens coordinate %lld not finite or beyond 1e9", (long long)i);
    if (masses) {
      m_max = 0.f;
      for (int64_t i = 0; i < n_lens; ++i) {
        if (!(std::isfinite(masses[i]) && masses[i] >= 0.f)) return fail(RS_EINVAL, "mass %lld not finite or negative", (long long)i);
        unit_masses = unit_masses && masses[i] == 1.0f;
        m_max = std::max(m_max, masses[i]);
      }
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rs_field* f = new (std::nothrow) rs_field();
  if (!f) return fail(RS_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&f->device);
  if (e != cudaSuccess) {
    delete f;
    return cuda_fail(e, "cudaGetDevice");
  }
  f->n_lens = n_lens;
  f->n_pad = (n_lens + rsdev::kLensPad - 1) / rsdev::kLensPad * rsdev::kLensPad;
  if (f->n_pad == 0) f->n_pad = rsdev::kLensPad;  // keep a valid (unused) tile for empty fields
  f->kappa_c = kappa_c;
  f->gamma = gamma;
  const bool has_mass = masses != nullptr;
  float* tmp_xy = nullptr;
  float* tmp_m = nullptr;
  auto cleanup = [&]() {
    cudaFree(f->lens4);
    cudaFree(f->mass2);
    cudaFree(f->status);
    cudaFree(tmp_xy);
    cudaFree(tmp_m);
    delete f;
  };
  // status word, and a second word for the mass check of device inputs
  if ((e = dev_alloc(&f->lens4, sizeof(float4) * f->n_pad)) != cudaSuccess ||
      (has_mass && (e = dev_alloc(&f->mass2, sizeof(float2) * f->n_pad)) != cudaSuccess) ||
      (e = dev_alloc(&f->status, 2 * sizeof(unsigned int))) != cudaSuccess) {
    int rc = cuda_fail(e, "cudaMalloc (field)");
    cleanup();
    return rc;
  }
  const float* src_xy = lens_xy;
  const float* src_m = masses;
  if (!inputs_on_device && n_lens > 0) {
    if ((e = dev_alloc(&tmp_xy, sizeof(float) * 2 * n_lens)) != cudaSuccess ||
        (has_mass && (e = dev_alloc(&tmp_m, sizeof(float) * n_lens)) != cudaSuccess)) {
      int rc = cuda_fail(e, "cudaMalloc (staging)");
      cleanup();
      return rc;
    }
    if ((e = cudaMemcpyAsync(tmp_xy, lens_xy, sizeof(float) * 2 * n_lens, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (has_mass && (e = cudaMemcpyAsync(tmp_m, masses, sizeof(float) * n_lens, cudaMemcpyHostToDevice, s)) != cudaSuccess)) {
      int rc = cuda_fail(e, "cudaMemcpyAsync (lenses)");
      cudaStreamSynchronize(s);
      cleanup();
      return rc;
    }
    src_xy = tmp_xy;
    src_m = tmp_m;
  }
  if ((e = cudaMemsetAsync(f->status, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess) {
    int rc = cuda_fail(e, "cudaMemsetAsync (status)");
    cudaStreamSynchronize(s);
    cleanup();
    return rc;
  }
  if (has_mass && inputs_on_device && n_lens > 0) {
    // unit-mass test and largest mass of device inputs: the two status words serve as the flag and
    // the maximum, read back and cleared
    unsigned int check[2] = {0u, 0u};
    const int blocks = (int)std::min<int64_t>((n_lens + 255) / 256, (int64_t)num_sms(f->device) * 8);
    mass_check_kernel<<<blocks, 256, 0, s>>>(masses, n_lens, f->status);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(check, f->status, sizeof(check), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess ||
        (e = cudaMemsetAsync(f->status, 0, sizeof(check), s)) != cudaSuccess) {
      int rc = cuda_fail(e, "mass check");
      cudaStreamSynchronize(s);
      cleanup();
      return rc;
    }
    unit_masses = check[0] == 0u;
    std::memcpy(&m_max, &check[1], sizeof(float));
  }
  {
    const int threads = 256;
    const int64_t want = (f->n_pad + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)num_sms(f->device) * 16);
    pack_lenses_kernel<<<blocks, threads, 0, s>>>(n_lens > 0 ? src_xy : nullptr, src_m, n_lens, f->n_pad, f->lens4,
                                                  has_mass ? f->mass2 : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      int rc = cuda_fail(e, "pack_lenses_kernel launch");
      cudaStreamSynchronize(s);
      cleanup();
      return rc;
    }
  }
  if (tmp_xy || tmp_m) {
    // staging buffers: free once the packing kernel has consumed them
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
      int rc = cuda_fail(e, "cudaStreamSynchronize (field upload)");
      cleanup();
      return rc;
    }
    cudaFree(tmp_xy);
    cudaFree(tmp_m);
    tmp_xy = tmp_m = nullptr;
  }
  f->dev.lens4 = f->lens4;
  f->dev.mass2 = has_mass ? f->mass2 : nullptr;
  f->dev.n_lens = (int32_t)n_lens;
  f->dev.has_mass = (has_mass && !unit_masses) ? 1 : 0;
  f->dev.lam1 = (1.0 - kappa_c) - gamma;
  f->dev.lam2 = (1.0 - kappa_c) + gamma;
  f->dev.lamabs = std::nextafter((float)std::max(std::fabs(f->dev.lam1), std::fabs(f->dev.lam2)), INFINITY);
  f->dev.mcap = near_cap(n_lens, f->dev.has_mass ? m_max : 1.f);
  f->dev.status = f->status;
  *out = f;
  return RS_OK;
}

int rs_destroy_field(rs_field_t f) {
  if (!f) return RS_OK;
  if (f->views > 0) return fail(RS_EINVAL, "the field has %d live lens-range views: destroy them first", f->views);
  DeviceGuard g(f->device);
  cudaDeviceSynchronize();
  cudaFree(f->lens4);
  cudaFree(f->mass2);
  cudaFree(f->status);
  cudaFree(f->motion);
  if (f->parent) --f->parent->views;
  delete f;
  return RS_OK;
}

// a view starts on a summation-period boundary (the group and renormalisation schedule then runs as in
// its parent); its lens tiles are copied exactly (rounded up to an even count), inside the parent's padding
static_assert(rsdev::kLensPad % 2 == 0 && rsdev::kRenorm % rsdev::kGroup == 0, "views on period boundaries");

int rs_create_field_view(rs_field_t parent, int64_t lens_begin, int64_t n_lens, rs_field_t* out) {
  if (!out) return fail(RS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!parent) return fail(RS_EINVAL, "parent field is NULL");
  if (lens_begin < 0 || n_lens < 0 || lens_begin > parent->n_lens || n_lens > parent->n_lens - lens_begin)
    return fail(RS_EINVAL, "lens range [%lld, %lld + %lld) not within the field's %lld lenses", (long long)lens_begin,
                (long long)lens_begin, (long long)n_lens, (long long)parent->n_lens);
  if (lens_begin % rsdev::kRenorm != 0) return fail(RS_EINVAL, "lens_begin must be a multiple of %d", rsdev::kRenorm);
  DeviceGuard g(parent->device);
  rs_field* f = new (std::nothrow) rs_field();
  if (!f) return fail(RS_ENOMEM, "host allocation failed");
  cudaError_t e = dev_alloc(&f->status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(f->status, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "view status word");
    cudaFree(f->status);
    delete f;
    return rc;
  }
  f->device = parent->device;
  f->n_lens = n_lens;
  f->n_pad = (n_lens + rsdev::kLensPad - 1) / rsdev::kLensPad * rsdev::kLensPad;
  f->kappa_c = parent->kappa_c;
  f->gamma = parent->gamma;
  f->lens4 = nullptr;  // not owned
  f->mass2 = nullptr;
  f->dev = parent->dev;
  // full lens tiles past the range stay inside the parent's padded arrays: lens_begin is a multiple
  // of the tile and the parent's padding reaches the next multiple of kLensPad
  f->dev.lens4 = parent->dev.lens4 + lens_begin;
  f->dev.mass2 = parent->dev.mass2 ? parent->dev.mass2 + lens_begin : nullptr;
  f->dev.n_lens = (int32_t)n_lens;
  f->dev.status = f->status;
  f->parent = parent;
  ++parent->views;
  *out = f;
  return RS_OK;
}

int rs_create_moving_field(const float* lens_xy, const float* vel_xy, const float* masses, int64_t n_lens,
                           double kappa_c, double gamma, int inputs_on_device, void* stream, rs_field_t* out) {
  if (!out) return fail(RS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_lens > 0 && !vel_xy) return fail(RS_EINVAL, "vel_xy is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // bounds of |x| and |v| for the coordinate check of rs_field_set_time (host copies of device inputs)
  std::vector<float> hxy, hv;
  const float* pxy = lens_xy;
  const float* pv = vel_xy;
  if (inputs_on_device && n_lens > 0) {
    hxy.resize(2 * n_lens);
    hv.resize(2 * n_lens);
    cudaError_t e = cudaMemcpy(hxy.data(), lens_xy, sizeof(float) * 2 * n_lens, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hv.data(), vel_xy, sizeof(float) * 2 * n_lens, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (moving-field bounds)");
    pxy = hxy.data();
    pv = hv.data();
  }
  double max_x = 0.0, max_v = 0.0;
  for (int64_t i = 0; i < 2 * n_lens; ++i) {
    if (!finite_coord((double)pxy[i])) return fail(RS_EINVAL, "lens coordinate %lld not finite or beyond 1e9", (long long)i);
    if (!std::isfinite(pv[i])) return fail(RS_EINVAL, "velocity %lld not finite", (long long)i);
    max_x = std::max(max_x, std::fabs((double)pxy[i]));
    max_v = std::max(max_v, std::fabs((double)pv[i]));
  }
  rs_field_t f = nullptr;
  int rc = rs_create_field(lens_xy, masses, n_lens, kappa_c, gamma, inputs_on_device, stream, &f);
  if (rc != RS_OK) return rc;
  float* tmp = nullptr;
  cudaError_t e = dev_alloc(&f->motion, sizeof(float4) * (size_t)std::max<int64_t>(n_lens, 1));
  if (e == cudaSuccess && n_lens > 0) {
    const float* dxy = lens_xy;
    const float* dv = vel_xy;
    if (!inputs_on_device) {
      e = dev_alloc(&tmp, sizeof(float) * 4 * n_lens);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, lens_xy, sizeof(float) * 2 * n_lens, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp + 2 * n_lens, vel_xy, sizeof(float) * 2 * n_lens, cudaMemcpyHostToDevice, s);
      dxy = tmp;
      dv = tmp + 2 * n_lens;
    }
    if (e == cudaSuccess) {
      const int threads = 256;
      const int blocks = (int)std::min<int64_t>((n_lens + threads - 1) / threads, (int64_t)num_sms(f->device) * 16);
      motion_pack_kernel<<<blocks, threads, 0, s>>>(dxy, dv, n_lens, f->motion);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // staging consumed; positions ready
  }
  cudaFree(tmp);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "moving-field upload");
    rs_destroy_field(f);
    return rc;
  }
  f->max_x = max_x;
  f->max_v = max_v;
  *out = f;
  return RS_OK;
}

int rs_field_set_time(rs_field_t f, double t, void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  if (!f->motion) return fail(RS_EINVAL, "field has no velocities (create it with rs_create_moving_field)");
  if (!std::isfinite(t)) return fail(RS_EINVAL, "time must be finite");
  if (!(f->max_x + f->max_v * std::fabs(t) <= kCoordLimit))
    return fail(RS_EINVAL, "lens coordinates at t = %g may exceed 1e9", t);
  int rc;
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  f->time = t;
  if (f->n_lens == 0) return RS_OK;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((f->n_lens + threads - 1) / threads, (int64_t)num_sms(f->device) * 16);
  move_lenses_kernel<<<blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(f->motion, f->n_lens, t,
                                                                                     f->lens4);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "move_lenses_kernel launch");
  return RS_OK;
}

int rs_field_time(rs_field_t f, double* t) {
  if (!f || !t) return fail(RS_EINVAL, "NULL argument");
  *t = f->parent ? f->parent->time : f->time;  // a view moves with its parent
  return RS_OK;
}

int rs_field_info(rs_field_t f, int64_t* n_lens, int* has_masses) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  if (n_lens) *n_lens = f->n_lens;
  if (has_masses) *has_masses = f->dev.has_mass;
  return RS_OK;
}

int rs_field_status(rs_field_t f, int clear, int* status) {
  if (!f || !status) return fail(RS_EINVAL, "NULL argument");
  DeviceGuard g(f->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  unsigned int v = 0;
  if ((e = cudaMemcpy(&v, f->status, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (status)");
  *status = (v & 0xffu) == rsdev::kStatusTimeout ? RS_ETIMEOUT : (v & rsdev::kStatusListFull) ? RS_EOVERFLOW : RS_OK;
  if (clear && v != 0) {
    if ((e = cudaMemset(f->status, 0, sizeof(unsigned int))) != cudaSuccess) return cuda_fail(e, "cudaMemset (status)");
  }
  return RS_OK;
}

int rs_shoot_rows(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w,
                  uint32_t* d_counts, uint64_t* d_out_of_window, void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  int rc;
  if ((rc = check_call(g, row_begin, row_end, w, d_counts)) != RS_OK) return rc;
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  ShootDesc d;
  if ((rc = fill_desc(f, g, row_begin, row_end, w, d_counts, d_out_of_window, &d)) != RS_OK) return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  cudaError_t e = cudaSuccess;
  if (g_certify) {
    // stream-ordered workspace: [count | pad | list of {field, ray}]
    d.rc_cap = rsint::recheck_capacity(d.n_rows * d.n0);
    if ((e = dev_alloc_async(&ws, 16 + sizeof(uint2) * (size_t)d.rc_cap, s)) != cudaSuccess)
      return cuda_fail(e, "cudaMallocAsync (re-evaluation list)");
    d.rc_count = reinterpret_cast<unsigned int*>(ws);
    d.rc_list = reinterpret_cast<uint2*>(reinterpret_cast<char*>(ws) + 16);
    e = cudaMemsetAsync(d.rc_count, 0, sizeof(unsigned int), s);
  }
  if (e == cudaSuccess) e = rsint::launch_shoot(g_cfg[f->dev.has_mass ? 1 : 0], d, s);
  if (e == cudaSuccess && ws) e = rsint::launch_recheck(&d, nullptr, d.rc_list, d.rc_count, d.rc_cap, recheck_grid(f->device), s);
  if (ws) {
    cudaError_t e2 = cudaFreeAsync(ws, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return cuda_fail(e, "shoot launch");
  return RS_OK;
}

int rs_shoot_culled(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w,
                    uint32_t* d_counts, uint64_t* d_out_of_window, uint64_t* d_rays_shot, void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  int rc;
  if ((rc = check_call(g, row_begin, row_end, w, d_counts)) != RS_OK) return rc;
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  ShootDesc d;
  if ((rc = fill_desc(f, g, row_begin, row_end, w, d_counts, d_out_of_window, &d)) != RS_OK) return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t n_cx = 0;
  const int64_t n_cells = rsint::cull_cells(d.n_rows, d.n0, &n_cx);
  const int64_t n_coarse = rsint::cull_coarse_cells(d.n_rows, d.n0);
  // stream-ordered workspace: [re-evaluation count | coarse count | kept count | re-evaluation list |
  // coarse cell list | cell list]
  const unsigned cap = g_certify ? rsint::recheck_capacity(d.n_rows * d.n0) : 0u;
  const size_t coarse_off = 32 + sizeof(uint2) * (size_t)cap;
  const size_t list_off = coarse_off + sizeof(unsigned) * (size_t)n_coarse;
  void* ws = nullptr;
  cudaError_t e = dev_alloc_async(&ws, list_off + sizeof(unsigned) * (size_t)n_cells, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (culled-shoot workspace)");
  char* base = reinterpret_cast<char*>(ws);
  unsigned* n_coarse_kept = reinterpret_cast<unsigned*>(base + 8);
  unsigned* n_kept = reinterpret_cast<unsigned*>(base + 16);
  unsigned* coarse = reinterpret_cast<unsigned*>(base + coarse_off);
  unsigned* cells = reinterpret_cast<unsigned*>(base + list_off);
  if (g_certify) {
    d.rc_cap = cap;
    d.rc_count = reinterpret_cast<unsigned int*>(base);
    d.rc_list = reinterpret_cast<uint2*>(base + 32);
  }
  e = cudaMemsetAsync(base, 0, 32, s);
  if (e == cudaSuccess)
    e = rsint::launch_cull(d, w->hi[0], w->hi[1], coarse, n_coarse_kept, cells, n_kept,
                           reinterpret_cast<unsigned long long*>(d_rays_shot), s);
  if (e == cudaSuccess) {
    const int64_t want = (n_cells + 3) / 4;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms(f->device) * 2));
    e = rsint::launch_shoot_cells(d, n_cx, cells, n_kept, grid, s);
  }
  if (e == cudaSuccess && g_certify)
    e = rsint::launch_recheck(&d, nullptr, d.rc_list, d.rc_count, d.rc_cap, recheck_grid(f->device), s);
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "culled shoot launch");
  return RS_OK;
}

int rs_shoot(rs_field_t f, const rs_ray_grid* g, const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window,
             void* stream) {
  if (!g) return fail(RS_EINVAL, "ray grid is NULL");
  return rs_shoot_rows(f, g, 0, g->n[1], w, d_counts, d_out_of_window, stream);
}

int rs_trace(rs_field_t f, const rs_ray_grid* g, const int64_t* d_ray_ij, int64_t k, double* d_y, double* d_alpha,
             double* d_err, void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if (k < 0) return fail(RS_EINVAL, "k < 0");
  if (k == 0) return RS_OK;
  if (!d_ray_ij || !d_y) return fail(RS_EINVAL, "d_ray_ij / d_y is NULL");
  if (k >= ((int64_t)1 << 31)) return fail(RS_EOVERFLOW, "k must be < 2^31");
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  cudaError_t e = rsint::launch_trace(f->dev, g->origin[0], g->origin[1], g->spacing[0], g->spacing[1], d_ray_ij, k,
                                      d_y, d_alpha, d_err, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "trace kernel launch");
  return RS_OK;
}

int rs_trace_certified(rs_field_t f, const rs_ray_grid* g, const int64_t* d_ray_ij, int64_t k, double* d_y,
                       double* d_alpha, void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if (k < 0) return fail(RS_EINVAL, "k < 0");
  if (k == 0) return RS_OK;
  if (!d_ray_ij || !d_y) return fail(RS_EINVAL, "d_ray_ij / d_y is NULL");
  if (k >= ((int64_t)1 << 31)) return fail(RS_EOVERFLOW, "k must be < 2^31");
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  cudaError_t e = rsint::launch_trace_ff(f->dev, g->origin[0], g->origin[1], g->spacing[0], g->spacing[1], d_ray_ij,
                                         k, d_y, d_alpha, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "certified trace kernel launch");
  return RS_OK;
}

int rs_selftest_bounded_wait(int64_t limit_ns, int* status) {
  if (!status) return fail(RS_EINVAL, "status is NULL");
  if (limit_ns < 0 || limit_ns > 2000000000LL) return fail(RS_EINVAL, "limit_ns must be in [0, 2e9]");
  unsigned int* d = nullptr;
  cudaError_t e = dev_alloc(&d, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (self-test)");
  selftest_wait_kernel<<<1, 32>>>((uint64_t)limit_ns, d);
  e = cudaGetLastError();
  unsigned int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof(v), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "self-test kernel");
  *status = v == 0 ? RS_OK : (int)v;
  return RS_OK;
}

int rs_set_certified_binning(int enabled) {
  g_certify = enabled ? 1 : 0;
  return RS_OK;
}

int rs_set_alloc_failure(int64_t n) {
  if (n < -1) return fail(RS_EINVAL, "n must be >= -1");
  g_alloc_fail_in.store(n);
  return RS_OK;
}

int rs_get_certified_binning(int* enabled) {
  if (!enabled) return fail(RS_EINVAL, "enabled is NULL");
  *enabled = g_certify;
  return RS_OK;
}

int rs_magnification(const uint32_t* d_counts, const rs_ray_grid* g, const rs_window* w, float* d_mu, void* stream) {
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if ((rc = check_window(w)) != RS_OK) return rc;
  if (!d_counts || !d_mu) return fail(RS_EINVAL, "d_counts / d_mu is NULL");
  const double pix_area = ((w->hi[0] - w->lo[0]) / (double)w->npix[0]) * ((w->hi[1] - w->lo[1]) / (double)w->npix[1]);
  const double n_av = pix_area / (g->spacing[0] * g->spacing[1]);
  if (!(std::isfinite(n_av) && n_av > 0.0)) return fail(RS_EINVAL, "N_av is not a positive finite number");
  const int64_t n = (int64_t)w->npix[0] * (int64_t)w->npix[1];
  int dev = 0;
  cudaGetDevice(&dev);
  const int vec = ((reinterpret_cast<uintptr_t>(d_counts) | reinterpret_cast<uintptr_t>(d_mu)) & 15u) == 0;
  const int threads = 256;
  const int64_t want = ((vec ? n / 4 : n) + threads - 1) / threads;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms(dev) * 8));
  magnification_kernel<<<blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_counts, d_mu, n,
                                                                                        (float)(1.0 / n_av), vec);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "magnification kernel launch");
  return RS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------ no allocation
//
// rs_shoot_rows_noalloc: rs_shoot_rows with certified binning whose re-evaluation list lives in
// this file's static device array instead of memory allocated per call.  For callers that must
// not allocate device memory once they run: code replayed inside a CUDA graph whose capture
// forbids allocation nodes, applications whose own allocator has reserved the device memory up
// front, and latency-critical loops that cannot afford an allocator call.

// Re-evaluation list shared by every rs_shoot_rows_noalloc call: a 256-byte header (the entry
// counter) followed by up to kStaticRecheckEntries {field, ray} entries.  4 MiB + 256 B on each
// device that loads the library, held until the process exits.
constexpr unsigned int kStaticRecheckEntries = 1u << 19;
static __device__ __align__(256) unsigned char g_static_recheck[256 + sizeof(uint2) * kStaticRecheckEntries];

namespace {

constexpr int kMaxDevices = 64;
constexpr int64_t kStaticMaxRays = (int64_t)kStaticRecheckEntries * 32;  // one list entry per 32 rays: 2^24
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};
void* g_static_ctx[kMaxDevices] = {};

// The current CUDA context (through the driver entry point, so the library needs no link to the
// driver library), or nullptr where it cannot be queried.
void* current_context() {
  using GetCtx = int (*)(void**);
  static GetCtx fn = []() -> GetCtx {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<GetCtx>(p);
  }();
  void* ctx = nullptr;
  if (fn == nullptr || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of g_static_recheck in the current device's context, looked up on the first call
// on a device and again whenever the context changed (after a device reset the module, and with it
// the array, is loaded anew).  In host code the array's name only stands in for the device symbol;
// its address must come from cudaGetSymbolAddress with the device current.
int static_recheck_ptr(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return fail(RS_EINVAL, "device index %d beyond %d", device, kMaxDevices);
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[device] || g_static_ctx[device] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_recheck);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static re-evaluation list)");
    g_static_ptr[device] = p;
    g_static_ctx[device] = ctx;
  }
  *out = g_static_ptr[device];
  return RS_OK;
}

}  // namespace

extern "C" int rs_shoot_rows_noalloc(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                                     const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window,
                                     void* stream) {
  if (!f) return fail(RS_EINVAL, "field is NULL");
  int rc;
  if ((rc = check_call(g, row_begin, row_end, w, d_counts)) != RS_OK) return rc;
  if ((rc = check_field_device(f)) != RS_OK) return rc;
  ShootDesc d;
  if ((rc = fill_desc(f, g, row_begin, row_end, w, d_counts, d_out_of_window, &d)) != RS_OK) return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  if (d.n_rows * d.n0 > kStaticMaxRays)
    return fail(RS_EOVERFLOW,
                "rs_shoot_rows_noalloc shoots at most 2^24 rays per call (its static re-evaluation list holds %u "
                "entries, one per 32 rays); got %lld rays: split the rows over several calls",
                kStaticRecheckEntries, (long long)(d.n_rows * d.n0));
  const unsigned int cap = rsint::recheck_capacity(d.n_rows * d.n0);
  void* base = nullptr;
  if ((rc = static_recheck_ptr(f->device, &base)) != RS_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  d.rc_count = reinterpret_cast<unsigned int*>(base);
  d.rc_list = reinterpret_cast<uint2*>(reinterpret_cast<char*>(base) + 256);
  d.rc_cap = cap;
  // the array keeps the previous call's contents: only the counter must start at zero
  cudaError_t e = cudaMemsetAsync(d.rc_count, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = rsint::launch_shoot(g_cfg[f->dev.has_mass ? 1 : 0], d, s);
  if (e == cudaSuccess) e = rsint::launch_recheck(&d, nullptr, d.rc_list, d.rc_count, d.rc_cap, recheck_grid(f->device), s);
  if (e != cudaSuccess) return cuda_fail(e, "shoot launch (no-allocation variant)");
  return RS_OK;
}

