// Host-side internals shared by the C-ABI translation units (rs_api*.cu): the field object, argument
// validation, error reporting, launch descriptors and the allocation wrappers.  Not part of the ABI.
#pragma once

#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/rs.h"
#include "rs_internal.h"

struct rs_field {
  int device;
  int64_t n_lens;
  int64_t n_pad;
  float4* lens4;
  float2* mass2;
  unsigned int* status;
  double kappa_c, gamma;
  rsdev::FieldDev dev;
  // moving fields: {x1, x2, v1, v2} at t = 0 per lens, bounds of |x| and |v|, current time
  float4* motion = nullptr;
  double max_x = 0.0, max_v = 0.0, time = 0.0;
  // lens-range views: the field a view reads (views own only their status word), and the number
  // of live views of a field (it cannot be destroyed while any is left)
  rs_field* parent = nullptr;
  int views = 0;
};

namespace rshost {

// Launch shape per mass mode (index 0: unit masses, 1: per-lens masses).
extern int g_cfg[2];
// Certified binning (float-float re-evaluation of rays inside their error band of a pixel edge).
extern int g_certify;
// Device memory for the per-ray state of a staged (lens-partitioned) shoot; larger calls run in row blocks.
extern size_t g_staged_budget;
// Allocation-failure injection (test support): when armed with n >= 0, the n-th following library
// allocation (0: the next one) reports cudaErrorMemoryAllocation instead of allocating.
extern std::atomic<int64_t> g_alloc_fail_in;
bool inject_alloc_failure();

template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

template <class T>
cudaError_t dev_alloc_async(T** p, size_t bytes, cudaStream_t s) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}

template <class T>
cudaError_t host_alloc(T** p, size_t bytes) {
  if (inject_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

// Message for rs_last_error (thread-local); returns code.
int fail(int code, const char* fmt, ...);
// RS_ENOMEM for an allocation failure, RS_ECUDA otherwise, with the CUDA error in the message.
int cuda_fail(cudaError_t e, const char* what);

// Coordinates (lens positions, ray grid, track samples) must be finite with |value| <= 1e9.
constexpr double kCoordLimit = 1e9;
inline bool finite_coord(double v) { return std::isfinite(v) && std::fabs(v) <= kCoordLimit; }

int check_grid(const rs_ray_grid* g);
int check_window(const rs_window* w);
// The arguments every shoot call shares: grid, row range, window and the counts buffer.
int check_call(const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w, const uint32_t* d_counts);
int check_field_device(const rs_field* f);

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

int num_sms(int device);
// CTAs of the float-float re-evaluation kernels (eight per SM).
int recheck_grid(int device);
// The launch descriptor of a shoot call over rows [row_begin, row_end) (RS_EOVERFLOW beyond 2^32 - 1 rays).
int fill_desc(const rs_field* f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w,
              uint32_t* d_counts, uint64_t* d_oow, rsdev::ShootDesc* d);
// The field's cap on the term m / r of any lens farther than the near radius from a ray (0 without lenses).
float near_cap(int64_t n_lens, float m_max);
// Repack n lenses (xy interleaved, m or null) into the padded layout of n_pad entries.
cudaError_t launch_pack_lenses(const float* xy, const float* m, int64_t n, int64_t n_pad, float4* lens4,
                               float2* mass2, int blocks, cudaStream_t s);

}  // namespace rshost
