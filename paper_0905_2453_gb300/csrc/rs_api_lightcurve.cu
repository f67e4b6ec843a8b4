// C-ABI layer, light curves (Section 1): validation and descriptor tables for rs_light_curves and
// light-curve plans.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rs_host.h"

using namespace rshost;

struct rs_lc_plan {
  int device;
  int n_tracks;
  int64_t total;
  int profile;
  double cut2;
  float ecut;
  int grid;
  rsint::LcTrack* d_table;
};

namespace {

// Validated light-curve launch parameters: the per-track descriptor table (tracks with samples, in
// output order), the number of samples and the profile constants.
struct LcPlan {
  std::vector<rsint::LcTrack> table;
  int64_t total = 0;
  int profile = 0;
  double cut2 = 0.0;
  float ecut = 0.f;
};

int lc_prepare(int n_maps, const float* const* d_mu, const rs_window* windows, int profile, double s,
               int n_tracks, const rs_track* tracks, LcPlan* plan) {
  if (profile != RS_PROFILE_GAUSSIAN && profile != RS_PROFILE_DISC)
    return fail(RS_EINVAL, "profile must be RS_PROFILE_GAUSSIAN or RS_PROFILE_DISC");
  if (!(std::isfinite(s) && s > 0.0)) return fail(RS_EINVAL, "profile size s must be finite and > 0");
  if (n_tracks < 0) return fail(RS_EINVAL, "n_tracks < 0");
  if (n_tracks > 0 && !tracks) return fail(RS_EINVAL, "tracks is NULL");
  int64_t total = 0;
  for (int t = 0; t < n_tracks; ++t) {
    if (tracks[t].n < 0) return fail(RS_EINVAL, "track %d: n < 0", t);
    total += tracks[t].n;
    if (total > ((int64_t)1 << 40)) return fail(RS_EOVERFLOW, "more than 2^40 samples in one call");
  }
  plan->total = total;
  plan->profile = profile;
  if (total == 0) return RS_OK;
  if (n_maps < 1 || !d_mu || !windows) return fail(RS_EINVAL, "n_maps >= 1 with non-NULL d_mu and windows needed");
  // profile support radius and the exponent scale: Gaussian E = d^2 / (2 s^2) cut at (6 s)^2 (the device
  // works with E log2(e), so that the weight is one base-2 exponential), disc E = d^2 / s^2 cut at 1
  const double R = profile == RS_PROFILE_GAUSSIAN ? 6.0 * s : s;
  const double cut2 = profile == RS_PROFILE_GAUSSIAN ? (6.0 * s) * (6.0 * s) : s * s;
  const double kLog2e = 1.4426950408889634;
  const double escale = profile == RS_PROFILE_GAUSSIAN ? kLog2e / (2.0 * s * s) : 1.0 / (s * s);
  const double ecut_d = profile == RS_PROFILE_GAUSSIAN ? 18.0 * kLog2e : 1.0;
  const float ecut = (float)ecut_d;
  if (!(std::isfinite(cut2) && cut2 > 0.0 && std::isfinite(escale))) return fail(RS_EINVAL, "profile size s out of range");
  std::vector<rsint::LcTrack>& table = plan->table;
  table.reserve(n_tracks);
  int64_t off = 0;
  for (int t = 0; t < n_tracks; ++t) {
    const rs_track& tr = tracks[t];
    if (tr.n == 0) continue;
    if (tr.map < 0 || tr.map >= n_maps) return fail(RS_EINVAL, "track %d: map %d outside [0, %d)", t, tr.map, n_maps);
    const rs_window* w = &windows[tr.map];
    int rc;
    if ((rc = check_window(w)) != RS_OK) return rc;
    if (!d_mu[tr.map]) return fail(RS_EINVAL, "map %d is NULL", tr.map);
    rsint::LcTrack d{};
    d.mu = d_mu[tr.map];
    d.np0 = w->npix[0];
    d.np1 = w->npix[1];
    double pix[2], rp[2];
    for (int k = 0; k < 2; ++k) {
      if (w->npix[k] > (1 << 24)) return fail(RS_EINVAL, "map %d: light curves need npix[%d] <= 2^24", tr.map, k);
      pix[k] = (w->hi[k] - w->lo[k]) / (double)w->npix[k];
      if (std::max(std::fabs(w->lo[k]), std::fabs(w->hi[k])) / pix[k] > 1073741824.0)
        return fail(RS_EINVAL, "map %d axis %d: max(|lo|, |hi|) / pixel must be <= 2^30", tr.map, k);
      rp[k] = R / pix[k];
      if (!(rp[k] <= 1048576.0)) return fail(RS_EINVAL, "profile spans more than 2^20 pixels along axis %d of map %d", k, tr.map);
      const double last = tr.y0[k] + (double)(tr.n - 1) * tr.step[k];
      if (!finite_coord(tr.y0[k]) || !std::isfinite(tr.step[k]) || !finite_coord(last))
        return fail(RS_EINVAL, "track %d: samples must be finite with |y| <= 1e9", t);
    }
    d.lo0 = w->lo[0];
    d.lo1 = w->lo[1];
    d.pix0 = pix[0];
    d.pix1 = pix[1];
    d.y00 = tr.y0[0];
    d.y01 = tr.y0[1];
    d.st0 = tr.step[0];
    d.st1 = tr.step[1];
    d.t00 = (tr.y0[0] - w->lo[0]) / pix[0] - 0.5;
    d.t01 = (tr.y0[1] - w->lo[1]) / pix[1] - 0.5;
    d.d0 = tr.step[0] / pix[0];
    d.d1 = tr.step[1] / pix[1];
    d.rp0 = rp[0];
    d.rp1 = rp[1];
    d.a0 = (float)(pix[0] * pix[0] * escale);
    d.a1 = (float)(pix[1] * pix[1] * escale);
    d.inv_a0 = 1.0f / d.a0;
    if (!(d.a0 > 0.f && d.a1 > 0.f && std::isfinite(d.a0) && std::isfinite(d.a1) && std::isfinite(d.inv_a0)))
      return fail(RS_EINVAL, "map %d: pixel / profile size ratio outside the float32 range", tr.map);
    // the float32 exponent is within ~8u ((R + pix0)^2 + (R + pix1)^2) escale + 4u E of the exact one
    // (offsets in pixel units carry u (|offset| + 1)); the band takes 2^-16 of that scale (~30x margin)
    d.band = (float)(std::ldexp((std::pow(R + pix[0], 2) + std::pow(R + pix[1], 2)) * escale + ecut_d, -16));
    d.n = tr.n;
    d.out_off = off;
    off += tr.n;
    table.push_back(d);
  }
  plan->cut2 = cut2;
  plan->ecut = ecut;
  return RS_OK;
}

int lc_grid(int device, int64_t total) {
  const int64_t want = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms(device) * 8));
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------------------------------------ light curves

int rs_light_curves(int n_maps, const float* const* d_mu, const rs_window* windows, int profile, double s,
                    int n_tracks, const rs_track* tracks, double* d_mu_out, double* d_dm_out, void* stream) {
  LcPlan plan;
  int rc = lc_prepare(n_maps, d_mu, windows, profile, s, n_tracks, tracks, &plan);
  if (rc != RS_OK || plan.total == 0) return rc;
  if (!d_mu_out) return fail(RS_EINVAL, "d_mu_out is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rsint::LcTrack* d_table = nullptr;
  const size_t bytes = plan.table.size() * sizeof(rsint::LcTrack);
  if ((e = dev_alloc_async(&d_table, bytes, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMallocAsync (track table)");
  e = cudaMemcpyAsync(d_table, plan.table.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = rsint::launch_light_curves(plan.profile, d_table, (int)plan.table.size(), plan.total, plan.cut2, plan.ecut,
                                   d_mu_out, d_dm_out, lc_grid(dev, plan.total), st);
  cudaFreeAsync(d_table, st);
  if (e != cudaSuccess) return cuda_fail(e, "light-curve kernel");
  return RS_OK;
}

int rs_light_curve_plan_create(int n_maps, const float* const* d_mu, const rs_window* windows, int profile,
                               double s, int n_tracks, const rs_track* tracks, rs_lc_plan_t* out) {
  if (!out) return fail(RS_EINVAL, "out is NULL");
  *out = nullptr;
  LcPlan plan;
  int rc = lc_prepare(n_maps, d_mu, windows, profile, s, n_tracks, tracks, &plan);
  if (rc != RS_OK) return rc;
  rs_lc_plan* p = new (std::nothrow) rs_lc_plan{};
  if (!p) return fail(RS_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  p->n_tracks = (int)plan.table.size();
  p->total = plan.total;
  p->profile = plan.profile;
  p->cut2 = plan.cut2;
  p->ecut = plan.ecut;
  p->grid = lc_grid(p->device, plan.total);
  if (p->n_tracks > 0) {
    const size_t bytes = plan.table.size() * sizeof(rsint::LcTrack);
    if ((e = dev_alloc(&p->d_table, bytes)) != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaMalloc (track table)");
    }
    if ((e = cudaMemcpy(p->d_table, plan.table.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(p->d_table);
      delete p;
      return cuda_fail(e, "cudaMemcpy (track table)");
    }
  }
  *out = p;
  return RS_OK;
}

int rs_light_curve_plan_samples(rs_lc_plan_t p, int64_t* n_samples) {
  if (!p || !n_samples) return fail(RS_EINVAL, "NULL argument");
  *n_samples = p->total;
  return RS_OK;
}

int rs_light_curve_plan_launch(rs_lc_plan_t p, double* d_mu_out, double* d_dm_out, void* stream) {
  if (!p) return fail(RS_EINVAL, "plan is NULL");
  if (p->total == 0) return RS_OK;
  if (!d_mu_out) return fail(RS_EINVAL, "d_mu_out is NULL");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != p->device) return fail(RS_EINVAL, "plan lives on device %d but device %d is current", p->device, cur);
  e = rsint::launch_light_curves(p->profile, p->d_table, p->n_tracks, p->total, p->cut2, p->ecut, d_mu_out, d_dm_out,
                                 p->grid, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "light-curve kernel");
  return RS_OK;
}

int rs_light_curve_plan_destroy(rs_lc_plan_t p) {
  if (!p) return RS_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->d_table) cudaFree(p->d_table);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
  return RS_OK;
}

}  // extern "C"
