// C-ABI layer, lens-partitioned shooting (Section 3.3): fields given as device shards
// (rs_shoot_staged) and lenses streamed from host memory (rs_shoot_streamed).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rs_host.h"

using rsdev::FieldDev;
using rsdev::ShootDesc;
using namespace rshost;

extern "C" {

int rs_set_staged_state_budget(uint64_t bytes) {
  if (bytes < ((uint64_t)1 << 20)) return fail(RS_EINVAL, "the staged state budget must be at least 1 MiB");
  g_staged_budget = (size_t)bytes;
  return RS_OK;
}

int rs_shoot_staged(int n_parts, const rs_field_t* parts, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                    const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream) {
  if (n_parts < 1 || !parts) return fail(RS_EINVAL, "need n_parts >= 1 lens partitions");
  for (int p = 0; p < n_parts; ++p) {
    if (!parts[p]) return fail(RS_EINVAL, "partition %d is NULL", p);
    const rs_field* a = parts[p];
    const rs_field* b = parts[0];
    if (a->device != b->device || (a->dev.mass2 != nullptr) != (b->dev.mass2 != nullptr) || a->kappa_c != b->kappa_c ||
        a->gamma != b->gamma)
      return fail(RS_EINVAL, "partition %d differs from partition 0 in device, stored masses, kappa_c or gamma", p);
    if (p + 1 < n_parts && a->n_lens % rsdev::kRenorm != 0)
      return fail(RS_EINVAL, "partition %d holds %lld lenses: all but the last must hold a multiple of %d", p,
                  (long long)a->n_lens, rsdev::kRenorm);
  }
  // one kernel for every partition: the weighted one if any partition has masses other than 1 (all
  // partitions then store masses)
  int weighted = 0;
  for (int p = 0; p < n_parts; ++p) weighted |= parts[p]->dev.has_mass;
  int rc;
  if ((rc = check_call(g, row_begin, row_end, w, d_counts)) != RS_OK) return rc;
  if ((rc = check_field_device(parts[0])) != RS_OK) return rc;
  ShootDesc d;
  if ((rc = fill_desc(parts[0], g, row_begin, row_end, w, d_counts, d_out_of_window, &d)) != RS_OK) return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // ray blocks whose carried state fits the budget (the state is 28 bytes per ray, padded to tiles)
  const size_t budget = g_staged_budget;
  const size_t per4 = rsint::staged_state_bytes(4, d.n0);
  const int64_t rows_blk = std::max<int64_t>(4, (int64_t)(budget / per4) * 4);
  const int64_t rows_max = std::min<int64_t>(rows_blk, d.n_rows);
  const size_t state_bytes = rsint::staged_state_bytes(rows_max, d.n0);
  const unsigned cap = g_certify ? rsint::recheck_capacity(rows_max * d.n0) : 0u;
  const size_t list_off = (state_bytes + 255) / 256 * 256;
  const size_t ff_off = list_off + 16 + sizeof(uint2) * (size_t)cap;
  void* ws = nullptr;
  cudaError_t e = dev_alloc_async(&ws, ff_off + sizeof(float4) * (size_t)cap, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (staged-shoot workspace)");
  char* base = reinterpret_cast<char*>(ws);
  uint64_t* state = reinterpret_cast<uint64_t*>(base);
  float4* ff = reinterpret_cast<float4*>(base + ff_off);
  if (g_certify) {
    d.rc_cap = cap;
    d.rc_count = reinterpret_cast<unsigned int*>(base + list_off);
    d.rc_list = reinterpret_cast<uint2*>(base + list_off + 16);
  }
  const int rgrid = recheck_grid(parts[0]->device);
  for (int64_t r0 = 0; r0 < d.n_rows && e == cudaSuccess; r0 += rows_blk) {
    ShootDesc db = d;
    db.j_begin = d.j_begin + r0;
    db.n_rows = std::min<int64_t>(rows_blk, d.n_rows - r0);
    if (g_certify) e = cudaMemsetAsync(db.rc_count, 0, sizeof(unsigned int), s);
    for (int p = 0; p < n_parts && e == cudaSuccess; ++p) {
      db.f = parts[p]->dev;
      db.f.has_mass = weighted;
      e = rsint::launch_staged(db, state, p == 0, p == n_parts - 1, s);
    }
    if (g_certify) {
      for (int p = 0; p < n_parts && e == cudaSuccess; ++p) {
        db.f = parts[p]->dev;
        db.f.has_mass = weighted;
        e = rsint::launch_recheck_part(db, db.rc_list, db.rc_count, db.rc_cap, ff, p == 0, rgrid, s);
      }
      if (e == cudaSuccess) e = rsint::launch_recheck_bin(db, db.rc_list, db.rc_count, db.rc_cap, ff, rgrid, s);
    }
  }
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "staged shoot launch");
  return RS_OK;
}

int rs_shoot_streamed(const float* h_lens_xy, const float* h_masses, int64_t n_lens, double kappa_c, double gamma,
                      int64_t lenses_per_pass, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                      const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream) {
  if (n_lens < 0) return fail(RS_EINVAL, "n_lens < 0");
  if (n_lens > 0 && !h_lens_xy) return fail(RS_EINVAL, "h_lens_xy is NULL");
  if (lenses_per_pass < rsdev::kLensPad || lenses_per_pass % rsdev::kLensPad != 0 || lenses_per_pass > ((int64_t)1 << 30))
    return fail(RS_EINVAL, "lenses_per_pass must be a multiple of %d in [%d, 2^30]", rsdev::kLensPad, rsdev::kLensPad);
  if (!std::isfinite(kappa_c) || !std::isfinite(gamma)) return fail(RS_EINVAL, "kappa_c and gamma must be finite");
  for (int64_t i = 0; i < 2 * n_lens; ++i)
    if (!finite_coord((double)h_lens_xy[i])) return fail(RS_EINVAL, "lens coordinate %lld not finite or beyond 1e9", (long long)i);
  bool unit_masses = true;
  float m_max = 0.f;
  if (h_masses)
    for (int64_t i = 0; i < n_lens; ++i) {
      if (!(std::isfinite(h_masses[i]) && h_masses[i] >= 0.f)) return fail(RS_EINVAL, "mass %lld not finite or negative", (long long)i);
      unit_masses = unit_masses && h_masses[i] == 1.0f;
      m_max = std::max(m_max, h_masses[i]);
    }
  int rc;
  if ((rc = check_call(g, row_begin, row_end, w, d_counts)) != RS_OK) return rc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const bool mass = h_masses != nullptr && !unit_masses;  // masses all 1: the unit-mass kernels, none copied
  const int64_t P = lenses_per_pass;
  const int64_t n_parts = std::max<int64_t>(1, (n_lens + P - 1) / P);
  // a partition buffer's descriptor; the lens arrays are filled pass by pass
  rs_field proto{};
  proto.device = dev;
  proto.kappa_c = kappa_c;
  proto.gamma = gamma;
  proto.dev.has_mass = mass ? 1 : 0;
  proto.dev.lam1 = (1.0 - kappa_c) - gamma;
  proto.dev.lam2 = (1.0 - kappa_c) + gamma;
  proto.dev.lamabs = std::nextafter((float)std::max(std::fabs(proto.dev.lam1), std::fabs(proto.dev.lam2)), INFINITY);
  // every pass carries the cap of the whole lens set, as a field of all the lenses would
  proto.dev.mcap = near_cap(n_lens, mass ? m_max : 1.f);
  ShootDesc d;
  if ((rc = fill_desc(&proto, g, row_begin, row_end, w, d_counts, d_out_of_window, &d)) != RS_OK) return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // resources: two device partition buffers {raw xy, raw m, packed lens4, packed mass2}, two pinned
  // staging buffers, a copy stream, events, the status word, the state and re-evaluation workspace
  struct Res {
    char* dbuf[2] = {nullptr, nullptr};
    char* hbuf[2] = {nullptr, nullptr};
    unsigned int* status = nullptr;
    void* ws = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    ~Res() {
      if (cs) cudaStreamSynchronize(cs);
      for (int b = 0; b < 2; ++b) {
        if (dbuf[b]) cudaFree(dbuf[b]);
        if (hbuf[b]) cudaFreeHost(hbuf[b]);
        if (ready[b]) cudaEventDestroy(ready[b]);
        if (freed[b]) cudaEventDestroy(freed[b]);
        if (copied[b]) cudaEventDestroy(copied[b]);
      }
      if (status) cudaFree(status);
      if (ws) cudaFree(ws);
      if (cs) cudaStreamDestroy(cs);
    }
  } r;
  const size_t raw_xy = sizeof(float) * 2 * (size_t)P, raw_m = mass ? sizeof(float) * (size_t)P : 0;
  const size_t off_m = raw_xy, off_l4 = (off_m + raw_m + 255) / 256 * 256;
  const size_t off_m2 = off_l4 + sizeof(float4) * (size_t)P, dbytes = off_m2 + (mass ? sizeof(float2) * (size_t)P : 0);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    if ((e = dev_alloc(&r.dbuf[b], dbytes)) != cudaSuccess) break;
    if ((e = host_alloc(&r.hbuf[b], raw_xy + raw_m)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&r.ready[b], cudaEventDisableTiming)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&r.freed[b], cudaEventDisableTiming)) != cudaSuccess) break;
    e = cudaEventCreateWithFlags(&r.copied[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r.cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dev_alloc(&r.status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(r.status, 0, sizeof(unsigned int));
  // state and re-evaluation workspace, as rs_shoot_staged
  const int64_t rows_blk = std::max<int64_t>(4, (int64_t)(g_staged_budget / rsint::staged_state_bytes(4, d.n0)) * 4);
  const int64_t rows_max = std::min<int64_t>(rows_blk, d.n_rows);
  const size_t state_bytes = rsint::staged_state_bytes(rows_max, d.n0);
  const unsigned cap = g_certify ? rsint::recheck_capacity(rows_max * d.n0) : 0u;
  const size_t list_off = (state_bytes + 255) / 256 * 256;
  const size_t ff_off = list_off + 16 + sizeof(uint2) * (size_t)cap;
  if (e == cudaSuccess) e = dev_alloc(&r.ws, ff_off + sizeof(float4) * (size_t)cap);
  if (e != cudaSuccess) return cuda_fail(e, "streamed-shoot resources");
  char* base = reinterpret_cast<char*>(r.ws);
  uint64_t* state = reinterpret_cast<uint64_t*>(base);
  float4* ff = reinterpret_cast<float4*>(base + ff_off);
  if (g_certify) {
    d.rc_cap = cap;
    d.rc_count = reinterpret_cast<unsigned int*>(base + list_off);
    d.rc_list = reinterpret_cast<uint2*>(base + list_off + 16);
  }
  FieldDev fdev[2];
  for (int b = 0; b < 2; ++b) {
    fdev[b] = proto.dev;
    fdev[b].lens4 = reinterpret_cast<const float4*>(r.dbuf[b] + off_l4);
    fdev[b].mass2 = mass ? reinterpret_cast<const float2*>(r.dbuf[b] + off_m2) : nullptr;
    fdev[b].status = r.status;
  }
  const int threads = 256;
  const int pblocks = (int)std::min<int64_t>((P + threads - 1) / threads, (int64_t)num_sms(dev) * 16);
  const int rgrid = recheck_grid(dev);
  bool used[2] = {false, false};
  // One sweep over the partitions: partition p goes through pinned buffer p % 2 (host copy once the
  // previous copy out of it finished), then to device buffer p % 2 (once the kernel that read it
  // finished) and is packed there; `pass` enqueues the kernel that consumes it on the caller's stream.
  auto sweep = [&](auto pass) -> cudaError_t {
    cudaError_t ee = cudaSuccess;
    for (int64_t p = 0; p < n_parts && ee == cudaSuccess; ++p) {
      const int b = (int)(p & 1);
      const int64_t a0 = p * P, np = std::min<int64_t>(P, n_lens - a0);
      if (used[b] && (ee = cudaEventSynchronize(r.copied[b])) != cudaSuccess) break;
      if (np > 0) {
        std::memcpy(r.hbuf[b], h_lens_xy + 2 * a0, sizeof(float) * 2 * (size_t)np);
        if (mass) std::memcpy(r.hbuf[b] + raw_xy, h_masses + a0, sizeof(float) * (size_t)np);
      }
      if (used[b] && (ee = cudaStreamWaitEvent(r.cs, r.freed[b], 0)) != cudaSuccess) break;
      if (np > 0 && (ee = cudaMemcpyAsync(r.dbuf[b], r.hbuf[b], raw_xy + raw_m, cudaMemcpyHostToDevice, r.cs)) !=
                        cudaSuccess)
        break;
      if ((ee = cudaEventRecord(r.copied[b], r.cs)) != cudaSuccess) break;
      ee = launch_pack_lenses(np > 0 ? reinterpret_cast<const float*>(r.dbuf[b]) : nullptr,
                              mass ? reinterpret_cast<const float*>(r.dbuf[b] + off_m) : nullptr, np, P,
                              reinterpret_cast<float4*>(r.dbuf[b] + off_l4),
                              mass ? reinterpret_cast<float2*>(r.dbuf[b] + off_m2) : nullptr, pblocks, r.cs);
      if (ee != cudaSuccess) break;
      if ((ee = cudaEventRecord(r.ready[b], r.cs)) != cudaSuccess) break;
      if ((ee = cudaStreamWaitEvent(s, r.ready[b], 0)) != cudaSuccess) break;
      FieldDev fd = fdev[b];
      fd.n_lens = (int32_t)np;
      if ((ee = pass(fd, p == 0, p == n_parts - 1)) != cudaSuccess) break;
      if ((ee = cudaEventRecord(r.freed[b], s)) != cudaSuccess) break;
      used[b] = true;
    }
    return ee;
  };
  for (int64_t r0 = 0; r0 < d.n_rows && e == cudaSuccess; r0 += rows_blk) {
    ShootDesc db = d;
    db.j_begin = d.j_begin + r0;
    db.n_rows = std::min<int64_t>(rows_blk, d.n_rows - r0);
    if (g_certify) e = cudaMemsetAsync(db.rc_count, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess)
      e = sweep([&](const FieldDev& fd, bool first, bool last) {
        ShootDesc dp = db;
        dp.f = fd;
        return rsint::launch_staged(dp, state, first, last, s);
      });
    if (e == cudaSuccess && g_certify) {
      e = sweep([&](const FieldDev& fd, bool first, bool) {
        ShootDesc dp = db;
        dp.f = fd;
        return rsint::launch_recheck_part(dp, db.rc_list, db.rc_count, db.rc_cap, ff, first, rgrid, s);
      });
      if (e == cudaSuccess) e = rsint::launch_recheck_bin(db, db.rc_list, db.rc_count, db.rc_cap, ff, rgrid, s);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "streamed shoot");
  unsigned int st = 0;
  if ((e = cudaMemcpy(&st, r.status, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (status)");
  if ((st & 0xffu) == rsdev::kStatusTimeout) return fail(RS_ETIMEOUT, "a bounded wait for a lens tile gave up");
  if (st & rsdev::kStatusListFull)
    return fail(RS_EOVERFLOW, "the certified-binning list overflowed: some rays kept their float32 decision "
                              "(shoot fewer rows per call)");
  return RS_OK;
}

// ------------------------------------------------------------------------------------------------ partition passes
//
// The steps of a lens-partitioned shoot with caller-owned buffers, for partitions held by different
// processes (Section 3.3 across GPUs): the per-ray state, the list of rays to re-evaluate and their
// float-float partial deflections travel between the holders of the partitions by any transport.

int rs_partition_buffer_bytes(const rs_ray_grid* g, int64_t row_begin, int64_t row_end, uint64_t* state_bytes,
                              uint64_t* list_bytes, uint64_t* ff_bytes) {
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if (row_begin < 0 || row_end < row_begin || row_end > g->n[1])
    return fail(RS_EINVAL, "row range [%lld, %lld) outside [0, %lld]", (long long)row_begin, (long long)row_end,
                (long long)g->n[1]);
  const int64_t rows = row_end - row_begin;
  if (g->n[0] > 0 && rows > 0 && (rows > ((int64_t)1 << 32) / g->n[0] || rows * g->n[0] >= ((int64_t)1 << 32)))
    return fail(RS_EOVERFLOW, "a pass covers at most 2^32 - 1 rays");
  const unsigned cap = rsint::recheck_capacity(rows * g->n[0]);
  if (state_bytes) *state_bytes = rsint::staged_state_bytes(rows, g->n[0]);
  if (list_bytes) *list_bytes = 16 + sizeof(uint2) * (uint64_t)cap;
  if (ff_bytes) *ff_bytes = sizeof(float4) * (uint64_t)cap;
  return RS_OK;
}

namespace {

int partition_desc(rs_field_t part, int weighted, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                   const rs_window* w, uint32_t* d_counts, uint64_t* d_oow, bool binning, ShootDesc* d) {
  if (!part) return fail(RS_EINVAL, "partition field is NULL");
  int rc;
  if ((rc = check_grid(g)) != RS_OK) return rc;
  if ((rc = check_window(w)) != RS_OK) return rc;
  if (binning && !d_counts) return fail(RS_EINVAL, "d_counts is NULL");
  if (row_begin < 0 || row_end < row_begin || row_end > g->n[1])
    return fail(RS_EINVAL, "row range [%lld, %lld) outside [0, %lld]", (long long)row_begin, (long long)row_end,
                (long long)g->n[1]);
  if (weighted && !part->dev.mass2)
    return fail(RS_EINVAL, "weighted passes need partitions created with masses (all partitions or none)");
  if (!weighted && part->dev.has_mass)
    return fail(RS_EINVAL, "the partition's masses are not all 1: every pass of the shoot must be weighted");
  if ((rc = check_field_device(part)) != RS_OK) return rc;
  if ((rc = fill_desc(part, g, row_begin, row_end, w, d_counts, d_oow, d)) != RS_OK) return rc;
  d->f.has_mass = weighted ? 1 : 0;
  return RS_OK;
}

}  // namespace

int rs_partition_pass(rs_field_t part, int weighted, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                      const rs_window* w, void* d_state, int first, int last, uint32_t* d_counts,
                      uint64_t* d_out_of_window, void* d_list, void* stream) {
  ShootDesc d;
  int rc;
  if ((rc = partition_desc(part, weighted, g, row_begin, row_end, w, d_counts, d_out_of_window, last != 0, &d)) !=
      RS_OK)
    return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  if (!d_state) return fail(RS_EINVAL, "d_state is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (last && g_certify) {
    if (!d_list) return fail(RS_EINVAL, "d_list is NULL (certified binning is on)");
    d.rc_cap = rsint::recheck_capacity(d.n_rows * d.n0);
    d.rc_count = reinterpret_cast<unsigned int*>(d_list);
    d.rc_list = reinterpret_cast<uint2*>(reinterpret_cast<char*>(d_list) + 16);
    e = cudaMemsetAsync(d.rc_count, 0, sizeof(unsigned int), s);
  }
  if (e == cudaSuccess) e = rsint::launch_staged(d, reinterpret_cast<uint64_t*>(d_state), first != 0, last != 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "partition pass launch");
  return RS_OK;
}

int rs_partition_recheck(rs_field_t part, int weighted, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                         const rs_window* w, const void* d_list, void* d_ff, int first, int last, uint32_t* d_counts,
                         uint64_t* d_out_of_window, void* stream) {
  ShootDesc d;
  int rc;
  if ((rc = partition_desc(part, weighted, g, row_begin, row_end, w, d_counts, d_out_of_window, last != 0, &d)) !=
      RS_OK)
    return rc;
  if (d.n_rows == 0 || d.n0 == 0) return RS_OK;
  if (!d_list || !d_ff) return fail(RS_EINVAL, "d_list / d_ff is NULL");
  const unsigned cap = rsint::recheck_capacity(d.n_rows * d.n0);
  const unsigned* count = reinterpret_cast<const unsigned int*>(d_list);
  const uint2* list = reinterpret_cast<const uint2*>(reinterpret_cast<const char*>(d_list) + 16);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = recheck_grid(part->device);
  cudaError_t e = rsint::launch_recheck_part(d, list, count, cap, reinterpret_cast<float4*>(d_ff), first != 0, grid, s);
  if (e == cudaSuccess && last) e = rsint::launch_recheck_bin(d, list, count, cap, reinterpret_cast<float4*>(d_ff), grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "partition re-evaluation launch");
  return RS_OK;
}

}  // extern "C"
