// C-ABI layer, batches (Section 4's many maps): the LPT-ordered work plan of many fields and its
// CUDA graph (memsets, persistent kernels per launch shape and mass mode, float-float re-evaluation).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rs_host.h"

using rsdev::FieldDev;
using rsdev::ShootDesc;
using namespace rshost;

struct rs_batch {
  int device;
  int n_fields;
  // work items grouped by (launch shape, mass mode): one persistent kernel per group; group
  // g = 2 * cfg + mass (mass 0: unit masses, 1: per-lens masses)
  static constexpr int kGroups = 2 * rsint::kNumCfg;
  int n_items[kGroups];
  int item_offset[kGroups];
  int grid[kGroups];
  ShootDesc* d_descs;
  int2* d_items;
  int* d_counter;
  uint2* d_rc_list;
  unsigned int* d_rc_count;
  unsigned int rc_cap;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" {

// ------------------------------------------------------------------------------------------------ batch

int rs_batch_create_shaped(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids, const rs_window* windows,
                           uint32_t* const* d_counts, uint64_t* d_out_of_window, const int* shapes, rs_batch_t* out) {
  if (!out) return fail(RS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_fields <= 0) return fail(RS_EINVAL, "n_fields must be >= 1");
  if (!fields || !grids || !windows || !d_counts) return fail(RS_EINVAL, "NULL array argument");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int rc;
  std::vector<ShootDesc> descs(n_fields);
  struct Item {
    double cost;
    int field;
    int tile;
  };
  constexpr int G = rs_batch::kGroups;
  std::vector<Item> items[G];
  int64_t n_total = 0;
  for (int k = 0; k < n_fields; ++k) {
    if (!fields[k]) return fail(RS_EINVAL, "fields[%d] is NULL", k);
    if (fields[k]->device != dev) return fail(RS_EINVAL, "fields[%d] lives on another device", k);
    if ((rc = check_grid(&grids[k])) != RS_OK) return rc;
    if ((rc = check_window(&windows[k])) != RS_OK) return rc;
    if (!d_counts[k]) return fail(RS_EINVAL, "d_counts[%d] is NULL", k);
    if ((rc = fill_desc(fields[k], &grids[k], 0, grids[k].n[1], &windows[k], d_counts[k],
                        d_out_of_window ? d_out_of_window + k : nullptr, &descs[k])) != RS_OK)
      return rc;
    const int mass = fields[k]->dev.has_mass ? 1 : 0;
    int cfg = g_cfg[mass];
    if (shapes) {
      const int* sh = shapes + 4 * k;
      cfg = rsint::find_cfg(sh[0], sh[1], sh[2], sh[3]);
      if (cfg < 0)
        return fail(RS_EINVAL, "shapes[%d] = (%d, %d, %d, %d) is not a compiled launch shape", k, sh[0], sh[1], sh[2],
                    sh[3]);
    }
    cfg = rsint::batch_cfg(cfg);
    const int grp = 2 * cfg + mass;
    const int warps = rsint::kCfgs[cfg].block / 32;
    const int64_t seg = 32 * (int64_t)rsint::kCfgs[cfg].rpt;
    const int64_t n0 = descs[k].n0, nr = descs[k].n_rows;
    if (n0 == 0 || nr == 0) continue;
    const int64_t ncol = (n0 + seg - 1) / seg;
    const int64_t nt = ((nr + warps - 1) / warps) * ncol;
    if (n_total + nt >= ((int64_t)1 << 31)) return fail(RS_EOVERFLOW, "too many work items");
    n_total += nt;
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t trow = t / ncol, tcol = t - trow * ncol;
      const int64_t rows = std::min<int64_t>(warps, nr - trow * warps);
      const int64_t cols = std::min<int64_t>(seg, n0 - tcol * seg);
      // per-ray cost: one interaction per lens plus a fixed epilogue (~ 64 interactions)
      const double cost = (double)(rows * cols) * ((double)fields[k]->n_lens + 64.0);
      items[grp].push_back({cost, k, (int)t});
    }
  }
  std::vector<int2> h_items;
  rs_batch* b = new (std::nothrow) rs_batch();
  if (!b) return fail(RS_ENOMEM, "host allocation failed");
  b->device = dev;
  b->n_fields = n_fields;
  for (int grp = 0; grp < G; ++grp) {
    std::stable_sort(items[grp].begin(), items[grp].end(),
                     [](const Item& x, const Item& y) { return x.cost > y.cost; });
    b->item_offset[grp] = (int)h_items.size();
    b->n_items[grp] = (int)items[grp].size();
    for (const Item& it : items[grp]) h_items.push_back(make_int2(it.field, it.tile));
    b->grid[grp] = 0;
    if (b->n_items[grp] == 0) continue;
    int bps = 0;
    if (rsint::batch_blocks_per_sm(grp / 2, (grp & 1) == 1, &bps) != cudaSuccess || bps < 1) bps = 1;
    b->grid[grp] = num_sms(dev) * bps;
  }
  auto cleanup = [&]() {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_descs);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_rc_list);
    cudaFree(b->d_rc_count);
    delete b;
  };
  if (g_certify) {
    int64_t total = 0;
    for (int k = 0; k < n_fields; ++k) total += descs[k].n_rows * descs[k].n0;
    b->rc_cap = rsint::recheck_capacity(total);
  }
  if ((e = dev_alloc(&b->d_descs, sizeof(ShootDesc) * n_fields)) != cudaSuccess ||
      (e = dev_alloc(&b->d_items, sizeof(int2) * std::max<size_t>(1, h_items.size()))) != cudaSuccess ||
      (e = dev_alloc(&b->d_counter, G * sizeof(int))) != cudaSuccess ||
      (b->rc_cap > 0 && (e = dev_alloc(&b->d_rc_list, sizeof(uint2) * (size_t)b->rc_cap)) != cudaSuccess) ||
      (b->rc_cap > 0 && (e = dev_alloc(&b->d_rc_count, sizeof(unsigned int))) != cudaSuccess)) {
    rc = cuda_fail(e, "cudaMalloc (batch)");
    cleanup();
    return rc;
  }
  for (int k = 0; k < n_fields; ++k) {
    descs[k].field_id = k;
    descs[k].rc_list = b->d_rc_list;
    descs[k].rc_count = b->d_rc_count;
    descs[k].rc_cap = b->rc_cap;
  }
  if ((e = cudaMemcpy(b->d_descs, descs.data(), sizeof(ShootDesc) * n_fields, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!h_items.empty() &&
       (e = cudaMemcpy(b->d_items, h_items.data(), sizeof(int2) * h_items.size(), cudaMemcpyHostToDevice)) != cudaSuccess)) {
    rc = cuda_fail(e, "cudaMemcpy (batch descriptors)");
    cleanup();
    return rc;
  }
  // Capture: zero every map and counter, then the persistent kernel.
  cudaStream_t cs;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
    rc = cuda_fail(e, "cudaStreamCreate");
    cleanup();
    return rc;
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < n_fields && e == cudaSuccess; ++k)
      e = cudaMemsetAsync(d_counts[k], 0, sizeof(uint32_t) * (size_t)windows[k].npix[0] * (size_t)windows[k].npix[1], cs);
    if (e == cudaSuccess && d_out_of_window) e = cudaMemsetAsync(d_out_of_window, 0, sizeof(uint64_t) * n_fields, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, G * sizeof(int), cs);
    if (e == cudaSuccess && b->rc_cap > 0) e = cudaMemsetAsync(b->d_rc_count, 0, sizeof(unsigned int), cs);
    // groups in decreasing order of their largest item (each group's items are already LPT-ordered)
    std::vector<int> order;
    for (int grp = 0; grp < G; ++grp)
      if (b->n_items[grp] > 0) order.push_back(grp);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return items[x][0].cost > items[y][0].cost; });
    for (size_t i = 0; i < order.size() && e == cudaSuccess; ++i) {
      const int grp = order[i];
      e = rsint::launch_batch(grp / 2, (grp & 1) == 1, b->d_descs, b->d_items + b->item_offset[grp], b->n_items[grp],
                              b->d_counter + grp, b->grid[grp], cs);
    }
    if (e == cudaSuccess && b->rc_cap > 0)
      e = rsint::launch_recheck(nullptr, b->d_descs, b->d_rc_list, b->d_rc_count, b->rc_cap, recheck_grid(dev), cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "batch graph capture");
    cleanup();
    return rc;
  }
  *out = b;
  return RS_OK;
}

int rs_batch_create(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids, const rs_window* windows,
                    uint32_t* const* d_counts, uint64_t* d_out_of_window, rs_batch_t* out) {
  return rs_batch_create_shaped(n_fields, fields, grids, windows, d_counts, d_out_of_window, nullptr, out);
}

int rs_batch_launch(rs_batch_t b, void* stream) {
  if (!b) return fail(RS_EINVAL, "batch is NULL");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) return fail(RS_EINVAL, "batch lives on device %d but device %d is current", b->device, cur);
  cudaError_t e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return RS_OK;
}

int rs_batch_destroy(rs_batch_t b) {
  if (!b) return RS_OK;
  DeviceGuard g(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_descs);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_rc_list);
  cudaFree(b->d_rc_count);
  delete b;
  return RS_OK;
}

int rs_shoot_batch(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids, const rs_window* windows,
                   uint32_t* const* d_counts, uint64_t* d_out_of_window, void* stream) {
  rs_batch_t b = nullptr;
  int rc = rs_batch_create(n_fields, fields, grids, windows, d_counts, d_out_of_window, &b);
  if (rc != RS_OK) return rc;
  rc = rs_batch_launch(b, stream);
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  rs_batch_destroy(b);
  if (rc != RS_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (batch)");
  return RS_OK;
}

}  // extern "C"
