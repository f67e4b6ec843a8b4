/*
 * rs.h -- C ABI of the GB300 inverse ray-shooting library (librs.so).
 *
 * Method: Thompson, Fluke, Barnes & Barsdell (2009), "Teraflop per second
 * gravitational lensing ray-shooting using graphics processing units".
 * For every ray x of a regular image-plane grid the library sums the
 * many-Schwarzschild deflection directly over all lenses (Eq. 2),
 *     alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2,
 * maps the ray to the source plane with the macro-model lens equation (Eq. 6),
 *     y1 = (1 - kappa_c - gamma) x1 - alpha1,   y2 = (1 - kappa_c + gamma) x2 - alpha2,
 * and counts rays per source pixel; the normalised counts are the
 * magnification map mu_ij = N_ij / N_av (Eq. 4).
 *
 * Conventions shared by every entry point
 *   - Return value: RS_OK (0) or one of the RS_E* codes below.  Nothing is
 *     thrown across the ABI.  rs_last_error() returns a message for the last
 *     nonzero status of the calling thread.
 *   - Pointers named d_* are CUDA device pointers on the current device.
 *     Pointers named h_* or without prefix are host pointers, unless a flag
 *     says otherwise.  No entry point frees memory it did not allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on it; host inputs are
 *     fully consumed (copied) before the call returns.
 *   - All kernels run on the device that is current when the call is made;
 *     a field must be used on the device it was created on.
 *   - Coordinates are in Einstein radii of a unit mass (the units of Eq. 2).
 *     Lens and ray coordinates must be finite with |value| <= 1e9 (squared
 *     distances and their pairwise products then stay within float32 range).
 *
 * Numerics (what the device computes)
 *   - Ray (i, j) sits at x_k = (float) fma(index_k, spacing_k, origin_k): the
 *     double fma rounded to float is the ray position.
 *   - Per lens-ray pair: float32 arithmetic with the hardware approximate
 *     reciprocal.  Lenses are taken in consecutive pairs; for a fixed subset of
 *     the pairs (three of every four with unit masses, every other pair with
 *     per-lens masses) one reciprocal of the product of the two squared
 *     distances serves both lenses (Montgomery's simultaneous inversion).
 *     Per ray, partial sums over consecutive groups of 64 lenses (in lens index
 *     order) are folded into a two-float (hi, lo) accumulator with an
 *     error-free TwoSum; (hi, lo) is renormalised after every 256 lenses.  With
 *     alpha = hi + lo, Eq. 6 and the pixel coordinate u are evaluated in
 *     float-float arithmetic (~2^-44 relative; rs_trace reports y in float64).
 *   - The per-ray arithmetic does not depend on launch configuration, so
 *     counts are bitwise reproducible and equal between rs_shoot,
 *     rs_shoot_rows sharding, and the batched path.
 *   - Binning (the definition, float64): u_k = (y_k - lo_k) * (npix_k / (hi_k - lo_k));
 *     a ray is in the window iff 0 <= u_k < npix_k on both axes (NaN fails),
 *     pixel p_k = floor(u_k).  With certified binning (below) the counts follow
 *     this definition applied to the exact deflection (within the scope stated there).  Counts are uint32, row-major [p2][p1].  A ray that
 *     hits a lens exactly has a non-finite deflection and is out of window.
 */
#ifndef RS_H
#define RS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define RS_OK 0
#define RS_EINVAL 1     /* invalid argument (NULL pointer, size, non-finite parameter, ...)   */
#define RS_ENOMEM 2     /* device or host allocation failed                                  */
#define RS_ECUDA 3      /* a CUDA runtime call failed (message has the CUDA error string)   */
#define RS_EOVERFLOW 4  /* a size exceeds a documented limit (e.g. >= 2^32 rays per call)   */
#define RS_ETIMEOUT 5   /* a device-side bounded wait gave up (see rs_field_status)         */

/* Opaque lens field: owns device copies of the lens arrays and the macro-model. */
typedef struct rs_field* rs_field_t;

/* Regular image-plane ray grid: ray (i, j), 0 <= i < n[0], 0 <= j < n[1], at
 * x = ((float)fma(i, spacing[0], origin[0]), (float)fma(j, spacing[1], origin[1])).
 * spacing > 0, all values finite, n >= 0. */
typedef struct {
  double origin[2];
  double spacing[2];
  int64_t n[2];
} rs_ray_grid;

/* Source-plane window: half-open [lo, hi) per axis split into npix pixels; hi > lo, 1 <= npix <= 2^22. */
typedef struct {
  double lo[2];
  double hi[2];
  int32_t npix[2];
} rs_window;

/*
 * rs_create_field -- upload a lens realisation (Eq. 2 lenses, Eq. 6 macro-model).
 *   lens_xy  : float[2*n_lens], interleaved (x1, x2) per lens.  May be NULL if n_lens == 0.
 *   masses   : float[n_lens] (finite, >= 0), or NULL for unit masses.  With NULL the
 *              equal-mass kernels are used (no mass is stored or read, Section 3.2).  Masses
 *              that are all exactly 1 also select the equal-mass kernels; they are still stored
 *              (the field may then be a lens partition next to weighted ones).  With device
 *              inputs that test is a reduction read back before the call returns.
 *   n_lens   : >= 0 and < 2^31.  n_lens == 0 gives the undeflected (macro-only) map.
 *   kappa_c  : smooth convergence sigma_c of Eq. 6; gamma: external shear (finite).
 *   inputs_on_device : 0 = lens_xy/masses are host pointers, 1 = device pointers.
 *   stream   : stream for the upload and repacking kernels.
 *   out      : receives the new field.  The field keeps its own copies; the
 *              inputs may be freed once the call returns (host) or once the
 *              stream has passed this point (device inputs).
 * Errors: RS_EINVAL (bad argument), RS_ENOMEM, RS_ECUDA.
 */
int rs_create_field(const float* lens_xy, const float* masses, int64_t n_lens, double kappa_c,
                    double gamma, int inputs_on_device, void* stream, rs_field_t* out);

/* rs_destroy_field -- release a field (synchronises its device first).  NULL is a no-op.
 * RS_EINVAL (nothing released) while lens-range views of the field are alive. */
int rs_destroy_field(rs_field_t f);

/*
 * rs_create_field_view -- a field made of lenses [lens_begin, lens_begin + n_lens) of `parent`,
 * reading the parent's device arrays (no copy; the view owns only its status word).  Uses: the
 * deflection of a subset of the lenses (Eq. 2 is a sum, so views of disjoint ranges superpose),
 * resident lens partitions for rs_shoot_staged, and short proxy runs on a prefix of a very large
 * field (the autotuner).  lens_begin must be a multiple of 256 (lens tiles and the summation
 * schedule start there, so views cut at multiples of 256 give rs_shoot_staged the parent's results
 * bit for bit).  The view takes the parent's kappa_c, gamma and mass mode, and sees the parent's
 * current lens positions (a view of a moving field moves with it; rs_field_set_time applies to
 * the parent only).  The parent cannot be destroyed while views are alive.  0 <= n_lens,
 * lens_begin + n_lens <= the parent's lens count.  Errors: RS_EINVAL, RS_ENOMEM, RS_ECUDA.
 */
int rs_create_field_view(rs_field_t parent, int64_t lens_begin, int64_t n_lens, rs_field_t* out);

/*
 * Moving lenses (Section 4: the stars move, so the caustic network and the map change with time;
 * one map per time step).  rs_create_moving_field -- as rs_create_field, plus vel_xy (float[2*n_lens],
 * interleaved (v1, v2) per lens, finite; host or device as inputs_on_device) in coordinate units per
 * unit time.  The field keeps positions and velocities at t = 0 on the device (16 extra bytes per
 * lens) and starts at t = 0.  Synchronous.
 * rs_field_set_time -- move the field's lenses to time t, in place and stream-ordered:
 *   x_i(t) = (float)((double)x_i + (double)v_i * t) per axis (product, then sum, no fused multiply-add).
 *   Work already enqueued on `stream` sees the old positions, work enqueued after it the new ones;
 *   work on other streams must be ordered by the caller.  Batches that include the field read its
 *   lenses at launch, so a planned batch of moving fields can be replayed after each time step.
 *   Errors: RS_EINVAL (not a moving field, t not finite, or |x| + |v| |t| beyond 1e9).
 * rs_field_time -- the field's current time (a lens-range view: its parent's).
 */
int rs_create_moving_field(const float* lens_xy, const float* vel_xy, const float* masses, int64_t n_lens,
                           double kappa_c, double gamma, int inputs_on_device, void* stream, rs_field_t* out);
int rs_field_set_time(rs_field_t f, double t, void* stream);
int rs_field_time(rs_field_t f, double* t);

/* Number of lenses, and whether the field's kernels weigh lenses by their masses (1: masses given
 * and not all exactly 1) or take unit masses (0).  The launch shape of rs_set_launch_config's mass
 * mode has_masses applies to the field. */
int rs_field_info(rs_field_t f, int64_t* n_lens, int* has_masses);

/*
 * rs_shoot -- shoot every ray of grid g through field f and ACCUMULATE (+=) the
 * binned counts into d_counts (uint32[npix[1]][npix[0]], device) and the number
 * of rays that miss the window into *d_out_of_window (uint64, device; may be NULL).
 * The caller zeroes the buffers before the first call.  Method: Eq. 2 and Eq. 6
 * per ray, binning as in the header comment, counts for Eq. 4.
 * Errors: RS_EINVAL, RS_EOVERFLOW (n[0]*n[1] >= 2^32), RS_ECUDA (launch failure).
 */
int rs_shoot(rs_field_t f, const rs_ray_grid* g, const rs_window* w, uint32_t* d_counts,
             uint64_t* d_out_of_window, void* stream);

/*
 * rs_shoot_rows -- as rs_shoot for grid rows j in [row_begin, row_end) only.
 * Shooting a partition of the rows into the same buffers gives exactly the
 * counts of one rs_shoot (ray positions depend only on (i, j)): the basis for
 * sharding a map over calls, devices or restarts (checkpoint = counts + next row).
 */
int rs_shoot_rows(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                  const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream);

/*
 * rs_shoot_culled -- rs_shoot_rows that skips rays which provably miss the window: the interactive
 * zoom of Section 4 (a sub-window re-shot at higher resolution only needs the rays that can land
 * in it).  Rays are grouped in cells of 16 x 16; for a cell with ray-box centre c and circumradius
 * rho, the deflection of every ray differs from alpha(c) by at most rho sum_i m_i / (d_i (d_i - rho))
 * (d_i = |c - x_i|), so the cell's source positions lie in a box around lam x - alpha(c); a cell
 * whose box (widened by the float32 error band of its rays and float64 rounding) misses the window
 * is skipped and its rays are counted out of window.  Cells with a lens within 1.02 rho of c are
 * always shot.  Results: the same counts and out-of-window count as rs_shoot_rows, bit for bit (the
 * shot cells use the same per-ray arithmetic and binning, certified binning included).
 *   d_rays_shot : uint64 device counter or NULL; ACCUMULATES the number of rays actually shot.
 * Other arguments, accumulation and errors as rs_shoot_rows.  Workspace is allocated
 * stream-ordered (4 bytes per cell plus the re-evaluation list).
 */
int rs_shoot_culled(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end, const rs_window* w,
                    uint32_t* d_counts, uint64_t* d_out_of_window, uint64_t* d_rays_shot, void* stream);

/*
 * rs_shoot_staged -- rs_shoot_rows for a field given as n_parts lens partitions (Section 3.3's
 * billion-lens scheme: the deflection of every ray is summed one partition at a time, the
 * partially deflected rays carried in device memory between the passes, and the rays are mapped
 * and binned after the last partition).  For fields of 2^31 lenses or more, or lenses held as
 * shards.  The lens order is partition 0's lenses, then partition 1's, ...; every partition but
 * the last must hold a multiple of 256 lenses, and all share device, kappa_c, gamma and whether
 * masses were given (masses given to all or to none; if any partition's masses are not all 1, every
 * partition runs the weighted kernels).
 * The carried state is the shoot kernel's own accumulator set (28 bytes per ray, stream-ordered
 * allocation; rays are processed in row blocks of at most 2 GiB of state), so the float32
 * deflections, error bands and counts equal those of one rs_shoot_rows over a single field
 * holding all the lenses, bit for bit; with certified binning on, the listed rays are
 * re-evaluated in float-float partition by partition (same guarantee as rs_shoot_rows).
 * Other arguments, accumulation and errors as rs_shoot_rows.
 */
int rs_shoot_staged(int n_parts, const rs_field_t* parts, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                    const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream);

/*
 * rs_shoot_streamed -- rs_shoot_staged for lenses held in HOST memory (out-of-core: more lenses than
 * fit the device, or than one field may hold).  The lenses (h_lens_xy: float[2*n_lens] interleaved,
 * h_masses: float[n_lens] or NULL for unit masses -- masses all exactly 1 count as unit masses and
 * are not uploaded --, n_lens may exceed 2^31) stream through the device
 * in passes of lenses_per_pass lenses (a multiple of 1024, at most 2^30) via two pinned staging
 * buffers and two device buffers: the host copy and upload of the next partition overlap the pass
 * over the current one on the GPU.  With certified binning on, a second sweep streams the lenses
 * again for the float-float re-evaluation of the listed rays.  Results as rs_shoot_staged (bit for
 * bit those of one pass over all lenses).  Synchronous: returns when the counts are complete.
 * Device memory: 72 bytes per lens of a pass plus the ray state.  Errors: as rs_shoot_rows, and
 * RS_ETIMEOUT if a bounded wait for a lens tile gave up.
 */
int rs_shoot_streamed(const float* h_lens_xy, const float* h_masses, int64_t n_lens, double kappa_c, double gamma,
                      int64_t lenses_per_pass, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                      const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream);

/* Device memory budget (bytes, >= 1 MiB; default 2 GiB) for the carried per-ray state of
 * rs_shoot_staged: calls whose state would exceed it run in row blocks (same results). */
int rs_set_staged_state_budget(uint64_t bytes);  /* also used by rs_shoot_streamed */

/*
 * Partition passes -- the steps of rs_shoot_staged with caller-owned buffers, for lens partitions held
 * by different processes or GPUs (Section 3.3's pipeline of partially deflected rays from GPU to GPU).
 * For rows [row_begin, row_end) of grid g, the holder of partition p calls rs_partition_pass with the
 * ray block's state buffer, after the holder of partition p - 1 (first = 1 for p = 0: the state starts
 * from zero); any transport (e.g. NCCL send/recv of the buffer) carries the state between them.  The
 * last partition's pass (last = 1) maps and bins the rays into d_counts / d_out_of_window (accumulated)
 * instead of storing the state; with certified binning on it lists the rays to re-evaluate in d_list.
 * Those rays then go around the partitions once more: every holder calls rs_partition_recheck with the
 * list (a copy of the last holder's) and the float-float buffer d_ff in the same order (first = 1 for
 * partition 0), and the last call (last = 1) bins them.  With the same partitions, the counts equal those
 * of rs_shoot_staged bit for bit.  Partitions as rs_shoot_staged (multiples of 256 lenses but the last;
 * masses given to all or to none); weighted = 1 runs every pass with per-lens masses (required when any
 * partition's masses are not all 1; every pass and re-evaluation of a shoot must use the same value).
 *   rs_partition_buffer_bytes: device bytes of the state (28 per ray, padded to CTA tiles), of the list
 *     (16 + 8 per entry; capacity max(4096, rays/32)) and of d_ff (16 per entry) for the row block.
 * Calls are asynchronous on `stream`; buffers are caller-owned device memory.
 */
int rs_partition_buffer_bytes(const rs_ray_grid* g, int64_t row_begin, int64_t row_end, uint64_t* state_bytes,
                              uint64_t* list_bytes, uint64_t* ff_bytes);
int rs_partition_pass(rs_field_t part, int weighted, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                      const rs_window* w, void* d_state, int first, int last, uint32_t* d_counts,
                      uint64_t* d_out_of_window, void* d_list, void* stream);
int rs_partition_recheck(rs_field_t part, int weighted, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                         const rs_window* w, const void* d_list, void* d_ff, int first, int last, uint32_t* d_counts,
                         uint64_t* d_out_of_window, void* stream);

/*
 * rs_trace -- source positions of listed rays through the float32 path, for checks.
 *   d_ray_ij : int64[2*k] device, (i, j) per ray (each within the grid).
 *   d_y      : double[2*k] device, receives (y1, y2) per ray (Eq. 6).
 *   d_alpha  : double[2*k] device or NULL, receives (alpha1, alpha2) per ray (Eq. 2).
 *   d_err    : double[2*k] device or NULL, receives per axis the half-width of the band
 *              around y inside which the float32 result cannot decide a pixel (see
 *              certified binning below); asking for it costs one more pass over the lenses.
 * The per-ray arithmetic is the one rs_shoot uses, bit for bit (the band included).
 */
int rs_trace(rs_field_t f, const rs_ray_grid* g, const int64_t* d_ray_ij, int64_t k, double* d_y,
             double* d_alpha, double* d_err, void* stream);

/*
 * rs_trace_certified -- source positions of listed rays with the deflection (Eq. 2) summed in
 * float-float arithmetic (~2^-44 relative per term): the evaluation certified binning uses.
 * Arguments as rs_trace (no d_err).
 */
int rs_trace_certified(rs_field_t f, const rs_ray_grid* g, const int64_t* d_ray_ij, int64_t k,
                       double* d_y, double* d_alpha, void* stream);

/*
 * Certified binning (on by default).  The float32 shoot attaches to every ray an error band:
 * 10 u sqrt(64 sum_g (P1_g^2 + P2_g^2)) + 2 u sum_g (|P1_g| + |P2_g|) + 16 u T (u = 2^-24, P_g the
 * float32 partial sums of its 64-lens groups): the random rounding, coherent errors (the far field
 * sees the ray's coordinate only to the precision of the lens-ray difference; a bias of the
 * approximate reciprocal), and the rounding of the largest single terms, which a group partial
 * hides where near lenses' terms cancel inside it: T = max(m_max, max m_i / r_i over the lenses
 * within r_i <= 1 of the ray), m_max the field's largest mass.  A ray whose source position lies
 * within that band of a pixel or window edge is not binned by the float32 result but re-evaluated
 * with rs_trace_certified's arithmetic and binned from that; the maps then agree with a float64
 * evaluation except for rays within ~1e-12 of an edge and rays whose float32 error exceeds the
 * band.  The band is an estimate of the error, not a rigorous bound (that bound, 72 u sum_i m_i / r_i,
 * would need a square root per lens and ray); the tests check that it covers the float32 error of
 * every ray traced on fields of 1 to 1e8 lenses, few-lens fields included, and that certified maps
 * of such fields equal the oracle's bit for bit.
 * rs_shoot allocates the list of such rays stream-ordered (cudaMallocAsync,
 * capacity max(4096, rays/32), at most 2^24 entries); rays beyond the capacity keep their
 * float32 decision and the field's status records RS_EOVERFLOW (rs_field_status).  Batches own their list.
 * rs_set_certified_binning(0) turns it off for calls (and batches planned) afterwards.
 */
int rs_set_certified_binning(int enabled);
int rs_get_certified_binning(int* enabled);

/*
 * rs_magnification -- Eq. 4: d_mu[p] = d_counts[p] / N_av (float, device), with
 * N_av = ((hi0-lo0)/npix0 * (hi1-lo1)/npix1) / (spacing0 * spacing1), the number
 * of rays a pixel receives without lensing.
 */
int rs_magnification(const uint32_t* d_counts, const rs_ray_grid* g, const rs_window* w, float* d_mu,
                     void* stream);

/*
 * Batched shooting of many independent fields in one persistent launch
 * (many realisations for a statistical light-curve study, Section 4).
 *
 * rs_batch_create -- plan a batch.  fields/grids/windows: host arrays of
 *   n_fields entries; d_counts: host array of n_fields device pointers (each
 *   uint32[npix1][npix0]); d_out_of_window: device uint64[n_fields] or NULL.
 *   The plan copies all descriptors to the device, orders the work items
 *   (field, ray tile) by decreasing cost, and captures one CUDA graph that
 *   zeroes the counts and the work counter and runs the persistent kernel.
 *   The fields must outlive the plan.  Unlike rs_shoot, the graph ZEROES the
 *   counts and out-of-window counters on every launch.
 * rs_batch_create_shaped -- as rs_batch_create with a launch shape per field: shapes = host int[4 *
 *   n_fields] of (block, rays per thread, lens tile, min_ctas) from rs_launch_configs (NULL: every field
 *   takes its mass mode's rs_set_launch_config shape).  The items of each (shape, mass mode) form one
 *   persistent launch of the graph; the counts are the same bits for every choice.  A shape compiled
 *   for three CTAs per SM runs in a batch as the shape with the same block, rays per thread and lens
 *   tile compiled for two (in that shape's launch).
 * rs_batch_launch -- replay the plan's graph on `stream`.
 * rs_batch_destroy -- release the plan (synchronises first).  NULL is a no-op.
 * rs_shoot_batch -- create + launch + destroy in one call (synchronous).
 */
typedef struct rs_batch* rs_batch_t;

int rs_batch_create(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids,
                    const rs_window* windows, uint32_t* const* d_counts, uint64_t* d_out_of_window,
                    rs_batch_t* out);
int rs_batch_create_shaped(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids,
                           const rs_window* windows, uint32_t* const* d_counts, uint64_t* d_out_of_window,
                           const int* shapes, rs_batch_t* out);
int rs_batch_launch(rs_batch_t b, void* stream);
int rs_batch_destroy(rs_batch_t b);
int rs_shoot_batch(int n_fields, const rs_field_t* fields, const rs_ray_grid* grids,
                   const rs_window* windows, uint32_t* const* d_counts, uint64_t* d_out_of_window,
                   void* stream);

/*
 * rs_field_status -- synchronise the field's device and report what kernels that used it
 * recorded: *status = RS_ETIMEOUT if a bounded wait gave up; else RS_EOVERFLOW if the list of
 * rays to re-evaluate (certified binning) of some call was full, so that some rays kept their
 * float32 decision (shoot fewer rows per call); else RS_OK.  For staged shoots the last
 * partition's field records the list state.  clear != 0 resets the flags.
 */
int rs_field_status(rs_field_t f, int clear, int* status);

/*
 * Launch shapes.  The library carries kernels for several (threads per CTA,
 * rays per thread, lenses per shared-memory stage, resident CTAs per SM the
 * kernel is compiled for) shapes (Section 2.2's choice of threads per block,
 * widened); all compute bitwise identical results (the lens tile is a multiple
 * of the 256-lens summation period), so the choice only affects speed.
 * rs_set_launch_config selects the shape used by rs_shoot / rs_shoot_rows /
 * rs_shoot_rows_noalloc (and by batches planned afterwards) for fields without
 * (has_masses = 0) or with per-lens masses; RS_EINVAL for a shape that is not
 * compiled.  rs_launch_configs lists the compiled shapes: up to `cap`
 * (block, rpt, lens_tile, min_ctas) quadruples into `shapes` (int[4*cap]);
 * returns the number available via *count.  rs_launch_occupancy reports how
 * many CTAs of a shape's shoot kernel are resident per SM on the current device
 * (SMs x that = one wave of CTAs).
 */
int rs_set_launch_config(int has_masses, int block, int rays_per_thread, int lens_tile, int min_ctas);
int rs_get_launch_config(int has_masses, int* block, int* rays_per_thread, int* lens_tile, int* min_ctas);
int rs_launch_configs(int* shapes, int cap, int* count);
int rs_launch_occupancy(int has_masses, int block, int rays_per_thread, int lens_tile, int min_ctas,
                        int* ctas_per_sm);

/*
 * Light curves (Section 1: a source of finite size moves across the magnification map; the
 * magnification it sees along its path, as a magnitude change, is the light curve that is
 * compared with observations).  The paper states no formula; this library computes, for each
 * sample position y of a straight track, the profile-weighted mean of the map
 *     mu(y) = sum_p w(|c_p - y|) mu_p / sum_p w(|c_p - y|),   dm(y) = -2.5 log10 mu(y),
 * over the pixels p of the map with centres c_p = (lo_k + (i_k + 0.5) pix_k)_k, pix_k = (hi_k - lo_k) / npix_k:
 *   RS_PROFILE_GAUSSIAN: w = exp(-d^2 / (2 s^2)) for d^2 <= (6 s)^2, else 0 (s = standard deviation);
 *   RS_PROFILE_DISC:     w = 1 for d^2 <= s^2, else 0 (s = radius).
 * A sample whose profile covers no pixel gives NaN; a zero mean gives dm = +inf.
 *
 * rs_track: samples y_k = y0 + k * step, k = 0 .. n-1, over map number `map` of the call.
 */
#define RS_PROFILE_GAUSSIAN 0
#define RS_PROFILE_DISC 1

typedef struct {
  int32_t map;     /* index into the call's maps, 0 <= map < n_maps                       */
  int32_t reserved;
  double y0[2];    /* first sample (finite, |y| <= 1e9)                                    */
  double step[2];  /* sample spacing (finite; the last sample must also satisfy |y| <= 1e9) */
  int64_t n;       /* number of samples, >= 0                                              */
} rs_track;

/*
 * rs_light_curves -- light curves of many tracks over many maps in one launch (the batched maps
 * of rs_batch_create feed it directly).
 *   n_maps   : >= 1 when any track has samples.
 *   d_mu     : host array of n_maps device pointers, map m = float[npix1][npix0] (row-major
 *              [p2][p1], e.g. the output of rs_magnification).  Read only.
 *   windows  : host array of n_maps source-plane windows, one per map.  Per axis npix <= 2^24
 *              and max(|lo|, |hi|) / pix <= 2^30.
 *   profile, s : RS_PROFILE_GAUSSIAN or RS_PROFILE_DISC and its size (finite, > 0; the profile's
 *              support may span at most 2^20 pixels from its centre along either axis).
 *   tracks   : host array of n_tracks tracks.  Track t's samples are written at consecutive
 *              positions starting at sum_{u < t} tracks[u].n.
 *   d_mu_out : double[sum n] device, receives mu(y_k).
 *   d_dm_out : double[sum n] device or NULL, receives dm(y_k).
 * Numerics: a pixel belongs to the profile exactly when the float64 test
 * ((lo + (i + 0.5) pix) - y)^2 summed over both axes (no fused multiply-add) <= the cut says
 * so; the kernel decides from a float32 estimate and repeats the float64 test for pixels within
 * a guard band of the cut, so the set of pixels is that of a float64 evaluation.  Weights are
 * float32 (expf of the float32 exponent), sums are compensated float32 pairs; mu(y) carries a
 * relative error of a few 1e-7 (rows of the support are summed in float32, at most 2 R / pix + 3
 * terms each, then folded into compensated pairs).  The descriptor table is allocated stream-ordered
 * (cudaMallocAsync) and freed on the stream.
 * Errors: RS_EINVAL (argument), RS_EOVERFLOW (more than 2^40 samples), RS_ENOMEM, RS_ECUDA.
 */
int rs_light_curves(int n_maps, const float* const* d_mu, const rs_window* windows, int profile, double s,
                    int n_tracks, const rs_track* tracks, double* d_mu_out, double* d_dm_out, void* stream);

/*
 * Light-curve plans: the same computation with the track table validated and uploaded once, for
 * repeated launches over the same map buffers (maps refreshed in place, e.g. by a batch) and for
 * CUDA-graph capture (a launch allocates nothing).
 * rs_light_curve_plan_create -- arguments as rs_light_curves; the map pointers are stored and read
 *   at every launch, so the maps must outlive the plan.  Synchronous upload; the current device.
 * rs_light_curve_plan_samples -- total number of samples (length of the outputs).
 * rs_light_curve_plan_launch -- enqueue the light-curve kernel on `stream`.
 * rs_light_curve_plan_destroy -- synchronise the plan's device and release it.  NULL is a no-op.
 */
typedef struct rs_lc_plan* rs_lc_plan_t;

int rs_light_curve_plan_create(int n_maps, const float* const* d_mu, const rs_window* windows, int profile,
                               double s, int n_tracks, const rs_track* tracks, rs_lc_plan_t* out);
int rs_light_curve_plan_samples(rs_lc_plan_t p, int64_t* n_samples);
int rs_light_curve_plan_launch(rs_lc_plan_t p, double* d_mu_out, double* d_dm_out, void* stream);
int rs_light_curve_plan_destroy(rs_lc_plan_t p);

/*
 * rs_shoot_rows_noalloc -- rs_shoot_rows with certified binning, allocating nothing.
 * The paper has no counterpart: this entry point serves callers that cannot allocate device
 * memory while they run (work replayed in a CUDA graph whose capture must not contain
 * allocation nodes; applications whose allocator reserved the device memory at start-up;
 * latency-critical loops that cannot wait on an allocator).
 * Identical results to rs_shoot_rows with certified binning on (the global switch
 * rs_set_certified_binning does not apply: this variant always certifies).  Its list of rays to
 * re-evaluate lives in a static device array of 2^19 entries (4 MiB + 256 B, resident on every
 * device that loads the library until the process exits) instead of a per-call allocation:
 *   - at most 2^24 rays per call (one list entry per 32 rays); larger row ranges return
 *     RS_EOVERFLOW without launching anything -- split them over several calls;
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current), and so does the first call after the device's context changed
 *     (a device reset loads the library's device code anew); make such a first call before any
 *     stream capture;
 *   - every call shares the array and the array keeps the last call's contents; each call
 *     clears the entry counter on its stream.  Calls that overlap on the GPU (different
 *     streams, or different host threads, without ordering between them) race on the array:
 *     order them on one stream or with events.
 * Arguments and accumulation semantics as rs_shoot_rows.
 */
int rs_shoot_rows_noalloc(rs_field_t f, const rs_ray_grid* g, int64_t row_begin, int64_t row_end,
                          const rs_window* w, uint32_t* d_counts, uint64_t* d_out_of_window, void* stream);

/*
 * rs_selftest_bounded_wait -- run one CTA that waits on an mbarrier phase nothing completes,
 * bounded by limit_ns (0 .. 2e9) of the device's global timer, the same bounded wait the
 * kernels use for lens-tile copies.  *status = RS_ETIMEOUT when the wait gave up (the expected
 * outcome), RS_OK otherwise.  Synchronous.  No paper counterpart: failure-detection support.
 */
int rs_selftest_bounded_wait(int64_t limit_ns, int* status);

/*
 * rs_set_alloc_failure -- allocation-failure injection (failure-detection support; no paper
 * counterpart).  n >= 0: the n-th following device or pinned-host allocation made by the library
 * (0: the next one, counted across threads) reports an out-of-memory error instead of allocating,
 * once; n = -1 disarms.  The failing call returns RS_ENOMEM after releasing what it had allocated.
 */
int rs_set_alloc_failure(int64_t n);

/* Thread-local message for the last nonzero status returned on this thread. */
const char* rs_last_error(void);

/* Library version string. */
const char* rs_version(void);

/*
 * rs_device_code_version -- the compute capability the library's device code was built for, as
 * the CUDA runtime reports it for one of its kernels (cudaFuncAttributes::binaryVersion: 103 for
 * sm_103a).  Needs a device; RS_ECUDA when the code cannot run on the current one.
 */
int rs_device_code_version(int* binary_version);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
