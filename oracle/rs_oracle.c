/*
 * FP64 CPU oracle for direct inverse ray-shooting (TEST INFRASTRUCTURE).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use this file.  It shares no code, header or constant with the CUDA path:
 * it is the plain definition of what that path computes, evaluated slowly in
 * double precision so that its results can serve as the truth.
 *
 * What it computes (Thompson, Fluke, Barnes & Barsdell 2009):
 *   - Eq. 2  (Section 1): alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2, a direct
 *            sum over all lenses, evaluated with the per-lens steps of the flop
 *            count in Appendix A:
 *              f1 = x1 - x_{i,1};  f2 = x2 - x_{i,2};
 *              d  = m_i / (f1 f1 + f2 f2);
 *              alpha1 += d f1;     alpha2 += d f2.
 *            Lenses are visited in index order; each component is accumulated
 *            with Neumaier's compensated summation so that the double result
 *            is accurate to a few units in the last place even for 1e8 lenses.
 *   - Eq. 6  (Section 3.2): y = diag(1 - gamma, 1 + gamma) x - sigma_c x - alpha,
 *            i.e. y1 = (1 - kappa_c - gamma) x1 - alpha1,
 *                 y2 = (1 - kappa_c + gamma) x2 - alpha2, with kappa_c = sigma_c.
 *            The macro factors are formed as (1 - kappa_c) - gamma and
 *            (1 - kappa_c) + gamma; y_k = lambda_k x_k - alpha_k (product
 *            rounded, then difference rounded: no fused multiply-add).
 *   - Eq. 4  (Section 1): mu_ij = N_ij / N_av, N_ij the rays binned into source
 *            pixel (i, j) and N_av the rays a pixel receives without lensing
 *            (pixel area / ray-cell area).
 *   - Binning (Section 2.1, step 4: the rays' source positions are mapped onto
 *            the pixel grid; the paper gives no formula).  Reading used here:
 *            u_k = (y_k - lo_k) * (npix_k / (hi_k - lo_k)); the ray lands in the
 *            window iff 0 <= u_k < npix_k on both axes (a NaN fails), in pixel
 *            p_k = floor(u_k); counts are row-major [p2][p1].  Every other ray
 *            is counted as out of window.
 *
 * Rays: the paper draws random rays; here ray (i, j) of a regular grid sits at
 *   x_k = (float)fma(index_k, spacing_k, origin_k)
 * (double fma, then rounded to float, then used as a double).  The float
 * value IS the ray position.
 *
 * A ray that hits a lens exactly (f1 = f2 = 0) gets a non-finite deflection
 * and is counted out of window.
 *
 * Built with -O2 -fopenmp -ffp-contract=off and no fast-math: every double
 * operation below is one IEEE operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Neumaier (improved Kahan-Babuska) compensated accumulator. */
typedef struct { double s, c; } nsum_t;

static inline void nsum_add(nsum_t* a, double t) {
  double u = a->s + t;
  if (fabs(a->s) >= fabs(t))
    a->c += (a->s - u) + t;
  else
    a->c += (t - u) + a->s;
  a->s = u;
}

static inline double nsum_value(const nsum_t* a) { return a->s + a->c; }

/* Position of ray (i, j): float(fma(i, spacing, origin)) per axis. */
static inline void ray_position(int64_t i, int64_t j, const double origin[2], const double spacing[2],
                                double x[2]) {
  x[0] = (double)(float)fma((double)i, spacing[0], origin[0]);
  x[1] = (double)(float)fma((double)j, spacing[1], origin[1]);
}

/* Eq. 2 with the Appendix A steps, compensated sums, lens index order. */
static void deflection(const float* lens_xy, const float* masses, int64_t n_lens, const double x[2],
                       double alpha[2]) {
  nsum_t a1 = {0.0, 0.0}, a2 = {0.0, 0.0};
  for (int64_t i = 0; i < n_lens; ++i) {
    double xi1 = (double)lens_xy[2 * i];
    double xi2 = (double)lens_xy[2 * i + 1];
    double m = masses ? (double)masses[i] : 1.0;
    double f1 = x[0] - xi1;
    double f2 = x[1] - xi2;
    double d = m / (f1 * f1 + f2 * f2);
    nsum_add(&a1, d * f1);
    nsum_add(&a2, d * f2);
  }
  alpha[0] = nsum_value(&a1);
  alpha[1] = nsum_value(&a2);
}

/* Eq. 6: source position of image position x. */
static inline void lens_map(double kappa_c, double gamma, const double x[2], const double alpha[2],
                            double y[2]) {
  double lam1 = (1.0 - kappa_c) - gamma;
  double lam2 = (1.0 - kappa_c) + gamma;
  y[0] = lam1 * x[0] - alpha[0];
  y[1] = lam2 * x[1] - alpha[1];
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Source positions of k listed rays.  ray_ij: int64 [k][2] = (i, j).
 * y_out: double [k][2].  alpha_out (may be NULL): double [k][2].
 * x_out (may be NULL): double [k][2], the ray positions used.
 */
void oracle_trace(const float* lens_xy, const float* masses, int64_t n_lens, double kappa_c, double gamma,
                  const double origin[2], const double spacing[2], const int64_t* ray_ij, int64_t k,
                  double* y_out, double* alpha_out, double* x_out) {
  int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
  for (r = 0; r < k; ++r) {
    double x[2], alpha[2], y[2];
    ray_position(ray_ij[2 * r], ray_ij[2 * r + 1], origin, spacing, x);
    deflection(lens_xy, masses, n_lens, x, alpha);
    lens_map(kappa_c, gamma, x, alpha, y);
    y_out[2 * r] = y[0];
    y_out[2 * r + 1] = y[1];
    if (alpha_out) {
      alpha_out[2 * r] = alpha[0];
      alpha_out[2 * r + 1] = alpha[1];
    }
    if (x_out) {
      x_out[2 * r] = x[0];
      x_out[2 * r + 1] = x[1];
    }
  }
}

/* Bin one source position; returns the flat pixel index or -1 when out of window. */
static inline int64_t bin_index(const double y[2], const double lo[2], const double scale[2],
                                const int32_t npix[2]) {
  double u1 = (y[0] - lo[0]) * scale[0];
  double u2 = (y[1] - lo[1]) * scale[1];
  if (!(u1 >= 0.0 && u1 < (double)npix[0] && u2 >= 0.0 && u2 < (double)npix[1])) return -1;
  int64_t p1 = (int64_t)floor(u1);
  int64_t p2 = (int64_t)floor(u2);
  return p2 * (int64_t)npix[0] + p1;
}

/*
 * Shoot rows j in [j_begin, j_end) of the grid (all n0 rays of each row) and
 * ACCUMULATE the binned counts (uint32 [npix2][npix1]) and the out-of-window
 * count.  Source positions are computed in parallel over rays; binning is a
 * single serial pass afterwards (as in the paper's OpenMP code, Section 2.1).
 * Returns 0, or -1 if a work buffer could not be allocated.
 */
int oracle_shoot_rows(const float* lens_xy, const float* masses, int64_t n_lens, double kappa_c,
                      double gamma, const double origin[2], const double spacing[2], int64_t n0,
                      int64_t j_begin, int64_t j_end, const double lo[2], const double hi[2],
                      const int32_t npix[2], uint32_t* counts, uint64_t* out_of_window) {
  double scale[2];
  scale[0] = (double)npix[0] / (hi[0] - lo[0]);
  scale[1] = (double)npix[1] / (hi[1] - lo[1]);
  const int64_t rows_per_chunk = n0 > 0 ? (int64_t)((1 << 20) / n0 + 1) : 1;
  double* ybuf = (double*)malloc(sizeof(double) * 2 * (size_t)(rows_per_chunk * (n0 > 0 ? n0 : 1)));
  if (!ybuf) return -1;
  uint64_t oow = 0;
  for (int64_t jb = j_begin; jb < j_end; jb += rows_per_chunk) {
    int64_t je = jb + rows_per_chunk < j_end ? jb + rows_per_chunk : j_end;
    int64_t nr = (je - jb) * n0;
    int64_t r;
#pragma omp parallel for schedule(dynamic, 64)
    for (r = 0; r < nr; ++r) {
      double x[2], alpha[2], y[2];
      ray_position(r % n0, jb + r / n0, origin, spacing, x);
      deflection(lens_xy, masses, n_lens, x, alpha);
      lens_map(kappa_c, gamma, x, alpha, y);
      ybuf[2 * r] = y[0];
      ybuf[2 * r + 1] = y[1];
    }
    for (r = 0; r < nr; ++r) {
      int64_t p = bin_index(&ybuf[2 * r], lo, scale, npix);
      if (p < 0)
        ++oow;
      else
        counts[p] += 1u;
    }
  }
  free(ybuf);
  if (out_of_window) *out_of_window += oow;
  return 0;
}

/*
 * Bin given source positions (double [k][2]) into counts; returns the number out of window.
 * Used by tests that build maps from listed positions.
 */
uint64_t oracle_bin_positions(const double* y, int64_t k, const double lo[2], const double hi[2],
                              const int32_t npix[2], uint32_t* counts) {
  double scale[2];
  scale[0] = (double)npix[0] / (hi[0] - lo[0]);
  scale[1] = (double)npix[1] / (hi[1] - lo[1]);
  uint64_t oow = 0;
  for (int64_t r = 0; r < k; ++r) {
    int64_t p = bin_index(&y[2 * r], lo, scale, npix);
    if (p < 0)
      ++oow;
    else
      counts[p] += 1u;
  }
  return oow;
}

/*
 * Eq. 4: mu = N_ij / N_av with N_av = (pixel area) / (ray-cell area)
 *      = ((hi1-lo1)/npix1 * (hi2-lo2)/npix2) / (spacing1 * spacing2).
 */
void oracle_magnification(const uint32_t* counts, const double spacing[2], const double lo[2],
                          const double hi[2], const int32_t npix[2], double* mu) {
  double pix_area = ((hi[0] - lo[0]) / (double)npix[0]) * ((hi[1] - lo[1]) / (double)npix[1]);
  double n_av = pix_area / (spacing[0] * spacing[1]);
  int64_t n = (int64_t)npix[0] * (int64_t)npix[1];
  for (int64_t p = 0; p < n; ++p) mu[p] = (double)counts[p] / n_av;
}

/*
 * Light curves (Section 1: a source profile is moved across the magnification map and the
 * magnification at each position is converted to a magnitude change).  The paper gives no
 * formula; the reading used here:
 *   - sample k of a track sits at y_k = y0 + k * step (double, per axis: fma-free y0 + k*step);
 *   - map pixel (i, j) has centre c = (lo0 + (i + 0.5) * pix0, lo1 + (j + 0.5) * pix1) with
 *     pix = (hi - lo) / npix (product then sum, no fma);
 *   - the source profile weighs pixels by the distance d of their centres from y_k,
 *     d^2 = dx*dx + dy*dy (no fma):
 *       profile 0, Gaussian of standard deviation s:  w = exp(-d^2 / (2 s^2)) if d^2 <= (6 s)^2, else 0;
 *       profile 1, uniform disc of radius s:          w = 1 if d^2 <= s^2, else 0;
 *   - mu_k = sum_p w_p mu_p / sum_p w_p over all pixels of the map (NaN when no pixel has weight);
 *   - magnitude change dm_k = -2.5 log10(mu_k).
 * mu: double [npix1][npix0] (row-major, [p2][p1]).  Every pixel of the map is visited for every
 * sample (slow, obviously complete).
 */
void oracle_light_curve(const double* mu, const int32_t npix[2], const double lo[2], const double hi[2],
                        int profile, double s, const double y0[2], const double step[2], int64_t n,
                        double* mu_out, double* mag_out) {
  const double pix0 = (hi[0] - lo[0]) / (double)npix[0];
  const double pix1 = (hi[1] - lo[1]) / (double)npix[1];
  const double cut2 = profile == 0 ? (6.0 * s) * (6.0 * s) : s * s;
  const double inv2s2 = 1.0 / (2.0 * s * s);
  int64_t k;
#pragma omp parallel for schedule(dynamic, 4)
  for (k = 0; k < n; ++k) {
    const double yx = y0[0] + (double)k * step[0];
    const double yy = y0[1] + (double)k * step[1];
    double sw = 0.0, swm = 0.0;
    for (int32_t j = 0; j < npix[1]; ++j) {
      const double cy = lo[1] + ((double)j + 0.5) * pix1;
      const double dy = cy - yy;
      for (int32_t i = 0; i < npix[0]; ++i) {
        const double cx = lo[0] + ((double)i + 0.5) * pix0;
        const double dx = cx - yx;
        const double d2 = dx * dx + dy * dy;
        if (d2 > cut2) continue;
        const double w = profile == 0 ? exp(-d2 * inv2s2) : 1.0;
        sw += w;
        swm += w * mu[(int64_t)j * npix[0] + i];
      }
    }
    const double m = sw > 0.0 ? swm / sw : NAN;
    mu_out[k] = m;
    if (mag_out) mag_out[k] = -2.5 * log10(m);
  }
}

/*
 * Lens positions of a moving field at time t (Section 4: the motion of individual stars changes
 * the caustic network; maps are then made per time step).  The paper gives no formula; the reading
 * used here: straight-line motion, x_i(t) = x_i + v_i t per axis, evaluated in double (product,
 * then sum, no fma) from the float32 position and velocity and rounded to float32, the precision of
 * the lens arrays.  xy, vel, out: float [2 n], interleaved (x1, x2) per lens.
 */
void oracle_lens_positions(const float* xy, const float* vel, int64_t n, double t, float* out) {
  for (int64_t i = 0; i < 2 * n; ++i) {
    const double moved = (double)xy[i] + (double)vel[i] * t;
    out[i] = (float)moved;
  }
}
