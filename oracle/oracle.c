/*
 * Oracle for the magnification-map path (Weisenbach 2025): plain FP64 CPU
 * reference.  TEST INFRASTRUCTURE ONLY -- see oracle.h for what may use it.
 *
 * Written for a reader who checks it against the paper by eye: the lens
 * equation in complex form, a direct sum over all stars, and per-pixel
 * Sutherland-Hodgman clipping of each mapped triangle.  No blocking, no tree,
 * no fixed point.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Parameters                                                               */
/* ------------------------------------------------------------------------ */

int or_derive_params(double kappa, double gamma, double smooth_fraction,
                     int64_t n_stars, const double *masses,
                     double half_length, int32_t npix, int32_t npix_y,
                     double rays_per_pixel,
                     double flux_fraction_f, const double *center_y,
                     const double *img_half_opt, const int64_t *ray_grid_opt,
                     or_params *out) {
  memset(out, 0, sizeof(*out));
  if (!(half_length > 0) || npix < 1 || npix_y < 0) return -1;
  if (!(smooth_fraction >= 0 && smooth_fraction <= 1)) return -1;
  out->kappa = kappa;
  out->gamma = gamma;
  out->smooth_fraction = smooth_fraction;
  /* Sec. 2.1: s = 1 - kappa_star / kappa */
  out->kappa_star = (1.0 - smooth_fraction) * kappa;
  /* Sec. 2.1, diagonal form of the lens equation */
  out->a1 = 1.0 - kappa + gamma;
  out->a2 = 1.0 - kappa - gamma;
  /* Sec. 3.1: macromodel magnification */
  double det = (1.0 - kappa) * (1.0 - kappa) - gamma * gamma;
  if (det == 0.0) return -1;
  out->mu_macro = 1.0 / det;

  double sm = 0, sm2 = 0;
  for (int64_t i = 0; i < n_stars; i++) {
    sm += masses[i];
    sm2 += masses[i] * masses[i];
  }
  out->mean_m = n_stars > 0 ? sm / (double)n_stars : 0.0;
  out->m2_over_m = sm > 0 ? sm2 / sm : 0.0;
  out->flux_fraction_f = flux_fraction_f > 0 ? flux_fraction_f : 1e-3;
  /* App. A: a fraction f of the deflection PDF lies beyond
   * r = theta_star sqrt(kappa_star <m^2> / (f <m>)) */
  out->r_border = sqrt(out->kappa_star * out->m2_over_m / out->flux_fraction_f);

  out->half_length = half_length;
  out->npix = npix;
  out->npix_y = npix_y > 0 ? npix_y : npix;
  out->delta = 2.0 * half_length / (double)npix;
  /* square pixels: the map is npix_y delta high */
  out->half_length_y = out->npix_y == npix ? half_length : 0.5 * out->npix_y * out->delta;
  out->center_y[0] = center_y ? center_y[0] : 0.0;
  out->center_y[1] = center_y ? center_y[1] : 0.0;

  /* Sec. 2.3: centre of the macro image of the map, and the half-widths of
   * the shooting region with the additive border r */
  out->img_center[0] = out->center_y[0] / out->a1;
  out->img_center[1] = out->center_y[1] / out->a2;
  int explicit_half = img_half_opt && img_half_opt[0] > 0 && img_half_opt[1] > 0;
  if (explicit_half) {
    out->img_half[0] = img_half_opt[0];
    out->img_half[1] = img_half_opt[1];
  } else {
    out->img_half[0] = (half_length + out->r_border) / fabs(out->a1);
    out->img_half[1] = (out->half_length_y + out->r_border) / fabs(out->a2);
  }

  /* Ray grid (Sec. 3.2, Table 1 caption): rays_per_pixel counts rays per
   * pixel in the absence of lensing, so the spacing is delta/sqrt(rpp).  A
   * derived grid keeps square cells and is centred on the region; an
   * explicit grid spans the region exactly. */
  int explicit_grid = ray_grid_opt && ray_grid_opt[0] >= 2 && ray_grid_opt[1] >= 2;
  for (int k = 0; k < 2; k++) {
    if (explicit_grid) {
      out->n[k] = ray_grid_opt[k];
      out->h[k] = 2.0 * out->img_half[k] / (double)(out->n[k] - 1);
      out->x0[k] = out->img_center[k] - out->img_half[k];
    } else {
      if (!(rays_per_pixel > 0)) return -1;
      double hh = out->delta / sqrt(rays_per_pixel);
      out->h[k] = hh;
      out->n[k] = (int64_t)ceil(2.0 * out->img_half[k] / hh) + 1;
      out->x0[k] = out->img_center[k] - 0.5 * (double)(out->n[k] - 1) * hh;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Lens equation, direct sum (Sec. 2.2; smooth sheet of Sec. 3.1)           */
/* ------------------------------------------------------------------------ */

/* App. B: for the sheet of convergence -kappa_star on |x| <= c1, |y| <= c2,
 * with corner c = c1 + i c2,
 *   alpha_s(z) = (-kappa_star i / pi) [ (c - zb) log(c - zb) - (cb - zb) log(cb - zb)
 *                 + (-c - zb) log(-c - zb) - (-cb - zb) log(-cb - zb) ]
 *                - kappa_star (c + cb + z + zb) B_(c1,c2)(z)
 *                - kappa_star 2 (c + cb) B_(inf,c2)(z) H(Re z - c1),
 * zb = conj(z), cb = conj(c), principal logarithms; B is the closed box
 * indicator and H the unit step with H(0) = 1. */
static double complex rect_sheet_alpha(double kappa_star, double c1, double c2,
                                       double complex z) {
  const double pi = 3.14159265358979323846;
  const double complex c = c1 + I * c2, cb = conj(c), zb = conj(z);
  const double complex t1 = (c - zb) * clog(c - zb), t2 = (cb - zb) * clog(cb - zb);
  const double complex t3 = (-c - zb) * clog(-c - zb), t4 = (-cb - zb) * clog(-cb - zb);
  double complex a = (-kappa_star * I / pi) * (t1 - t2 + t3 - t4);
  const double x = creal(z), y = cimag(z);
  const int in_strip = (-c2 <= y && y <= c2);
  if (in_strip && -c1 <= x && x <= c1) a -= kappa_star * (c + cb + z + zb);
  if (in_strip && x - c1 >= 0.0) a -= kappa_star * 2.0 * (c + cb);
  return a;
}

void or_alpha_rect(const or_params *p, double x, double y, double *ax, double *ay) {
  double complex a = 0;
  if (p->star_rect[0] > 0 && p->star_rect[1] > 0)
    a = rect_sheet_alpha(p->kappa_star, p->star_rect[0], p->star_rect[1], x + I * y);
  *ax = creal(a);
  *ay = cimag(a);
}

static void lens_map_point(const or_params *p, int64_t n_stars,
                           const double *masses, const double *pos_xy,
                           double x, double y, double *wx, double *wy) {
  double complex z = x + I * y;
  /* alpha_star(z) = theta_star^2 sum_i m_i / (conj(z) - conj(z_i)) */
  double complex alpha_star = 0;
  for (int64_t i = 0; i < n_stars; i++) {
    double complex zi = pos_xy[2 * i] + I * pos_xy[2 * i + 1];
    alpha_star += masses[i] / (conj(z) - conj(zi));
  }
  /* sheet of convergence -kappa_star over the star region: inside a star
   * disk -kappa_star z; over a rectangle the closed form of App. B */
  double complex alpha_s = -p->kappa_star * z;
  if (p->star_rect[0] > 0 && p->star_rect[1] > 0)
    alpha_s = rect_sheet_alpha(p->kappa_star, p->star_rect[0], p->star_rect[1], z);
  double complex w = (1.0 - p->kappa) * z + p->gamma * conj(z) - alpha_star - alpha_s;
  *wx = creal(w);
  *wy = cimag(w);
}

typedef struct {
  const or_params *p;
  int64_t n_stars;
  const double *masses, *pos_xy;
  int64_t begin, end;
  const double *z_xy; /* explicit points, or NULL for grid vertices */
  int64_t row0;       /* first vertex row when z_xy == NULL */
  int64_t col0, width;/* vertex columns [col0, col0 + width) when z_xy == NULL */
  double *w_xy;
} deflect_job;

static void *deflect_worker(void *arg) {
  deflect_job *J = (deflect_job *)arg;
  const or_params *p = J->p;
  for (int64_t k = J->begin; k < J->end; k++) {
    double x, y;
    if (J->z_xy) {
      x = J->z_xy[2 * k];
      y = J->z_xy[2 * k + 1];
    } else {
      int64_t i = J->col0 + k % J->width;
      int64_t j = J->row0 + k / J->width;
      x = p->x0[0] + (double)i * p->h[0];
      y = p->x0[1] + (double)j * p->h[1];
    }
    lens_map_point(p, J->n_stars, J->masses, J->pos_xy, x, y, &J->w_xy[2 * k],
                   &J->w_xy[2 * k + 1]);
  }
  return NULL;
}

static void run_deflect(const or_params *p, int64_t n_stars,
                        const double *masses, const double *pos_xy, int64_t n,
                        const double *z_xy, int64_t row0, int64_t col0,
                        int64_t width, double *w_xy, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  deflect_job jobs[256];
  for (int t = 0; t < nthreads; t++) {
    jobs[t].p = p;
    jobs[t].n_stars = n_stars;
    jobs[t].masses = masses;
    jobs[t].pos_xy = pos_xy;
    jobs[t].begin = n * t / nthreads;
    jobs[t].end = n * (t + 1) / nthreads;
    jobs[t].z_xy = z_xy;
    jobs[t].row0 = row0;
    jobs[t].col0 = col0;
    jobs[t].width = width;
    jobs[t].w_xy = w_xy;
  }
  if (nthreads == 1) {
    deflect_worker(&jobs[0]);
    return;
  }
  for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, deflect_worker, &jobs[t]);
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

void or_deflect(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t n, const double *z_xy,
                double *w_xy, int nthreads) {
  run_deflect(p, n_stars, masses, pos_xy, n, z_xy, 0, 0, 1, w_xy, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Polygon clipping and area (Sec. 3.2, Fig. 3)                             */
/* ------------------------------------------------------------------------ */

#define MAXV 16

/* Keep the part of the polygon with s*(coord - c) >= 0, coord = x (axis 0) or
 * y (axis 1): one Sutherland-Hodgman pass against one half-plane. */
static int clip_half_plane(const double *in, int nin, double *out, int axis,
                           double c, double s) {
  int nout = 0;
  for (int k = 0; k < nin; k++) {
    const double *P = &in[2 * k];
    const double *Q = &in[2 * ((k + 1) % nin)];
    double dp = s * (P[axis] - c);
    double dq = s * (Q[axis] - c);
    int pin = dp >= 0, qin = dq >= 0;
    if (pin) {
      out[2 * nout] = P[0];
      out[2 * nout + 1] = P[1];
      nout++;
    }
    if (pin != qin) {
      double t = dp / (dp - dq);
      out[2 * nout] = P[0] + t * (Q[0] - P[0]);
      out[2 * nout + 1] = P[1] + t * (Q[1] - P[1]);
      out[2 * nout + axis] = c; /* the crossing lies on the line */
      nout++;
    }
  }
  return nout;
}

/* Shoelace formula: signed area of a simple polygon. */
static double shoelace(const double *v, int n) {
  double a = 0;
  for (int k = 0; k < n; k++) {
    int k1 = (k + 1) % n;
    a += v[2 * k] * v[2 * k1 + 1] - v[2 * k1] * v[2 * k + 1];
  }
  return 0.5 * a;
}

double or_tri_rect_area(const double *tri, double xlo, double ylo, double xhi,
                        double yhi) {
  double a[2 * MAXV], b[2 * MAXV];
  int n = 3;
  memcpy(a, tri, 6 * sizeof(double));
  n = clip_half_plane(a, n, b, 0, xlo, +1.0);
  if (n < 3) return 0.0;
  n = clip_half_plane(b, n, a, 0, xhi, -1.0);
  if (n < 3) return 0.0;
  n = clip_half_plane(a, n, b, 1, ylo, +1.0);
  if (n < 3) return 0.0;
  n = clip_half_plane(b, n, a, 1, yhi, -1.0);
  if (n < 3) return 0.0;
  return fabs(shoelace(a, n));
}

/* ------------------------------------------------------------------------ */
/* Inverse polygon mapping (Sec. 3.2)                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  const or_params *p;
  const double *w_xy; /* vertices of rows [vrow0, ...], columns [col0, col1] */
  int64_t vrow0;
  int64_t col0, col1; /* cell columns [col0, col1) */
  int64_t crow_begin, crow_end; /* cell rows handled by this worker */
  double *acc;                  /* npix_y*npix partial sums */
  or_map_stats st;
} map_job;

/* One triangle with vertices already in pixel units: every pixel of its
 * bounding box (within the map) gets area(T n pixel) / |area(T)|. */
static void apportion_triangle(const double *tri, int npix, int npix_y, double *acc,
                               or_map_stats *st) {
  st->triangles++;
  for (int k = 0; k < 6; k++)
    if (!isfinite(tri[k])) {
      st->dropped++;
      return;
    }
  double xmin = fmin(tri[0], fmin(tri[2], tri[4]));
  double xmax = fmax(tri[0], fmax(tri[2], tri[4]));
  double ymin = fmin(tri[1], fmin(tri[3], tri[5]));
  double ymax = fmax(tri[1], fmax(tri[3], tri[5]));
  /* wholly outside the map: nothing to apportion (not counted as dropped) */
  if (xmax < 0 || ymax < 0 || xmin >= npix || ymin >= npix_y) return;
  double area_t = shoelace(tri, 3);
  if (area_t == 0.0) {
    st->dropped++;
    return;
  }
  int64_t px0 = (int64_t)floor(xmin), px1 = (int64_t)floor(xmax);
  int64_t py0 = (int64_t)floor(ymin), py1 = (int64_t)floor(ymax);
  if (px0 < 0) px0 = 0;
  if (py0 < 0) py0 = 0;
  if (px1 > npix - 1) px1 = npix - 1;
  if (py1 > npix_y - 1) py1 = npix_y - 1;
  for (int64_t py = py0; py <= py1; py++)
    for (int64_t px = px0; px <= px1; px++) {
      double a = or_tri_rect_area(tri, (double)px, (double)py,
                                  (double)(px + 1), (double)(py + 1));
      if (a > 0) {
        acc[py * (int64_t)npix + px] += a / fabs(area_t);
        st->pieces++;
      }
    }
}

static void *map_worker(void *arg) {
  map_job *J = (map_job *)arg;
  const or_params *p = J->p;
  int64_t width = J->col1 - J->col0 + 1; /* vertices per stored row */
  double inv = 1.0 / p->delta;
  double lo0 = p->center_y[0] - p->half_length;
  double lo1 = p->center_y[1] - p->half_length_y;
  for (int64_t j = J->crow_begin; j < J->crow_end; j++) {
    const double *r0 = J->w_xy + 2 * (j - J->vrow0) * width - 2 * J->col0;
    const double *r1 = r0 + 2 * width;
    for (int64_t i = J->col0; i < J->col1; i++) {
      /* vertices of cell (i, j) in pixel units */
      double v00[2] = {(r0[2 * i] - lo0) * inv, (r0[2 * i + 1] - lo1) * inv};
      double v10[2] = {(r0[2 * i + 2] - lo0) * inv, (r0[2 * i + 3] - lo1) * inv};
      double v01[2] = {(r1[2 * i] - lo0) * inv, (r1[2 * i + 1] - lo1) * inv};
      double v11[2] = {(r1[2 * i + 2] - lo0) * inv, (r1[2 * i + 3] - lo1) * inv};
      /* two triangles split along the v00-v11 diagonal */
      double t1[6] = {v00[0], v00[1], v10[0], v10[1], v11[0], v11[1]};
      double t2[6] = {v00[0], v00[1], v11[0], v11[1], v01[0], v01[1]};
      apportion_triangle(t1, p->npix, p->npix_y, J->acc, &J->st);
      apportion_triangle(t2, p->npix, p->npix_y, J->acc, &J->st);
    }
  }
  return NULL;
}

static int map_tile_from_vertices(const or_params *p, const double *w_xy,
                                  int64_t row_begin, int64_t row_end, int64_t col_begin,
                                  int64_t col_end, double *mu_out, double *acc_out,
                                  or_map_stats *stats, int nthreads) {
  if (row_begin < 0 || row_end <= row_begin || row_end > p->n[1] - 1) return -1;
  if (col_begin < 0 || col_end <= col_begin || col_end > p->n[0] - 1) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  int64_t rows = row_end - row_begin;
  if (nthreads > rows) nthreads = (int)rows;
  size_t npx = (size_t)p->npix * (size_t)p->npix_y;
  double *part = (double *)calloc(npx * (size_t)nthreads, sizeof(double));
  if (!part) return -1;
  map_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; t++) {
    jobs[t].p = p;
    jobs[t].w_xy = w_xy;
    jobs[t].vrow0 = row_begin;
    jobs[t].col0 = col_begin;
    jobs[t].col1 = col_end;
    jobs[t].crow_begin = row_begin + rows * t / nthreads;
    jobs[t].crow_end = row_begin + rows * (t + 1) / nthreads;
    jobs[t].acc = part + npx * (size_t)t;
    memset(&jobs[t].st, 0, sizeof(or_map_stats));
  }
  if (nthreads == 1)
    map_worker(&jobs[0]);
  else {
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, map_worker, &jobs[t]);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  }
  /* deterministic reduction in thread order; magnification = fraction sum
   * times image-plane triangle area over pixel area (Sec. 3.2) */
  double scale = 0.5 * p->h[0] * p->h[1] / (p->delta * p->delta);
  or_map_stats st = {0, 0, 0};
  for (size_t q = 0; q < npx; q++) {
    double s = 0;
    for (int t = 0; t < nthreads; t++) s += part[npx * (size_t)t + q];
    if (acc_out) acc_out[q] = s;
    if (mu_out) mu_out[q] = s * scale;
  }
  for (int t = 0; t < nthreads; t++) {
    st.triangles += jobs[t].st.triangles;
    st.dropped += jobs[t].st.dropped;
    st.pieces += jobs[t].st.pieces;
  }
  if (stats) *stats = st;
  free(part);
  return 0;
}

int or_map_from_vertices(const or_params *p, const double *w_xy,
                         int64_t row_begin, int64_t row_end,
                         double *mu_out, double *acc_out, or_map_stats *stats,
                         int nthreads) {
  return map_tile_from_vertices(p, w_xy, row_begin, row_end, 0, p->n[0] - 1, mu_out,
                                acc_out, stats, nthreads);
}

int or_map_tile_from_vertices(const or_params *p, const double *w_xy, int64_t row_begin,
                              int64_t row_end, int64_t col_begin, int64_t col_end,
                              double *mu_out, double *acc_out, or_map_stats *stats,
                              int nthreads) {
  return map_tile_from_vertices(p, w_xy, row_begin, row_end, col_begin, col_end, mu_out,
                                acc_out, stats, nthreads);
}

int or_map_tile(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t row_begin, int64_t row_end,
                int64_t col_begin, int64_t col_end, double *mu_out, double *acc_out,
                or_map_stats *stats, int nthreads) {
  if (row_end <= 0) {
    row_begin = 0;
    row_end = p->n[1] - 1;
  }
  if (col_end <= 0) {
    col_begin = 0;
    col_end = p->n[0] - 1;
  }
  if (row_begin < 0 || row_end <= row_begin || row_end > p->n[1] - 1) return -1;
  if (col_begin < 0 || col_end <= col_begin || col_end > p->n[0] - 1) return -1;
  int64_t width = col_end - col_begin + 1;
  int64_t nv = (row_end - row_begin + 1) * width;
  double *w = (double *)malloc((size_t)nv * 2 * sizeof(double));
  if (!w) return -1;
  run_deflect(p, n_stars, masses, pos_xy, nv, NULL, row_begin, col_begin, width, w,
              nthreads);
  int rc = map_tile_from_vertices(p, w, row_begin, row_end, col_begin, col_end, mu_out,
                                  acc_out, stats, nthreads);
  free(w);
  return rc;
}

int or_map(const or_params *p, int64_t n_stars, const double *masses,
           const double *pos_xy, int64_t row_begin, int64_t row_end,
           double *mu_out, double *acc_out, or_map_stats *stats, int nthreads) {
  return or_map_tile(p, n_stars, masses, pos_xy, row_begin, row_end, 0, 0, mu_out, acc_out,
                     stats, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Inverse ray shooting (Sec. 3.2; the IRS column of Table 1)               */
/* ------------------------------------------------------------------------ */

int or_irs_tile(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t row_begin, int64_t row_end,
                int64_t col_begin, int64_t col_end, int64_t *counts, double *mu_out,
                int64_t *dropped, int nthreads) {
  if (row_end < 0) row_end = p->n[1] - 1;
  if (col_end < 0) col_end = p->n[0] - 1;
  if (row_begin < 0 || row_end < row_begin || row_end > p->n[1] - 1) return -1;
  if (col_begin < 0 || col_end < col_begin || col_end > p->n[0] - 1) return -1;
  int64_t width = col_end - col_begin + 1;
  int64_t nv = (row_end - row_begin + 1) * width;
  double *w = (double *)malloc((size_t)nv * 2 * sizeof(double));
  size_t npx = (size_t)p->npix * (size_t)p->npix_y;
  int64_t *cnt = (int64_t *)calloc(npx, sizeof(int64_t));
  if (!w || !cnt) {
    free(w);
    free(cnt);
    return -1;
  }
  run_deflect(p, n_stars, masses, pos_xy, nv, NULL, row_begin, col_begin, width, w, nthreads);
  /* each ray counts once, in the pixel its source position lies in */
  const double lox = p->center_y[0] - p->half_length, loy = p->center_y[1] - p->half_length_y;
  int64_t nd = 0;
  for (int64_t k = 0; k < nv; k++) {
    double wx = w[2 * k], wy = w[2 * k + 1];
    if (!isfinite(wx) || !isfinite(wy)) {
      nd++;
      continue;
    }
    double u = floor((wx - lox) / p->delta), v = floor((wy - loy) / p->delta);
    if (u >= 0 && u < p->npix && v >= 0 && v < p->npix_y)
      cnt[(size_t)v * (size_t)p->npix + (size_t)u]++;
  }
  double scale = p->h[0] * p->h[1] / (p->delta * p->delta);
  for (size_t q = 0; q < npx; q++) {
    if (counts) counts[q] = cnt[q];
    if (mu_out) mu_out[q] = (double)cnt[q] * scale;
  }
  if (dropped) *dropped = nd;
  free(w);
  free(cnt);
  return 0;
}
