/*
 * Oracle for the magnification-map path of "Rootin' Tootin' Efficient Ray
 * Shootin'" (Weisenbach 2025): a plain, slow, FP64 CPU implementation of the
 * quantity the FMM + inverse-polygon-mapping method approximates.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path under
 * paper_2506_02114_gb300/.
 *
 * What it computes (all FP64, theta_star = 1 units):
 *   - the complex lens equation with a circular smooth sheet (Sec. 2.2 and the
 *     footnote of Sec. 3.1):  w = (1-kappa) z + gamma conj(z)
 *                                 - sum_i m_i / (conj(z) - conj(z_i))
 *                                 + kappa_star z
 *     summed directly over every star in index order (no FMM);
 *   - the shooting region of Sec. 2.3 with the border radius of App. A;
 *   - inverse polygon mapping (Sec. 3.2): every grid cell is split into two
 *     triangles, mapped to the source plane, and each pixel receives
 *     area(T intersect pixel) / |area(T)|; the intersection is found by
 *     clipping T against the four half-planes of that single pixel
 *     (Sutherland-Hodgman) and measured with the shoelace formula;
 *   - inverse ray shooting (Sec. 3.2 and Table 1's IRS column): every grid
 *     vertex is one ray, counted in the pixel its source position falls in;
 *     the magnification is the count times the image-plane area per ray over
 *     the pixel area;
 *   - the smooth sheet of a rectangular star region (App. B): the closed
 *     form with its four complex logarithms and the boxcar / step terms that
 *     keep it continuous across the branch cuts, valid inside and outside.
 *
 * Parity pins: see tests/test_oracle_pins.py.  No function here is
 * "parity unpinned".
 */
#ifndef MM_ORACLE_H
#define MM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  /* lens model (Sec. 2.1-2.2) */
  double kappa, gamma, smooth_fraction;
  double kappa_star;          /* (1 - s) kappa, Sec. 2.1 */
  double a1, a2;              /* 1 - kappa + gamma, 1 - kappa - gamma (Sec. 2.1) */
  double mu_macro;            /* 1 / ((1-kappa)^2 - gamma^2), Sec. 3.1 */
  /* mass moments of the given stars */
  double mean_m, m2_over_m;   /* <m>, <m^2>/<m> */
  double flux_fraction_f;     /* App. A, default 1e-3 */
  double r_border;            /* theta_star sqrt(kappa_star <m^2>/(f <m>)), App. A */
  /* source-plane map (square, Sec. 2.3) */
  double half_length;         /* half-width (x) of the map */
  int32_t npix;               /* pixels along x */
  int32_t npix_y;             /* pixels along y (square pixels) */
  double delta;               /* pixel side 2 half_length / npix */
  double center_y[2];
  /* image-plane shooting region (Sec. 2.3) and ray grid (Sec. 3.2) */
  double img_center[2];
  double img_half[2];
  int64_t n[2];               /* rays (grid vertices) per axis */
  double h[2];                /* ray spacing per axis */
  double x0[2];               /* position of vertex (0,0) */
  /* star region: star_rect = (c1, c2) > 0 places the smooth sheet of
   * convergence -kappa_star on the rectangle |x| <= c1, |y| <= c2 (App. B);
   * zeros (the default) on the disk holding the stars (footnote of Sec. 3.1) */
  double star_rect[2];
  double half_length_y;       /* half-height of the map: npix_y delta / 2 */
} or_params;

typedef struct {
  int64_t triangles;          /* triangles processed */
  int64_t dropped;            /* non-finite triangles, and zero-area ones whose
                                 bounding box meets the map */
  int64_t pieces;             /* non-empty triangle/pixel intersections */
} or_map_stats;

/* Derive every scalar of the run.  img_half_opt / ray_grid_opt may be NULL
 * (or hold zeros) to take the derived values; center_y may be NULL (origin).
 * The map is npix (x) by npix_y (y) square pixels of side 2 half_length /
 * npix; npix_y = 0 means npix (a square map).
 * Returns 0 on success, -1 on invalid arguments. */
int or_derive_params(double kappa, double gamma, double smooth_fraction,
                     int64_t n_stars, const double *masses,
                     double half_length, int32_t npix, int32_t npix_y,
                     double rays_per_pixel,
                     double flux_fraction_f, const double *center_y,
                     const double *img_half_opt, const int64_t *ray_grid_opt,
                     or_params *out);

/* Deflection alpha_s(z) of the rectangular sheet of p->star_rect (App. B),
 * at one point; zero when p->star_rect is unset. */
void or_alpha_rect(const or_params *p, double x, double y, double *ax, double *ay);

/* w at n image-plane points z (interleaved x,y) for the given stars. */
void or_deflect(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t n, const double *z_xy,
                double *w_xy, int nthreads);

/* Magnification map (npix_y rows of npix, row = y pixel index) from the cell
 * rows [row_begin, row_end) of the ray grid (row_end <= 0 means all rows).
 * mu_out receives the magnification; acc_out (may be NULL) the raw sum of
 * area fractions per pixel.  Returns 0 on success. */
int or_map(const or_params *p, int64_t n_stars, const double *masses,
           const double *pos_xy, int64_t row_begin, int64_t row_end,
           double *mu_out, double *acc_out, or_map_stats *stats, int nthreads);

/* Map of the tile of cells rows [row_begin, row_end) x columns
 * [col_begin, col_end) (col_end <= 0: all columns). */
int or_map_tile(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t row_begin, int64_t row_end,
                int64_t col_begin, int64_t col_end, double *mu_out, double *acc_out,
                or_map_stats *stats, int nthreads);

/* Same as or_map but from precomputed source positions w_xy of the vertices
 * of rows [row_begin, row_end] (inclusive), (row_end-row_begin+1)*n[0] points. */
int or_map_from_vertices(const or_params *p, const double *w_xy,
                         int64_t row_begin, int64_t row_end,
                         double *mu_out, double *acc_out, or_map_stats *stats,
                         int nthreads);

/* Same as or_map_tile but from precomputed source positions w_xy of the
 * vertices of rows [row_begin, row_end] and columns [col_begin, col_end]
 * (both inclusive), row-major, (col_end-col_begin+1) points per row. */
int or_map_tile_from_vertices(const or_params *p, const double *w_xy, int64_t row_begin,
                              int64_t row_end, int64_t col_begin, int64_t col_end,
                              double *mu_out, double *acc_out, or_map_stats *stats,
                              int nthreads);

/* Inverse ray shooting over the vertices of rows [row_begin, row_end] and
 * columns [col_begin, col_end] (both inclusive; row_end < 0 or col_end < 0
 * means up to the grid's last vertex): counts (npix_y rows of npix, may be NULL) gets
 * the rays per pixel, mu_out (may be NULL) count * h_x h_y / delta^2, and
 * *dropped the rays with a non-finite source position.  Pixel (px, py)
 * holds the rays with floor((w - (center - half_length)) / delta) = (px, py).
 * Returns 0 on success. */
int or_irs_tile(const or_params *p, int64_t n_stars, const double *masses,
                const double *pos_xy, int64_t row_begin, int64_t row_end,
                int64_t col_begin, int64_t col_end, int64_t *counts, double *mu_out,
                int64_t *dropped, int nthreads);

/* Area of the intersection of a triangle (x0,y0,x1,y1,x2,y2) with the
 * axis-aligned rectangle [xlo,xhi] x [ylo,yhi]; always >= 0. */
double or_tri_rect_area(const double *tri, double xlo, double ylo, double xhi,
                        double yhi);

#ifdef __cplusplus
}
#endif
#endif
