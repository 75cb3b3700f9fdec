/*
 * libmm -- GB300-native magnification maps for gravitational microlensing:
 * fast-multipole ray deflection plus inverse polygon mapping (Weisenbach
 * 2025, "Rootin' Tootin' Efficient Ray Shootin'").
 *
 * A map is the pixel-averaged magnification of a square source-plane region
 * for the lens equation of Sec. 2.2 (complex form)
 *
 *     w = (1 - kappa) z + gamma conj(z) - alpha_star(z) - alpha_s(z),
 *     alpha_star(z) = sum_i m_i / (conj(z) - conj(z_i))         (theta_star = 1)
 *     alpha_s(z)    = -kappa_star z                (circular sheet, Sec. 3.1)
 *
 * built by shooting a regular grid of rays from the image-plane region of
 * Sec. 2.3 / App. A, splitting each grid cell into two triangles and
 * apportioning each mapped triangle's area exactly among the pixels it covers
 * (Sec. 3.2).  The deflection uses the quadtree fast multipole method of
 * Sec. 3.3 and App. C.
 *
 * Conventions for every call:
 *   - All functions return mm_status; no C++ exception crosses this ABI.
 *     mm_last_error() returns a thread-local message for the last failure.
 *   - Positions are interleaved (x, y) doubles; units are Einstein radii of a
 *     unit mass (theta_star = 1).
 *   - A map is npix_y rows of npix values (npix_y = npix unless
 *     mm_options.npix_y is set), row-major, row index = y pixel; pixel
 *     (px, py) covers [c_x - L + px*d, c_x - L + (px+1)*d) x
 *     [c_y - L_y + py*d, c_y - L_y + (py+1)*d), with L = half_length,
 *     d = 2L/npix, L_y = npix_y d / 2 and c the map centre.
 *   - A handle owns all of its device memory and is used by one host thread
 *     at a time.  Different handles may run concurrently on different streams.
 *     Its buffers come from the device's default memory pool (stream-ordered
 *     allocation); the library raises that pool's release threshold, so the
 *     memory of a destroyed handle stays with the process for the next one.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL is the
 *     legacy default stream.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_map mm_map; /* opaque handle */

typedef enum {
  MM_OK = 0,
  MM_EINVAL = 1,   /* invalid argument; nothing was changed */
  MM_ENOMEM = 2,   /* device or host allocation failed */
  MM_ECUDA = 3,    /* a CUDA call failed (message in mm_last_error) */
  MM_ETIMEOUT = 4, /* a bounded device-side wait gave up; handle is unusable */
  MM_ESTATE = 5    /* call not valid in the handle's state */
} mm_status;

typedef enum {
  MM_FMM_FP32 = 0,  /* FMM deflection, FP32 per ray, FP64 expansions (default) */
  MM_PLAIN_FP64 = 1, /* direct sum over every star in FP64 (no tree) */
  MM_FMM_IRS = 2     /* inverse ray shooting (Sec. 3.2, Table 1's IRS column):
                        the deflection of MM_FMM_FP32, then every grid vertex
                        (ray) adds one count to the pixel it lands in; mu =
                        count h_x h_y / delta^2, and mm_get_map_fixed returns
                        the counts.  triangles_dropped counts rays with a
                        non-finite position; no batching, no autotuning. */
} mm_mode;

/* Options; a zero-initialised struct (or NULL) selects the defaults. */
typedef struct {
  int32_t mode;             /* mm_mode */
  int32_t time_stages;      /* 1: record CUDA events around each stage of
                               mm_run; read them with mm_get_stats */
  double img_half[2];       /* > 0: explicit half-widths of the image-plane
                               shooting region (else Sec. 2.3 / App. A) */
  int64_t ray_grid[2];      /* >= 2: explicit rays per axis spanning exactly
                               the region (else spacing d/sqrt(rays_per_pixel),
                               square cells, grid centred on the region) */
  double flux_fraction_f;   /* App. A flux fraction beyond the border; 0 -> 1e-3 */
  double center_y[2];       /* map centre in the source plane (Sec. 2.3) */
  int64_t row_begin;        /* shoot only cell rows [row_begin, row_end) of the */
  int64_t row_end;          /*   ray grid; both 0 -> every row */
  int32_t rows_per_item;    /* rows of cells per warp work item, 1..4096; 0 ->
                               the largest of 256, 128, ..., 16 that leaves every
                               resident warp >= 16 items */
  int32_t sub_levels;       /* FMM mode: each leaf's local expansion is re-centred
                               exactly on its 4^s sub-cells (s levels below the
                               leaf); a sub-cell sums directly only the leaf's
                               near stars within its 5 x 5 block of sub-cells and
                               takes the others into its expansion (P2L); the
                               expansion is evaluated to the fewest terms whose
                               truncation bound matches order p at the leaf
                               centre (App. C error model).  -1: none (the
                               leaf-level scheme); 0: the default (2); 1 or 2: s.
                               Capped so that leaves plus sub-cells stay within
                               21 tree levels. */
  int64_t col_begin;        /* shoot only cell columns [col_begin, col_end) of */
  int64_t col_end;          /*   the ray grid; both 0 -> every column */
  int32_t no_cull;          /* FMM mode: 1 computes every vertex; 0 (default)
                               skips vertex rows of the warp proven, from
                               per-sub-cell bounds on the macro term, the
                               evaluated series and the direct stars'
                               deflection, to land beyond the same map edge
                               as the row below (the map is unchanged: such
                               cells lie wholly outside it) */
  int32_t big_queue_slots;  /* queue for the second mapping pass, in triangles:
                               0 -> when the map's accumulators (16 B per
                               pixel) fit half the GPU's L2, the larger
                               triangles the autotuner counted (its
                               jobs_per_mcell, scaled to the grid) plus a
                               quarter, else 1 per 12 cells, within 2^16 ..
                               2^27 (2^20, then none, when the device has not
                               that much memory free); else none.  -1 -> none
                               (the first pass deals every larger triangle);
                               n > 0 -> n.  With a queue and a map that fits,
                               the first pass runs in consecutive segments of
                               work items, each followed by the second pass,
                               so that the expected larger triangles fit.
                               Batches that still do not fit are dealt by the
                               first pass (same map). */
  int32_t autotune;         /* FMM mode, 1: mm_create first times candidate
                               settings and keeps the fastest: leaf_size in
                               {16, 32, 64} when its argument is 0, sub_levels in
                               {1, 2} when 0, rows_per_item in {automatic, 64,
                               512} when 0.  Each candidate plan covers the
                               whole grid (or band) and shoots every k-th row
                               block of work items (k <= 16, a uniform sample),
                               scored as tree + expansions + k x mapping time,
                               the best of two timed runs.  p is not tuned: when
                               0 it stays the smallest order App. C.3's error
                               rule allows (a larger p only adds work).  The
                               choice changes the map only within the FMM
                               tolerances (leaf_size, sub_levels) and not at all
                               through rows_per_item.  Ignored in
                               MM_PLAIN_FP64 mode and when nothing is left 0. */
  int32_t reserved0;        /* 0 */
  const char *tune_cache;   /* autotune: path of a JSON-lines file of earlier
                               choices (NULL: none), read first and appended
                               to after a timed choice.  One object per line:
                               {"key": K, "leaf_size": L, "sub_levels": S,
                               "rows_per_item": R, "jobs_per_mcell": J,
                               "ms_estimate": T} (J: larger triangles per 2^20
                               cells counted by the chosen candidate's sampled
                               run, -1 or absent when not known), K built
                               from the GPU's compute capability, the requested
                               fmm_order, leaf_size, sub_levels and
                               rows_per_item, and floor(log2) of N_star, the
                               rays and npix; the last matching line wins.
                               Unreadable files and malformed lines are
                               ignored; a failed write is not an error.  Read
                               only during mm_create. */
  double critical_mu;       /* statistics: a mapped triangle whose local |mu|
                               (image area / source area) exceeds this counts
                               as near-critical (mm_stats); 0 -> 1e3 */
  double star_rect[2];      /* > 0 (both): the stars fill the rectangle
                               |x| <= c1, |y| <= c2 (half-widths c1, c2) and
                               the smooth sheet of convergence -kappa_star
                               covers that rectangle (App. B); the ray grid
                               must lie strictly inside it.  In FMM modes the
                               sheet's part beyond -kappa_star z, analytic in
                               the rectangle, joins each sub-cell's expansion
                               (no per-ray cost); its series converges like
                               sqrt(2) L_s / (distance to the nearest
                               corner), and mm_create fails with MM_EINVAL
                               where that ratio exceeds 1/2 for a sub-cell
                               of the grid.  0 (both): stars in a disk around
                               the origin, sheet -kappa_star z (Sec. 3.1). */
  int32_t npix_y;           /* > 0: the map has npix_y rows of npix square
                               pixels of side 2 half_length / npix (half-height
                               npix_y delta / 2); 0: npix rows (square map) */
  int32_t reserved1;        /* 0 */
} mm_options;

/* Every derived scalar of a run (host-side numbers; no GPU needed). */
typedef struct {
  double kappa, gamma, smooth_fraction;
  double kappa_star;        /* (1 - s) kappa, Sec. 2.1 */
  double a1, a2;            /* 1 - kappa + gamma, 1 - kappa - gamma */
  double mu_macro;          /* 1 / ((1-kappa)^2 - gamma^2), Sec. 3.1 */
  double mean_m, m2_over_m; /* <m>, <m^2>/<m> of the given stars */
  double flux_fraction_f;
  double r_border;          /* sqrt(kappa_star <m^2> / (f <m>)), App. A */
  double half_length;
  int32_t npix;             /* pixels along x */
  int32_t npix_y;           /* pixels along y (square pixels) */
  double delta;             /* pixel side 2 half_length / npix */
  double center_y[2];
  double img_center[2];     /* centre of the shooting region, Sec. 2.3 */
  double img_half[2];       /* half-widths of the shooting region */
  int64_t n[2];             /* rays (grid vertices) per axis */
  double h[2];              /* ray spacing per axis */
  double x0[2];             /* image-plane position of vertex (0, 0) */
  double half_length_y;     /* half-height of the map, npix_y delta / 2 */
} mm_params;

typedef struct {
  mm_params params;
  int32_t mode;
  int32_t fmm_order;        /* expansion order p actually used */
  int32_t leaf_size;        /* maximum stars used directly (App. C.1), default 32 */
  int32_t depth;            /* deepest tree level */
  int32_t eval_order;       /* terms of the re-centred expansion evaluated per ray */
  int32_t sub_levels;       /* sub-cell levels s actually used */
  int64_t n_stars;
  int64_t nodes;            /* tree nodes over all levels */
  int64_t leaves;           /* leaves over all levels */
  int64_t active_leaves;    /* leaves containing ray-grid vertices */
  double root_half_length;
  double min_leaf_half_length; /* smallest half-length of an active leaf */
  double mean_near_stars;   /* mean near-field (direct) stars per active-leaf
                               vertex, weighted by vertices */
  int64_t rays;             /* grid vertices shot by mm_run (band included) */
  int64_t cells;            /* grid cells mapped by mm_run */
  int64_t triangles_dropped;/* non-finite triangles, and zero-area ones whose
                               box meets the map (last run) */
  int64_t triangles_clipped;/* triangles spanning more than one pixel of the map */
  int64_t triangles_line;   /*   of which two pixels split by one grid line */
  int64_t triangles_quad;   /*   of which 2 x 2 pixels (both grid lines crossed) */
  int64_t triangles_box;    /*   of which with a box of at most 64 map pixels */
  int64_t triangles_rows;   /*   of which larger (pixel rows shared by a warp) */
  int64_t rows_culled;      /* warp rows of vertices not computed (culling) */
  int64_t kernel_launches;  /* library kernels launched by the last run (CUB's
                               sort/scan kernels and memsets not counted) */
  /* stage times of the last mm_run in ms (time_stages = 1), else -1;
     ms_shoot = ms_first_pass (deflection and the one-, two- and 2x2-pixel
     triangles) + ms_second_pass (the queued larger triangles).  For the
     handle that led the last mm_run_batch (hs[0]), ms_first_pass is the
     batch's one shared first-pass launch over every map. */
  double ms_tree, ms_expansions, ms_shoot, ms_normalize, ms_total;
  double ms_first_pass, ms_second_pass;
  int32_t rows_per_item;    /* rows of cells per work item in use */
  int32_t autotuned;        /* 0: not tuned; 1: tuned by timing; 2: taken from
                               the tune_cache file */
  double ms_autotune;       /* host wall time mm_create spent tuning, 0 if none */
  int64_t triangles_near_critical; /* triangles not wholly beyond one map edge
                               with local |mu| above critical_mu (last run) */
  uint32_t error_bits;      /* the handle's device error word: 1 quadtree
                               invariant, 2 a vertex outside every active leaf,
                               4 a star-rectangle corner near a sub-cell, 8 a
                               map index out of range (only the MM_DEBUG build
                               checks, and skips the access) */
  int32_t queue_slots;      /* capacity of the second-pass queue, in triangles
                               (0: none; see mm_options.big_queue_slots) */
} mm_stats;

/*
 * Derive the run's scalars without touching a GPU: kappa_star (Sec. 2.1),
 * mu_macro (Sec. 3.1), the border r (App. A), the shooting region (Sec. 2.3)
 * and the ray grid (Sec. 3.2 / Table 1 caption).  masses: host, n_stars
 * values (may be NULL when n_stars == 0).  Returns MM_EINVAL for the
 * arguments mm_create rejects.
 */
mm_status mm_derive_params(double kappa_tot, double shear, double smooth_fraction,
                           int64_t n_stars, const double *masses,
                           double half_length, int32_t npix, double rays_per_pixel,
                           const mm_options *opt, mm_params *out);

/*
 * Create a map handle.  Copies the stars to the device (the caller may free
 * masses/pos_xy on return), derives every parameter, builds the quadtree once
 * to size its workspace, and allocates all device memory the handle needs.
 *
 *   kappa_tot, shear, smooth_fraction: kappa, gamma, s of Sec. 2.1;
 *     kappa_star = (1 - s) kappa.
 *   n_stars, masses[n_stars], pos_xy[2*n_stars]: host arrays, masses > 0.
 *   half_length, npix: square map of side 2*half_length, npix pixels a side.
 *   rays_per_pixel: rays per pixel in the absence of lensing (Table 1
 *     caption); ignored when opt->ray_grid is given.
 *   fmm_order: expansion order p (App. C.3); 0 picks
 *     p > log2(<m^2>/<m> / (L eps)) with eps = d/10 and L the smallest active
 *     leaf half-length; accepted range [0, 64].
 *   leaf_size: maximum number of stars in a node and its neighbours used
 *     directly (Sec. 3.3); 0 -> 32; accepted range [0, 1024].
 *   opt: may be NULL.
 *   out: receives the handle.
 *
 * Errors: MM_EINVAL for |(1-kappa)^2 - gamma^2| < 1e-12, s outside [0,1],
 * kappa_star > 0 with no stars, masses <= 0 or non-finite positions, npix < 1,
 * half_length <= 0, fmm_order or leaf_size out of range, a ray grid above
 * 2^31 rays per axis, or (kappa_star > 0, img_half not explicit) a ray grid
 * the stars do not cover: its box must lie inside the stars' bounding box
 * and, for a star disk (no star_rect), each of its four corners within the
 * disk the stars fill, radius max |z_i| about the origin -- the circular
 * sheet deflects by -kappa_star z only inside that disk (Sec. 3.1).  With
 * star_rect the grid must lie strictly inside the rectangle instead.
 * MM_ENOMEM / MM_ECUDA otherwise.
 */
mm_status mm_create(double kappa_tot, double shear, double smooth_fraction,
                    int64_t n_stars, const double *masses, const double *pos_xy,
                    double half_length, int32_t npix, double rays_per_pixel,
                    int32_t fmm_order, int32_t leaf_size, const mm_options *opt,
                    mm_map **out);

/*
 * Compute the map on the given stream: tree build (Morton sort, levels,
 * interaction lists), multipole up-sweep, local down-sweep, fused ray
 * deflection + inverse polygon mapping into a fixed-point accumulator, and
 * normalisation to magnification.  Asynchronous: returns once enqueued.
 * The caller synchronises the stream before reading results from the host.
 * mm_create's plan already builds the tree and expansions for the handle's
 * stars; the first run after it uses them (its tree and expansion stage
 * times read 0) and every later run rebuilds them.
 */
mm_status mm_run(mm_map *h, void *stream);

/*
 * Run n handles (all created in MM_FMM_FP32 mode on the current device) with
 * one persistent deflection+mapping launch whose work queue spans every map.
 * The maps' trees and expansions before it, and their second passes and
 * normalisation after it, run side by side on up to 8 streams that hs[0]
 * owns, forked from and joined back to `stream` with events.
 * Asynchronous like mm_run, with no host synchronisation: the batch's
 * descriptor array is assembled on the device (hs[0] holds it), so the call
 * can be captured in a CUDA graph once an earlier call with at least n
 * handles led by hs[0] has sized that array and created those streams.
 * Each map is bit-identical to its own mm_run.
 */
mm_status mm_run_batch(mm_map *const *hs, int32_t n, void *stream);

/*
 * Run the map over a rectangle of the handle's cells only: cell rows
 * [row_begin, row_end) and columns [col_begin, col_end) of the ray grid,
 * inside the handle's own rows and columns (mm_options row/column band).
 * The plan mm_create made for the whole handle -- tree, expansions, leaf
 * records, lookup grid, culling bounds, second-pass queue -- is used
 * unchanged, and each triangle's contribution depends only on its vertices,
 * so the fixed-point maps (mm_get_map_fixed) of rectangles that partition the
 * handle's cells add up bit for bit to mm_run's map.  This is how one map is
 * sharded over devices by ray-grid bands (Sec. 6 names several GPUs as the
 * remaining speed-up): each device runs its band on its own handle, the u64
 * maps are summed (integer sums, exact in any order) and mm_normalize_fixed
 * turns the sum into magnification.  It also lets a full-size plan be
 * checked tile by tile.  Asynchronous like mm_run; afterwards mm_get_map,
 * mm_get_map_fixed and mm_get_stats describe this rectangle's run.  In
 * MM_FMM_IRS mode the rays counted are the rectangle's vertices, its last
 * row and column included.  MM_EINVAL for an empty rectangle or one outside
 * the handle's cells.
 */
mm_status mm_run_cells(mm_map *h, int64_t row_begin, int64_t row_end, int64_t col_begin,
                       int64_t col_end, void *stream);

/*
 * Normalise a fixed-point accumulator into magnification with the handle's
 * scale (Sec. 3.2: mu = acc 2^-32 (h_x h_y / 2) / delta^2 for polygon
 * mapping; count h_x h_y / delta^2 for ray counting).  acc: DEVICE pointer
 * to npix_y rows of npix uint64, as mm_get_map_fixed returns them or their
 * sum over several handles of the same map (mm_run_cells bands); out: DEVICE
 * pointer to npix_y * npix floats.  Bit-identical to mm_get_map's values for
 * the same accumulator.  Enqueued on `stream`; the caller keeps both buffers
 * alive until it completes.
 */
mm_status mm_normalize_fixed(const mm_map *h, const uint64_t *acc, float *out, void *stream);

/*
 * Copy the magnification map (npix_y rows of npix floats) into out.  on_device = 0:
 * out is host memory (the call synchronises); 1: out is device memory and the
 * copy is enqueued on the handle's last stream.
 */
mm_status mm_get_map(const mm_map *h, float *out, int32_t on_device);

/*
 * Copy the raw accumulator (npix_y rows of npix uint64): the sum over triangles of
 * round(fraction * 2^32) per pixel.  Integer sums make it bit-identical from
 * run to run.  Same on_device rule as mm_get_map.
 */
mm_status mm_get_map_fixed(const mm_map *h, uint64_t *out, int32_t on_device);

/*
 * Deflection probe: source positions w (interleaved, n points) of image-plane
 * points z (interleaved), evaluated by the same device code the map uses.
 * Host pointers; synchronous.  FMM mode: points must lie in the shooting
 * region (others give NaN).  Runs the tree and expansions if mm_run has not.
 */
mm_status mm_shoot_points(mm_map *h, int64_t n, const double *z_xy, double *w_xy);

/* Statistics and derived parameters of the handle and its last run
 * (synchronises the handle's last stream). */
mm_status mm_get_stats(const mm_map *h, mm_stats *out);

/*
 * Plain FP64 map into caller-provided buffers, allocating nothing.  The paper
 * has no counterpart: this serves callers that cannot call cudaMalloc --
 * those that have handed all device memory to their own pool allocator (a
 * library allocation would fail or escape their accounting) and those that
 * cannot accept the device-wide synchronisation a cudaMalloc may imply.
 *
 * Computes the same map as mm_create(mode = MM_PLAIN_FP64, explicit ray
 * grid) + mm_run + mm_get_map(on_device = 1): direct FP64 sum over every star
 * for each ray vertex, then inverse polygon mapping, on `stream`.  The call
 * returns once the map is complete: it synchronises `stream` to read the
 * kernels' error word, and returns MM_ECUDA (map_out not valid) when a
 * kernel reported an error (the MM_DEBUG build's index checks).
 *
 *   kappa_tot, shear, smooth_fraction: as in mm_create.
 *   masses[n_stars], pos_xy[2*n_stars]: DEVICE pointers of the current
 *     device (or managed memory), interleaved (x, y).  Host pointers and
 *     other devices' buffers are rejected with MM_EINVAL before any work.
 *   half_length, npix, center_y[2] (host, may be NULL = origin): the map.
 *   ray_grid[2] (host): rays per axis; grid_origin[2], grid_spacing[2]
 *     (host): image-plane position of vertex (0, 0) and the ray spacings,
 *     e.g. mm_params.n, .x0 and .h of an equivalent handle.
 *   map_out: DEVICE pointer of the current device, npix*npix floats,
 *     row-major, row = y (square maps only).
 *
 * Scratch lives in one fixed device array inside the library (about 9.5 MB,
 * held by every GPU that loads it until the process exits), so sizes are
 * bounded: n_stars <= 16384, npix <= 256, ray_grid[0]*ray_grid[1] <= 2^19;
 * larger requests return MM_EINVAL with a message and do nothing.  The first
 * call on each device looks up that array's device address (with the device
 * current) and keeps it for the life of the process; make that first call
 * before any stream capture.  cudaDeviceReset() on a device invalidates the
 * kept address: do not call this entry point on a device after resetting it.  All calls share
 * the array and each call clears what it accumulates, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race and
 * corrupt each other's maps: serialise them.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 */
mm_status mm_map_plain_fp64_noalloc(double kappa_tot, double shear, double smooth_fraction,
                                    int64_t n_stars, const double *masses, const double *pos_xy,
                                    double half_length, int32_t npix, const double *center_y,
                                    const int64_t *ray_grid, const double *grid_origin,
                                    const double *grid_spacing, float *map_out, void *stream);

/*
 * Measured peaks for the rooflines of this library's kernels (the paper has
 * no counterpart).  Each kind is a short microbenchmark on the current
 * device: one warm-up launch, then the best of three launches timed with
 * CUDA events on `stream` (synchronous).
 *   MM_PEAK_FP32_FMA:  8 independent fmaf chains per thread, 8 blocks of 256
 *                      threads per SM; *value in TFLOP/s (2 flops per FMA).
 *   MM_PEAK_FP64_FMA:  the same in double; TFLOP/s.
 *   MM_PEAK_L2_RED_U64: each thread adds 1 to 2048 scattered 64-bit words of
 *                      a 32 MiB array (L2-resident) with an atomic add whose
 *                      result is unused, the form of the map's fixed-point
 *                      accumulation; *value in 1e9 reductions per second.
 *   MM_PEAK_L2_RED_U64_ROWS: the same, but a warp's 32 lanes add to 32
 *                      consecutive words at a scattered position (a pixel
 *                      row's pixels dealt across a warp).
 * ms (may be NULL) receives the timed launch's duration.  The call allocates
 * (and frees) its 32 MiB array with cudaMalloc.
 */
typedef enum {
  MM_PEAK_FP32_FMA = 0,
  MM_PEAK_FP64_FMA = 1,
  MM_PEAK_L2_RED_U64 = 2,
  MM_PEAK_L2_RED_U64_ROWS = 3
} mm_peak_kind;

mm_status mm_measure_peak(int32_t kind, double *value, double *ms, void *stream);

/* Thread-local message describing the last failed call ("" if none). */
const char *mm_last_error(void);

/* Release the handle and all its device memory.  NULL is accepted. */
void mm_destroy(mm_map *h);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
