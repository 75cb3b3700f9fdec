// Host-side launchers of the libmm kernels (one declaration per kernel
// family; definitions live next to the kernels).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "mm_common.cuh"

namespace mm {

// Message returned by mm_last_error on this thread (api.cu).
void set_last_error(const char *msg);

// ---- tree (tree.cu) --------------------------------------------------------
struct TreeDev {
  // sorted stars (Morton order), SoA, FP64
  const uint64_t *keys;
  const double *sx, *sy, *sm;
  int64_t n_stars;
  double R0;                  // root half-length (power of two)
  // nodes (flattened over levels)
  const uint64_t *code;
  const int32_t *lvl, *sbeg, *send, *first_child;
  const int64_t *level_off;   // [MM_DMAX + 2]
  int32_t depth;
};

cudaError_t launch_star_keys(const double *pos, int64_t n, double R0, uint64_t *keys,
                             int32_t *idx, cudaStream_t st);
cudaError_t launch_gather_stars(const double *pos, const double *m, const int32_t *idx,
                                int64_t n, double *sx, double *sy, double *sm,
                                cudaStream_t st);
cudaError_t launch_root_init(int64_t n_stars, uint64_t *code, int32_t *lvl, int32_t *sbeg,
                             int32_t *send, cudaStream_t st);
cudaError_t launch_level_split(const TreeDev &T, int level, int64_t n, int limit,
                               int32_t *split, cudaStream_t st);
cudaError_t launch_level_children(const TreeDev &T, int level, int64_t n, const int32_t *split,
                                  const int32_t *scan, uint64_t *code, int32_t *lvl,
                                  int32_t *sbeg, int32_t *send, int32_t *first_child,
                                  cudaStream_t st);
cudaError_t launch_axis_cells(double x0, double h, int64_t n, double R0, int32_t *out,
                              cudaStream_t st);
// flags[node] = 1 for active leaves (leaf containing ray vertices); also
// node_act[node] = 1 for every active node
cudaError_t launch_active_flags(const TreeDev &T, int64_t n_nodes, const int32_t *col_cell,
                                int64_t col_lo, int64_t col_hi, const int32_t *row_cell,
                                int64_t row_lo, int64_t row_hi, int32_t *node_act,
                                int32_t *leaf_flag, cudaStream_t st);
cudaError_t launch_compact_leaves(int64_t n_nodes, const int32_t *leaf_flag,
                                  const int32_t *leaf_scan, int32_t *node_active,
                                  int32_t *active_list, cudaStream_t st);
cudaError_t launch_lookup_grid(const TreeDev &T, const int32_t *node_active, int glevel,
                               int sub, int gx0, int gy0, int gw, int gh, int32_t *grid,
                               cudaStream_t st);

// ---- expansions (fmm.cu) ---------------------------------------------------
struct FmmConst {
  int p;                      // expansion order of the FMM
  int p_eval;                 // terms kept of each sub-cell's re-centred expansion
  int sub;                    // sub-cell levels s: 4^s sub-cells per leaf
  int npix, npix_y;           // map pixels along x and y (culling bounds)
  int cull;                   // 1: compute the culling bounds
  double kappa, gamma, kappa_star;
  double x0, y0, hx, hy;      // ray grid
  double x1, y1;              // the grid's last vertex
  double lox, loy, delta;     // map lower-left corner and pixel side
  double rect_c1, rect_c2;    // > 0: rectangular star region |x| <= c1, |y| <= c2 (App. B)
};

cudaError_t launch_p2m(const TreeDev &T, int64_t n_nodes, int p, double2 *mp, cudaStream_t st);
cudaError_t launch_m2m(const TreeDev &T, int level, int64_t n, int p, const double2 *MMop,
                       double2 *mp, cudaStream_t st);
cudaError_t launch_local(const TreeDev &T, int level, int64_t n, int p, const int32_t *node_act,
                         const double2 *MLop, const double2 *LLop, const double2 *mp,
                         double2 *loc, unsigned *err, cudaStream_t st);
cudaError_t launch_near_count(const TreeDev &T, const FmmConst &C, int64_t n_active,
                              const int32_t *active_list, int32_t *near_cnt, unsigned *err,
                              cudaStream_t st);
cudaError_t launch_leaf_finalize(const TreeDev &T, const FmmConst &C, int64_t n_active,
                                 const int32_t *active_list, const int32_t *near_off,
                                 const int32_t *near_cnt,
                                 const double2 *loc, LeafRec *leaf, NearPos *near_pos,
                                 float *near_m, float2 *coef, unsigned *err, cudaStream_t st);
void build_operator_tables(int p, std::vector<double2> &MM, std::vector<double2> &ML,
                           std::vector<double2> &LL);

// ---- shooting + mapping (shoot.cu) -----------------------------------------
// The second pass over the map's queued larger triangles (no-op without a queue).
// dst[i] = *src[i] with work_begin[i], on the device (n descriptors)
cudaError_t launch_batch_gather(const MapDev *const *src, const int64_t *work_begin, int n,
                                MapDev *dst, int &launches, cudaStream_t st);
// inverse ray shooting of one map's work items (no second pass)
cudaError_t launch_shoot_irs(const MapDev &m, int64_t total_work, bool square,
                             unsigned long long *counter, unsigned *err, cudaStream_t st);
cudaError_t launch_big_ipm(const MapDev &m, cudaStream_t st);
// h_single: the map by value when n_maps == 1 (else NULL: maps from d_maps)
cudaError_t launch_shoot_ipm(const MapDev *d_maps, const MapDev *h_single, int n_maps,
                             int64_t total_work, bool square,
                             unsigned long long *counter, unsigned *err, int grid,
                             cudaStream_t st);
cudaError_t launch_normalize(const unsigned long long *acc, const unsigned long long *span,
                             int npix, int npix_y, double scale, float *out, cudaStream_t st);
// out[k] = acc[k] * scale for n fixed-point values (the normalisation of an
// accumulator already folded with its row-difference array)
cudaError_t launch_scale_fixed(const unsigned long long *acc, int64_t n, double scale,
                               float *out, cudaStream_t st);
cudaError_t launch_fold_span(unsigned long long *acc, const unsigned long long *span, int npix,
                             int npix_y,
                             unsigned long long *out, cudaStream_t st);
cudaError_t launch_probe(const MapDev *d_maps, bool square, int64_t n, const double *z,
                         double *w, double x0, double y0, double hx, double hy, double R0,
                         double lox, double loy, double delta, unsigned *err, cudaStream_t st);

// ---- plain FP64 path (direct64.cu) -----------------------------------------
struct DirectConst {
  double kappa, gamma, kappa_star;
  double x0, y0, hx, hy;
  double lox, loy, delta;
  double rect_c1, rect_c2;    // > 0: rectangular star region (App. B); 0: disk
};
// vertices of columns [col0, col0 + width) and rows [row_lo, row_hi], row-major
cudaError_t launch_direct64_vertices(const double *sx, const double *sy, const double *sm,
                                     int64_t n_stars, const DirectConst &C, int64_t col0,
                                     int64_t width, int64_t row_lo, int64_t row_hi, Vtx *out,
                                     cudaStream_t st);
cudaError_t launch_direct64_points(const double *sx, const double *sy, const double *sm,
                                   int64_t n_stars, const DirectConst &C, int64_t n,
                                   const double *z, double *w, cudaStream_t st);
cudaError_t launch_ipm_vertices(const MapDev *d_map, const Vtx *verts, int64_t width,
                                int64_t row_lo, int64_t row_hi, unsigned long long *counter,
                                unsigned *err, int grid, cudaStream_t st);

}  // namespace mm
