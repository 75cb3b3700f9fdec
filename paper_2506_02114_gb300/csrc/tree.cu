// Adaptive quadtree on the device (Sec. 3.3 and App. C.1).
//
// The root is the square [-R0, R0)^2 centred on the origin.  A node splits
// into four children when the stars in the node and its same-level
// neighbour cells (those sharing a side or a corner) exceed leaf_size.  With
// this rule a split node's eight same-level neighbours always exist, every
// leaf's near field (itself, its same-level neighbours and the adjacent
// leaves one level up) holds at most leaf_size stars, and the interaction
// lists of App. C.2 are exact: at most 27 same-level nodes and at most 5
// leaves one level up.
//
// Build: Morton keys of the stars (21 bits per axis), a radix sort, then one
// level at a time: split flags from nine key-range counts per node, an
// exclusive scan of the flags, and the children written in Morton order so
// that each level's node array stays sorted by code.
#include <cub/cub.cuh>

#include "mm_kernels.h"

namespace mm {

__device__ __forceinline__ int cell_of(double x, double R0) {
  const double scale = (double)(1 << MM_DMAX) / (2.0 * R0);
  double c = floor(__dmul_rn(__dadd_rn(x, R0), scale));
  c = fmin(fmax(c, 0.0), (double)((1 << MM_DMAX) - 1));
  return (int)c;
}

__global__ void k_star_keys(const double *__restrict__ pos, int64_t n, double R0,
                            uint64_t *keys, int32_t *idx) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int cx = cell_of(pos[2 * t], R0), cy = cell_of(pos[2 * t + 1], R0);
  keys[t] = morton2((uint32_t)cx, (uint32_t)cy);
  idx[t] = (int32_t)t;
}

__global__ void k_gather_stars(const double *__restrict__ pos, const double *__restrict__ m,
                               const int32_t *__restrict__ idx, int64_t n, double *sx,
                               double *sy, double *sm) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int32_t k = idx[t];
  sx[t] = pos[2 * k];
  sy[t] = pos[2 * k + 1];
  sm[t] = m[k];
}

__global__ void k_root_init(int64_t n_stars, uint64_t *code, int32_t *lvl, int32_t *sbeg,
                            int32_t *send) {
  code[0] = 0;
  lvl[0] = 0;
  sbeg[0] = 0;
  send[0] = (int32_t)n_stars;
}

// Number of stars whose key lies in the level-`level` cell (x, y).
__device__ __forceinline__ int64_t count_cell(const TreeDev &T, int level, int x, int y) {
  const int sh = 2 * (MM_DMAX - level);
  uint64_t c = morton2((uint32_t)x, (uint32_t)y);
  uint64_t lo = c << sh, hi = (c + 1) << sh;
  int64_t a = lower_bound_u64(T.keys, 0, T.n_stars, lo);
  int64_t b = lower_bound_u64(T.keys, a, T.n_stars, hi);
  return b - a;
}

__global__ void k_level_split(TreeDev T, int level, int64_t n, int limit, int32_t *split) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t node = T.level_off[level] + t;
  if (level >= MM_DMAX) {
    split[t] = 0;
    return;
  }
  uint32_t cx, cy;
  morton_decode(T.code[node], cx, cy);
  const int side = 1 << level;
  int64_t count = T.send[node] - T.sbeg[node];
  for (int dy = -1; dy <= 1; dy++)
    for (int dx = -1; dx <= 1; dx++) {
      if (dx == 0 && dy == 0) continue;
      int x = (int)cx + dx, y = (int)cy + dy;
      if (x < 0 || y < 0 || x >= side || y >= side) continue;
      count += count_cell(T, level, x, y);
    }
  split[t] = count > limit ? 1 : 0;
}

__global__ void k_level_children(TreeDev T, int level, int64_t n, const int32_t *split,
                                 const int32_t *scan, uint64_t *code, int32_t *lvl,
                                 int32_t *sbeg, int32_t *send, int32_t *first_child) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t node = T.level_off[level] + t;
  if (!split[t]) {
    first_child[node] = -1;
    return;
  }
  const int64_t base = T.level_off[level + 1] + 4 * (int64_t)scan[t];
  first_child[node] = (int32_t)base;
  const uint64_t c = T.code[node];
  const int sh = 2 * (MM_DMAX - level - 1);
  int64_t b = T.sbeg[node];
  const int64_t e = T.send[node];
  for (int q = 0; q < 4; q++) {
    uint64_t cc = (c << 2) | (uint64_t)q;
    int64_t end = (q == 3) ? e : lower_bound_u64(T.keys, b, e, (cc + 1) << sh);
    code[base + q] = cc;
    lvl[base + q] = level + 1;
    sbeg[base + q] = (int32_t)b;
    send[base + q] = (int32_t)end;
    b = end;
  }
}

__global__ void k_axis_cells(double x0, double h, int64_t n, double R0, int32_t *out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double x = __dadd_rn(x0, __dmul_rn((double)t, h));
  out[t] = cell_of(x, R0);
}

__global__ void k_active_flags(TreeDev T, int64_t n_nodes, const int32_t *col_cell,
                               int64_t col_lo, int64_t col_hi, const int32_t *row_cell,
                               int64_t row_lo, int64_t row_hi, int32_t *node_act,
                               int32_t *leaf_flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes) return;
  const int CX0 = col_cell[col_lo], CX1 = col_cell[col_hi];
  const int CY0 = row_cell[row_lo], CY1 = row_cell[row_hi];
  uint32_t cx, cy;
  morton_decode(T.code[t], cx, cy);
  const int sh = MM_DMAX - T.lvl[t];
  const int64_t x0 = (int64_t)cx << sh, x1 = (((int64_t)cx + 1) << sh) - 1;
  const int64_t y0 = (int64_t)cy << sh, y1 = (((int64_t)cy + 1) << sh) - 1;
  const int act = (x1 >= CX0 && x0 <= CX1 && y1 >= CY0 && y0 <= CY1) ? 1 : 0;
  node_act[t] = act;
  leaf_flag[t] = (act && T.first_child[t] < 0) ? 1 : 0;
}

__global__ void k_compact_leaves(int64_t n_nodes, const int32_t *leaf_flag,
                                 const int32_t *leaf_scan, int32_t *node_active,
                                 int32_t *active_list) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes) return;
  if (leaf_flag[t]) {
    node_active[t] = leaf_scan[t];
    active_list[leaf_scan[t]] = (int32_t)t;
  } else {
    node_active[t] = -1;
  }
}

// Lookup grid over the active region at level glevel: the active leaf
// covering each cell, or -(node + 1) for a split node at glevel.
// Grid cell (gx, gy) of level glevel: the sub-cell record of the active leaf
// containing it when the leaf is at least `sub` levels coarser (the cell then
// lies in one sub-cell), else -(node + 1) for the node where the device walk
// continues.
__global__ void k_lookup_grid(TreeDev T, const int32_t *node_active, int glevel, int sub,
                              int gx0, int gy0, int gw, int gh, int32_t *grid) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)gw * gh) return;
  const int gx = gx0 + (int)(t % gw), gy = gy0 + (int)(t / gw);
  int node = 0, l = 0;
  for (; l < glevel; l++) {
    int fc = T.first_child[node];
    if (fc < 0) break;
    int sh = glevel - l - 1;
    node = fc + (((gx >> sh) & 1) | (((gy >> sh) & 1) << 1));
  }
  const int a = (T.first_child[node] < 0) ? node_active[node] : -1;
  if (a >= 0 && l + sub <= glevel) {
    const int sh = glevel - l - sub, mask = (1 << sub) - 1;
    grid[t] = (a << (2 * sub)) + (((gy >> sh) & mask) << sub) + ((gx >> sh) & mask);
  } else {
    grid[t] = -(node + 1);
  }
}

static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_star_keys(const double *pos, int64_t n, double R0, uint64_t *keys,
                             int32_t *idx, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_star_keys<<<blocks_for(n, 256), 256, 0, st>>>(pos, n, R0, keys, idx);
  return cudaGetLastError();
}

cudaError_t launch_gather_stars(const double *pos, const double *m, const int32_t *idx,
                                int64_t n, double *sx, double *sy, double *sm,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather_stars<<<blocks_for(n, 256), 256, 0, st>>>(pos, m, idx, n, sx, sy, sm);
  return cudaGetLastError();
}

cudaError_t launch_root_init(int64_t n_stars, uint64_t *code, int32_t *lvl, int32_t *sbeg,
                             int32_t *send, cudaStream_t st) {
  k_root_init<<<1, 1, 0, st>>>(n_stars, code, lvl, sbeg, send);
  return cudaGetLastError();
}

cudaError_t launch_level_split(const TreeDev &T, int level, int64_t n, int limit,
                               int32_t *split, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_level_split<<<blocks_for(n, 128), 128, 0, st>>>(T, level, n, limit, split);
  return cudaGetLastError();
}

cudaError_t launch_level_children(const TreeDev &T, int level, int64_t n, const int32_t *split,
                                  const int32_t *scan, uint64_t *code, int32_t *lvl,
                                  int32_t *sbeg, int32_t *send, int32_t *first_child,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_level_children<<<blocks_for(n, 128), 128, 0, st>>>(T, level, n, split, scan, code, lvl,
                                                       sbeg, send, first_child);
  return cudaGetLastError();
}

cudaError_t launch_axis_cells(double x0, double h, int64_t n, double R0, int32_t *out,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_axis_cells<<<blocks_for(n, 256), 256, 0, st>>>(x0, h, n, R0, out);
  return cudaGetLastError();
}

cudaError_t launch_active_flags(const TreeDev &T, int64_t n_nodes, const int32_t *col_cell,
                                int64_t col_lo, int64_t col_hi, const int32_t *row_cell,
                                int64_t row_lo, int64_t row_hi, int32_t *node_act,
                                int32_t *leaf_flag, cudaStream_t st) {
  if (n_nodes <= 0) return cudaSuccess;
  k_active_flags<<<blocks_for(n_nodes, 256), 256, 0, st>>>(T, n_nodes, col_cell, col_lo, col_hi,
                                                           row_cell, row_lo, row_hi, node_act,
                                                           leaf_flag);
  return cudaGetLastError();
}

cudaError_t launch_compact_leaves(int64_t n_nodes, const int32_t *leaf_flag,
                                  const int32_t *leaf_scan, int32_t *node_active,
                                  int32_t *active_list, cudaStream_t st) {
  if (n_nodes <= 0) return cudaSuccess;
  k_compact_leaves<<<blocks_for(n_nodes, 256), 256, 0, st>>>(n_nodes, leaf_flag, leaf_scan,
                                                             node_active, active_list);
  return cudaGetLastError();
}

cudaError_t launch_lookup_grid(const TreeDev &T, const int32_t *node_active, int glevel,
                               int sub, int gx0, int gy0, int gw, int gh, int32_t *grid,
                               cudaStream_t st) {
  int64_t n = (int64_t)gw * gh;
  if (n <= 0) return cudaSuccess;
  k_lookup_grid<<<blocks_for(n, 256), 256, 0, st>>>(T, node_active, glevel, sub, gx0, gy0, gw,
                                                    gh, grid);
  return cudaGetLastError();
}

}  // namespace mm
