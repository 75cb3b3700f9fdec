// Shared device-side types and helpers of the libmm CUDA path (sm_103a).
//
// Coordinates: theta_star = 1.  The quadtree root is the square
// [-R0, R0)^2 with R0 a power of two, so every cell edge at every level is an
// exact binary fraction.  Cell indices at the finest level MM_DMAX are 21-bit
// integers; a level-l cell index is the finest index shifted right by
// (MM_DMAX - l).  Morton codes interleave x (even bits) and y (odd bits).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MM_DMAX 21            // deepest quadtree level
#define MM_PMAX 64            // largest expansion order accepted by the ABI
#define MM_SUB_MAX 2          // largest sub-cell level count (16 sub-cells per leaf)
#define MM_SUB_DEFAULT 2      // sub-cell levels when the options leave it to the library
#define MM_NEAR_K 2           // with sub-cells, a sub-cell sums directly the leaf's near
                              // stars in its (2K+1)^2 block of sub-cells; the rest go
                              // into its local expansion
#define MM_STRIP 31           // cell columns per warp work item (32 vertex columns)
#define MM_MED_PIXELS 64      // bounding box (map pixels) up to which a larger
                              // triangle is counted as medium in the statistics

namespace mm {

// Error word bits written by kernels (read back by the host).
enum : unsigned int {
  ERR_TREE_INVARIANT = 1u,    // a split node lacks a same-level neighbour
  ERR_LOOKUP = 2u,            // a ray vertex fell outside every active leaf
  ERR_RECT_CORNER = 4u,       // a record's rectangular-sheet series converges too
                              // slowly (a star-rectangle corner is near it)
  ERR_BOUNDS = 8u,            // MM_DEBUG builds: a map or row-difference index out of
                              // range (the access was skipped)
};

// Per sub-cell of an active leaf: everything a ray vertex in it needs (64
// bytes).  Each active leaf t owns the 4^s records [4^s t, 4^s (t + 1)), one
// per sub-cell of side 2 L / 2^s (s = MapDev::sub, row-major, y major); the
// leaf's local expansion is re-centred on each sub-cell.  Positions are
// measured in ray-grid units from the grid vertex (i_ref, j_ref) closest to
// the sub-cell centre, which sits at (i_ref + fcx, j_ref + fcy).
struct __align__(16) LeafRec {
  int32_t i_ref, j_ref;
  float fcx, fcy;
  int32_t Ui, Vi;             // integer part of the centre's image in pixels
  float Uf, Vf;               // fractional part (FP64-accurate)
  float zsx, zsy;             // h_x / L_s, h_y / L_s : grid units -> zeta units
  int32_t near_off, near_cnt; // the sub-cell's direct-sum stars in near_pos/near_m
  int32_t coef_off;           // first of coef_stride(p_eval) far-field coefficient slots
  int32_t node;               // tree node id of the leaf
  // Culling: every vertex of the sub-cell whose squared distance |g|^2 (grid
  // units, as the near field measures it) to each direct star exceeds
  // cull_r2 lands beyond map edge cull_side (MM_CULL_*); 0: no guarantee.
  int32_t cull_side;
  float cull_r2;
};

// Map edges a culled vertex lies beyond.
enum { MM_CULL_NONE = 0, MM_CULL_LEFT = 1, MM_CULL_RIGHT = 2, MM_CULL_BOTTOM = 3, MM_CULL_TOP = 4 };

// Direct-sum star in its record's grid frame: grid position relative to
// (i_ref, j_ref) = (Kx + fx, Ky + fy), K integer-valued, |f| <= 0.5.
struct __align__(16) NearPos {
  float Kx, fx, Ky, fy;
};

// A mapped ray vertex in canonical pixel form: integer pixel plus the
// position inside it; px == INT_MIN marks a non-finite vertex.
struct __align__(16) Vtx {
  int px, py;
  float fx, fy;
};

struct TriJob;  // a triangle larger than 2 x 2 pixels (ipm.cuh)
#define MM_TRIJOB_BYTES 48

// Everything the deflection + mapping kernel needs about one map.
struct MapDev {
  // ray grid
  int64_t n0, n1;             // vertices per axis
  int64_t row_begin, row_end; // cell rows [row_begin, row_end)
  int64_t col_begin, col_end; // cell columns [col_begin, col_end)
  int32_t strips, rows_per_item;
  int64_t row_blocks;
  int64_t item_stride;        // >= 1: work item k covers row block k * item_stride
                              // (> 1 only for the autotuner's sampled runs)
  int64_t work_begin;         // first global work item of this map
  // leaf lookup
  const int32_t *col_cell, *row_cell;   // finest-level cell index per vertex column / row
  const int32_t *grid;                  // lookup grid: sub-cell record id, or -(node+1)
  int32_t glevel, gshift, gx0, gy0, gw, gh;
  const int32_t *first_child;           // per node: first child id, -1 for a leaf
  const int32_t *node_active;           // per node: active leaf id or -1
  const int32_t *node_level;            // per node: tree level
  int32_t sub;                          // sub-cell levels s (4^s records per leaf)
  // leaves
  const LeafRec *leaf;
  const NearPos *near_pos;
  const float *near_m;
  const float2 *coef;
  int32_t p;                  // terms of the re-centred expansion evaluated per ray
  int32_t cull;               // 1: skip the deflection of vertex rows proven beyond the map
  int32_t square_cells;       // 1 when h_x == h_y
  // per-ray constants (pixel units)
  float A1, A2;               // (1 - kappa + kappa_star +- gamma) h / delta
  float sx, sy;               // 1/(h_x delta), h_y/(h_x^2 delta)
  float rho;                  // (h_y/h_x)^2
  float crit_area2;           // 2 x source triangle area (px^2) below which the
                              // triangle counts as near-critical
  // map
  int32_t npix, npix_y;       // pixels along x (row length) and y (rows)
  unsigned *err;              // the handle's error word
  unsigned long long *acc;    // npix_y*npix fixed point, 2^32 = one triangle
  unsigned long long *span;   // npix_y*(npix+1) row difference array
  // statistics (per map)
  unsigned long long *stat;   // triangle counters, see IpmCounters
  // larger triangles handed to the second kernel (capacity 0: none)
  TriJob *bigq;
  unsigned long long *bigq_n; // [0] triangles queued, [1] the second kernel's batch counter
  int64_t bigq_cap;
};

// Far-field coefficient slots per sub-cell record: the p_eval - 1
// coefficients rounded up to an even count (>= 2), loaded as float4 pairs.
__host__ __device__ __forceinline__ int coef_stride(int p_eval) {
  return p_eval <= 2 ? 2 : ((p_eval - 1 + 1) & ~1);
}

// Interleave two 21-bit integers: x in even bits, y in odd bits.
__host__ __device__ __forceinline__ uint64_t morton2(uint32_t x, uint32_t y) {
  uint64_t r = 0;
#pragma unroll
  for (int b = 0; b < MM_DMAX; b++) {
    r |= (uint64_t)((x >> b) & 1u) << (2 * b);
    r |= (uint64_t)((y >> b) & 1u) << (2 * b + 1);
  }
  return r;
}

__host__ __device__ __forceinline__ void morton_decode(uint64_t c, uint32_t &x, uint32_t &y) {
  x = 0;
  y = 0;
#pragma unroll
  for (int b = 0; b < MM_DMAX; b++) {
    x |= (uint32_t)((c >> (2 * b)) & 1u) << b;
    y |= (uint32_t)((c >> (2 * b + 1)) & 1u) << b;
  }
}

// First index in [lo, hi) with a[idx] >= key (a sorted ascending).
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t lo, int64_t hi,
                                                   uint64_t key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Smooth sheet of a rectangular star region (App. B).  For the sheet of
// convergence -kappa_star on |x| <= c1, |y| <= c2 and a point z inside it,
// alpha_s(z) = -kappa_star z + A(z) with
//   A(z)  = (-kappa_star i / pi) F(conj z) - kappa_star (2 c1 + conj z),
//   F(t)  = f_c(t) - f_cb(t) + f_-c(t) - f_-cb(t),   f_a(t) = (a - t) log(a - t),
// c = c1 + i c2, cb = conj c, principal logarithms (no branch cut meets the
// interior).  A depends on conj z alone, so At(z) = conj A(z) is analytic
// inside:  At(z) = (kappa_star i / pi) G(z) - kappa_star (2 c1 + z) with
// G = f_cb - f_c + f_-cb - f_-c; the -kappa_star z part stays in the macro
// factor 1 - kappa + kappa_star, exactly as for a star disk.
// ---------------------------------------------------------------------------

// the four corners a of G and their signs: cb (+), c (-), -cb (+), -c (-)
__device__ __forceinline__ void rect_corner(double c1, double c2, int k, double &ax, double &ay,
                                            double &sgn) {
  ax = (k < 2) ? c1 : -c1;
  ay = (k & 1) ? c2 : -c2;
  if (k >= 2) ay = -ay;  // -cb = -c1 + i c2, -c = -c1 - i c2
  sgn = (k & 1) ? -1.0 : 1.0;
}

// principal log of x + i y
__device__ __forceinline__ double2 clog64(double x, double y) {
  return make_double2(log(hypot(x, y)), atan2(y, x));
}

// At(z) inside the rectangle (the value; A(z) = conj of it)
__device__ __forceinline__ double2 rect_sheet_At(double ks, double c1, double c2, double x,
                                                 double y) {
  double gx = 0.0, gy = 0.0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    double ax, ay, sg;
    rect_corner(c1, c2, k, ax, ay, sg);
    const double dx = ax - x, dy = ay - y;  // a - z
    const double2 l = clog64(dx, dy);
    gx += sg * (dx * l.x - dy * l.y);
    gy += sg * (dx * l.y + dy * l.x);
  }
  const double f = ks / 3.14159265358979323846;  // (kappa_star i / pi) G
  return make_double2(-f * gy - ks * (2.0 * c1 + x), f * gx - ks * y);
}

}  // namespace mm
