// Inverse polygon mapping on the device (Sec. 3.2, Fig. 3): a mapped
// triangle's unit of flux is split among the pixels it covers in proportion
// to area(T n pixel) / |area(T)|.  Each share is rounded to a multiple of
// 2^-32 triangle and summed as an integer in a uint64 map, so sums are exact
// and independent of the order of the atomics.
//
// Vertices arrive in a canonical pixel form (integer pixel + fraction in
// [0, 1)) that does not depend on which warp computed them, so the two
// triangles sharing an edge see bit-identical edge geometry.  A triangle is
// processed in the frame of its first vertex's pixel, where FP32 coordinates
// of small triangles are exact to ~1e-7 pixel.
//
// Area of T inside a box.  Projecting the plane onto a closed box B by
// clamping, (x, y) -> (clamp(x, B), clamp(y, B)), maps T's boundary to a
// closed curve in B that winds around every interior point of B exactly as
// often as T's boundary does (a horizontal ray from such a point meets both
// curves in the same signed crossings) and around no point outside B, so the
// shoelace sum of the projected boundary is area(T n B).  Each edge is cut
// where it crosses the box's lines, so every projected piece is straight.
// With the box translated to [0, 1]^2 every term is O(1): no cancellation,
// no polygon arrays, everything in registers.  The same identity with a
// quadrant (x < X, y < Y) gives the three areas that split a triangle
// covering a 2 x 2 pixel box; for a pixel of a larger triangle the shoelace
// sum is taken edge by edge as the integral of the clamped x over the
// clamped y.  These are exactly the areas that the column-then-row
// Sutherland-Hodgman clipping of Fig. 3 produces.
//
// Paths:
//   * the triangle lies inside one pixel (the common case at ~100 rays per
//     pixel): that pixel gains exactly 2^32;
//   * it spans two pixels split by one grid line: the vertex alone on its
//     side cuts off a similar triangle whose area fraction is a product of
//     two edge parameters, finished here;
//   * it spans 2 x 2 pixels: queued per warp in shared memory and
//     apportioned 32 at a time from three quadrant areas by
//     inclusion-exclusion;
//   * larger (cells next to a star map to triangles up to hundreds of
//     pixels wide; cells along a caustic to long slivers): queued per warp;
//     the pixel rows of 32 such triangles are dealt out to the lanes, each
//     row adds the constant 1/|area| to its run of fully covered pixels
//     through a per-row difference array, and the partially covered pixels
//     of those rows are then dealt out one per lane and measured from the
//     row's edge pieces (row_pieces, piece_mean).  Work is proportional to
//     the perimeter, not the area, and no lane loops on its own.
#pragma once
#include <climits>

#include "mm_common.cuh"

namespace mm {

#define MM_VTX_INVALID INT_MIN
#define MM_FIX_ONE 4294967296ull  // one whole triangle in fixed-point units

__device__ __forceinline__ float rcp_approx_f(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Share of a triangle in fixed-point units (2^32 = the whole triangle).  An
// FP32 fraction carries 24 significant bits, so it is rounded at 2^-24 and
// shifted: 32-bit conversions only (64-bit ones would run on the FP64 pipe).
__device__ __forceinline__ unsigned long long frac_to_fixed(float f) {
  f = __saturatef(f);  // clamp to [0, 1] (NaN -> 0)
  return (unsigned long long)__float2uint_rn(f * 16777216.0f) << 8;
}

// ---------------------------------------------------------------------------
// accumulation
// ---------------------------------------------------------------------------

// MM_DEBUG builds check every accumulator and row-difference index against
// its array before the atomic and, out of range, skip the access and set
// ERR_BOUNDS in the error word (read back through mm_get_stats).  Other
// builds compile the check to nothing.
#ifdef MM_DEBUG
__device__ __forceinline__ bool mm_index_ok(unsigned *err, long long idx, long long n) {
  if (idx >= 0 && idx < n) return true;
  atomicOr(err, ERR_BOUNDS);
  return false;
}
#define MM_INDEX_OK(err, idx, n) mm_index_ok((err), (long long)(idx), (long long)(n))
#else
#define MM_INDEX_OK(err, idx, n) true
#endif

// Add v fixed-point units to map pixel (gx, gy) if it lies in the map
// (pixel indices stay within +-2^30: vertices are clamped to +-2^28 pixels
// about their sub-cell's centre image, and boxes to +-1e9 of a vertex).
__device__ __forceinline__ void deposit(const MapDev &M, int gx, int gy, unsigned long long v) {
  if (v && gx >= 0 && gx < M.npix && gy >= 0 && gy < M.npix_y &&
      MM_INDEX_OK(M.err, (long long)gy * M.npix + gx, (long long)M.npix * M.npix_y))
    atomicAdd(&M.acc[(long long)gy * M.npix + gx], v);
}

// The map's accumulators alone, passed as scalars to the out-of-line row
// and pixel dealing (so the kernel's MapDev, a launch parameter, is never
// copied to local memory to be addressed).
struct MapAcc {
  unsigned long long *acc, *span;
  int npix, npix_y;
  unsigned *err;
};

// Lane-private run accumulator: consecutive one-pixel triangles of a lane's
// column usually hit the same pixel; they are summed in a register.
struct RunAcc {
  long long idx;  // map index of the pixel being summed, -1 for none
  unsigned long long val;
};

__device__ __forceinline__ void run_flush(const MapDev &M, RunAcc &a) {
  if (a.idx >= 0 && MM_INDEX_OK(M.err, a.idx, (long long)M.npix * M.npix_y))
    atomicAdd(&M.acc[a.idx], a.val);
  a.idx = -1;
  a.val = 0;
}

// Add v to in-map pixel idx.
__device__ __forceinline__ void run_add(const MapDev &M, RunAcc &a, long long idx,
                                        unsigned long long v) {
  if (idx == a.idx) {
    a.val += v;
    return;
  }
  if (a.idx >= 0 && MM_INDEX_OK(M.err, a.idx, (long long)M.npix * M.npix_y))
    atomicAdd(&M.acc[a.idx], a.val);
  a.idx = idx;
  a.val = v;
}

// ---------------------------------------------------------------------------
// areas
// ---------------------------------------------------------------------------

// Split of T by one grid line u = L (u = x or y, coordinates u0, u1, u2):
// the vertex alone on its side cuts off a triangle similar to T, whose
// share of the area is d^2 / ((u_a - u_l)(u_b - u_l)), d = L - u_l (the
// two edge parameters at the line, multiplied).  Returns that share and
// whether the lone vertex lies on the low side u < L.
__device__ __forceinline__ float lone_vertex_share(float u0, float u1, float u2, float L,
                                                   bool &lone_low) {
  const bool b0 = u0 < L, b1 = u1 < L, b2 = u2 < L;
  lone_low = (b0 + b1 + b2) == 1;
  float ul = u2, ua = u0, ub = u1;
  if (b0 == lone_low) {
    ul = u0;
    ua = u1;
    ub = u2;
  } else if (b1 == lone_low) {
    ul = u1;
    ua = u0;
    ub = u2;
  }
  const float d = L - ul;
  return d * d * rcp_approx_f((ua - ul) * (ub - ul));
}

// Fixed-point share of T on the low side u < L of one grid line it crosses.
// The line is chosen from the vertices' integer pixels, and a vertex's FP32
// coordinate in a neighbouring pixel's frame can round onto the line (k + f
// with f within 2^-24 of 1), leaving no vertex strictly below it: then
// nothing of T lies below the line (and all of it when none lies above).
__device__ __forceinline__ unsigned long long low_side_fixed(float u0, float u1, float u2,
                                                             float L) {
  const int nlow = (u0 < L) + (u1 < L) + (u2 < L);
  bool lone_low;
  const float v = lone_vertex_share(u0, u1, u2, L, lone_low);
  const float low = nlow == 0 ? 0.f : (nlow == 3 ? 1.f : (lone_low ? v : 1.f - v));
  return frac_to_fixed(low);
}

// Contribution of edge P -> Q to the signed area of T n {x < X, y < Y}
// (Green's theorem on the boundary clamped to the quadrant): the edge's
// piece below Y, times the mean of min(x - X, 0) over it.  The terms in X
// itself sum to zero around T and are left out.
__device__ __forceinline__ float quadrant_edge(float px, float py, float qx, float qy, float X,
                                               float Y) {
  const float ys = fminf(py, Y), ye = fminf(qy, Y);
  const float xY = fmaf(Y - py, (qx - px) * rcp_approx_f(qy - py), px);  // x on the edge at Y
  const float xs = py <= Y ? px : xY, xe = qy <= Y ? qx : xY;
  const float a = fminf(xs, xe) - X, b = fmaxf(xs, xe) - X;
  const float m = b <= 0.f ? 0.5f * (a + b) : (a >= 0.f ? 0.f : -0.5f * a * a * rcp_approx_f(b - a));
  return ye != ys ? (ye - ys) * m : 0.f;
}

// ---------------------------------------------------------------------------
// triangles within a 2 x 2 pixel box: warp queue
// ---------------------------------------------------------------------------

// Frame pixel (ox, oy), first vertex (x0, y0) inside it, the other two
// relative to the first.
struct __align__(16) SmallTri {
  int ox, oy;
  float x0, y0, d1x, d1y, d2x, d2y;
};

// A triangle across both grid lines of a 2 x 2 pixel block: the shares left
// of X and below Y from the lone vertex on each line, the lower-left share
// from the quadrant integral; the four pixel shares are differences of
// those in fixed point and add up to exactly one triangle.
__device__ __forceinline__ void small_tri_apportion(const MapDev &M, const SmallTri &e) {
  const int c0 = (int)floorf(e.x0 + fminf(0.f, fminf(e.d1x, e.d2x)));
  const int r0 = (int)floorf(e.y0 + fminf(0.f, fminf(e.d1y, e.d2y)));
  // the grid lines, relative to the first vertex
  const float X = (float)(c0 + 1) - e.x0, Y = (float)(r0 + 1) - e.y0;
  const long long vL = (long long)low_side_fixed(0.f, e.d1x, e.d2x, X);
  const long long vB = (long long)low_side_fixed(0.f, e.d1y, e.d2y, Y);
  const float lb = quadrant_edge(0.f, 0.f, e.d1x, e.d1y, X, Y) +
                   quadrant_edge(e.d1x, e.d1y, e.d2x, e.d2y, X, Y) +
                   quadrant_edge(e.d2x, e.d2y, 0.f, 0.f, X, Y);
  const float A2 = e.d1x * e.d2y - e.d2x * e.d1y;  // twice the signed area
  const long long vLB = (long long)frac_to_fixed(2.f * lb * rcp_approx_f(A2));
  const long long one = (long long)MM_FIX_ONE;
  const int gx = e.ox + c0, gy = e.oy + r0;
  deposit(M, gx, gy, (unsigned long long)vLB);
  deposit(M, gx, gy + 1, (unsigned long long)max(vL - vLB, 0ll));
  deposit(M, gx + 1, gy, (unsigned long long)max(vB - vLB, 0ll));
  deposit(M, gx + 1, gy + 1, (unsigned long long)max(one - vL - vB + vLB, 0ll));
}

// A triangle across one grid line of two pixels: the low pixel (gx, gy),
// the line u = L along axis o (0: x, 1: y; the high pixel is the next one
// along that axis) and the triangle's coordinates along that axis.
struct __align__(16) LineTri {
  int gx, gy;
  float u0, u1, u2, L;
  int o, pad;
};

// The two pixels' shares: complements in fixed point, one triangle in all.
__device__ __forceinline__ void line_tri_apportion(const MapDev &M, const LineTri &e) {
  const unsigned long long vlow = low_side_fixed(e.u0, e.u1, e.u2, e.L);
  deposit(M, e.gx, e.gy, vlow);
  deposit(M, e.gx + 1 - e.o, e.gy + e.o, MM_FIX_ONE - vlow);
}

// Per-warp queue of LineTri in shared memory (capacity 64 >= 31 + 31 + 2):
// the two-pixel triangles are shared out 32 at a time, so the warp runs
// their apportioning with every lane busy instead of in a branch that only
// some lanes take (used by the single-map first pass, whose registers allow
// it; elsewhere the triangle is apportioned where it is found).
struct LineQueue {
  LineTri *q;
  int n;
};

__device__ __forceinline__ void lq_push(const MapDev &M, LineQueue &lq, bool want,
                                        const LineTri &e, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int pos = lq.n + __popc(m & ((1u << lane) - 1u));
  if (want) lq.q[pos] = e;
  lq.n += __popc(m);
  __syncwarp();
  while (lq.n >= 32) {
    const LineTri t = lq.q[lq.n - 32 + lane];
    __syncwarp();
    lq.n -= 32;
    line_tri_apportion(M, t);
  }
}

__device__ __forceinline__ void lq_drain(const MapDev &M, LineQueue &lq, int lane) {
  if (lq.n > 0) {
    LineTri t;
    const bool have = lane < lq.n;
    if (have) t = lq.q[lane];
    __syncwarp();
    if (have) line_tri_apportion(M, t);
    lq.n = 0;
  }
  __syncwarp();
}

// Per-warp queue of SmallTri in shared memory (capacity 64 >= 31 + 31 + 2).
struct WarpQueue {
  SmallTri *q;
  int n;
};

__device__ __forceinline__ void wq_push(const MapDev &M, WarpQueue &wq, bool want,
                                        const SmallTri &e, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int pos = wq.n + __popc(m & ((1u << lane) - 1u));
  if (want) wq.q[pos] = e;
  wq.n += __popc(m);
  __syncwarp();
  while (wq.n >= 32) {
    const SmallTri t = wq.q[wq.n - 32 + lane];
    __syncwarp();
    wq.n -= 32;
    small_tri_apportion(M, t);
  }
}

__device__ __forceinline__ void wq_drain(const MapDev &M, WarpQueue &wq, int lane) {
  if (wq.n > 0) {
    SmallTri t;
    const bool have = lane < wq.n;
    if (have) t = wq.q[lane];
    __syncwarp();
    if (have) small_tri_apportion(M, t);
    wq.n = 0;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// one triangle
// ---------------------------------------------------------------------------

// Per-lane triangle counters, reduced per warp into MapDev::stat:
// [0] dropped, [1] multi-pixel (clipped) in the map, [2] within a 2 x 2 box
// crossing both grid lines, [3] box of at most MM_MED_PIXELS pixels (pixel
// jobs), [4] larger (row jobs), [5] two pixels split by one grid line, [6]
// vertex rows not computed because culling proved them beyond the map.
#define MM_N_COUNTERS 8
struct IpmCounters {
  unsigned dropped, clipped, small, strip, big, line, culled, critical;
};

// A triangle shared out to the whole warp: frame pixel, frame coordinates,
// 2 / signed area and the inverse slope dx/dy of each edge k -> k + 1
// (infinite or NaN for a horizontal edge, which is never used).
struct __align__(16) TriJob {
  int ox, oy;
  float t[6];
  float inv2;
  float k[3];
};
static_assert(sizeof(TriJob) == MM_TRIJOB_BYTES, "TriJob layout");

enum { TRI_DONE = 0, TRI_SMALL = 1, TRI_BIG = 2, TRI_LINE = 3 };

// Apportion one triangle (a, b, c).  Triangles within one pixel are
// finished here, and so are those split by one grid line unless LINEQ, which
// returns TRI_LINE (le filled) for the line queue; returns TRI_SMALL (se
// filled) for a triangle covering 2 x 2 pixels, to be pushed on the quad
// queue, and TRI_BIG (job filled) for a larger one, whose pixel rows and then
// partially covered pixels the warp deals out to its lanes (warp_tri_jobs).
template <bool LINEQ>
__device__ __forceinline__ int ipm_triangle(const MapDev &M, const Vtx &a,
                                            const Vtx &b, const Vtx &c, RunAcc &ra,
                                            IpmCounters &cnt, SmallTri &se, TriJob &job,
                                            LineTri &le) {
  if (a.px == MM_VTX_INVALID || b.px == MM_VTX_INVALID || c.px == MM_VTX_INVALID) {
    cnt.dropped++;
    return TRI_DONE;
  }
  // the pixel box from the vertices' pixels (a vertex's pixel is the floor
  // of its coordinate), and wholly beyond one edge of the map (most
  // triangles of a shooting region): integer tests before any arithmetic
  const int xlo = min(a.px, min(b.px, c.px)), xhi = max(a.px, max(b.px, c.px));
  const int ylo = min(a.py, min(b.py, c.py)), yhi = max(a.py, max(b.py, c.py));
  if (xhi < 0 || xlo >= M.npix || yhi < 0 || ylo >= M.npix_y) return TRI_DONE;
  const int ox = a.px, oy = a.py;
  float t[6];
  t[0] = a.fx;
  t[1] = a.fy;
  // pixel indices stay within +-2^29, so differences fit in 32 bits
  t[2] = (float)(b.px - ox) + b.fx;
  t[3] = (float)(b.py - oy) + b.fy;
  t[4] = (float)(c.px - ox) + c.fx;
  t[5] = (float)(c.py - oy) + c.fy;
  const float area2 = (t[2] - t[0]) * (t[5] - t[1]) - (t[4] - t[0]) * (t[3] - t[1]);
  if (!(area2 != 0.f) || !isfinite(area2)) {
    cnt.dropped++;
    return TRI_DONE;
  }
  // near-critical: local |mu| = image area / source area above the threshold
  cnt.critical += fabsf(area2) < M.crit_area2;
  if (xlo == xhi && ylo == yhi) {
    // all three vertices in one (closed) map pixel: all of the area is there
    run_add(M, ra, (long long)oy * M.npix + ox, MM_FIX_ONE);
    return TRI_DONE;
  }
  // pixel range in the frame of vertex a
  const int cx0 = xlo - ox, cx1 = xhi - ox, cy0 = ylo - oy, cy1 = yhi - oy;
  if ((cx1 - cx0) + (cy1 - cy0) == 1) {
    // (two adjacent pixels that passed the test above: at least one is in
    // the map, so the map restriction below is not needed)
    cnt.clipped++;
    // Two pixels split by one grid line u = L (u = x or y).  The vertex alone
    // on its side cuts off a triangle similar to the corner it spans, of
    // area fraction d^2 / ((u_a - u_l)(u_b - u_l)) with d = L - u_l (the two
    // edge parameters at the line, multiplied).  The shares are complements
    // in fixed point, so the pair sums to exactly one triangle.
    const int o = cy1 - cy0;  // 0: vertical line, 1: horizontal line
    const float L = (float)(o ? cy0 : cx0) + 1.f;
    // (selects, not t[o]: a run-time index would put t in local memory)
    const float u0 = o ? t[1] : t[0], u1 = o ? t[3] : t[2], u2 = o ? t[5] : t[4];
    if (LINEQ) {
      le.gx = ox + cx0;  // the low pixel (indices within +-2^29)
      le.gy = oy + cy0;
      le.u0 = u0;
      le.u1 = u1;
      le.u2 = u2;
      le.L = L;
      le.o = o;
      cnt.line++;
      return TRI_LINE;
    }
    const unsigned long long vlow = low_side_fixed(u0, u1, u2, L);
    const bool b0 = u0 < L;  // vertex a on the low side
    // the pixel holding vertex a goes through the run accumulator
    const int glx = ox + cx0, gly = oy + cy0;  // low pixel
    const int gax = b0 ? glx : glx + 1 - o, gay = b0 ? gly : gly + o;
    const int gbx = b0 ? glx + 1 - o : glx, gby = b0 ? gly + o : gly;
    const unsigned long long va = b0 ? vlow : MM_FIX_ONE - vlow;
    if (va && gax >= 0 && gax < M.npix && gay >= 0 && gay < M.npix_y)
      run_add(M, ra, (long long)gay * M.npix + gax, va);
    deposit(M, gbx, gby, MM_FIX_ONE - va);
    cnt.line++;
    return TRI_DONE;
  }
  // restrict to the map: frame columns [-ox, npix-1-ox]
  const int mcl = -ox, mch = M.npix - 1 - ox;
  const int mrl = -oy, mrh = M.npix_y - 1 - oy;
  const int cl = cx0 > mcl ? cx0 : mcl, ch = cx1 < mch ? cx1 : mch;
  const int rl = cy0 > mrl ? cy0 : mrl, rh = cy1 < mrh ? cy1 : mrh;
  if (cl > ch || rl > rh) return TRI_DONE;  // misses the map
  cnt.clipped++;
  if (cx1 - cx0 <= 1 && cy1 - cy0 <= 1) {
    se.ox = ox;
    se.oy = oy;
    se.x0 = t[0];
    se.y0 = t[1];
    se.d1x = t[2] - t[0];
    se.d1y = t[3] - t[1];
    se.d2x = t[4] - t[0];
    se.d2y = t[5] - t[1];
    cnt.small++;
    return TRI_SMALL;
  }
  job.ox = ox;
  job.oy = oy;
#pragma unroll
  for (int k = 0; k < 6; k++) job.t[k] = t[k];
  {
    // 2 / area from the difference of products rounded once (Kahan's FMA
    // method): the area of a long thin triangle cancels heavily in FP32
    const float pa = t[2] - t[0], pd = t[5] - t[1], pb = t[4] - t[0], pc = t[3] - t[1];
    const float wbc = pb * pc;
    const float a2 = fmaf(pa, pd, -wbc) + fmaf(-pb, pc, wbc);
    job.inv2 = 2.0f / ((a2 != 0.f && isfinite(a2)) ? a2 : area2);
  }
#pragma unroll
  for (int e = 0; e < 3; e++)
    job.k[e] = (t[(2 * e + 2) % 6] - t[2 * e]) / (t[(2 * e + 3) % 6] - t[2 * e + 1]);
  if ((long long)(ch - cl + 1) * (rh - rl + 1) <= MM_MED_PIXELS)
    cnt.strip++;
  else
    cnt.big++;
  return TRI_BIG;
}

// ---------------------------------------------------------------------------
// larger triangles: the whole warp, lanes over pixel rows, then over the
// partially covered pixels of those rows
// ---------------------------------------------------------------------------

// Pixel areas of a larger triangle (Green's theorem on the clamped
// boundary, as above): area(T n [0, 1]^2) is the sum over T's edges of the
// integral over y in [0, 1] of clamp(x(y), 0, 1) along the edge, signed by
// the direction of y.  The clamped y-range of an edge and its x there depend
// only on the pixel row, so they are found once per row (row_pieces) and
// each pixel of the row only shifts them by its column (piece_integral).

// x on edge P -> Q (inverse slope k) at height y, extrapolated from the
// nearer endpoint, which halves the error the rounding of k makes on long
// edges.
__device__ __forceinline__ float edge_x_at(float y, float px, float py, float qx, float qy,
                                          float k) {
  const float d1 = y - py, d2 = y - qy;
  return fabsf(d1) <= fabsf(d2) ? fmaf(d1, k, px) : fmaf(d2, k, qx);
}

// Mean of clamp(x, 0, 1) over x in [a, b] (a piece shifted to its pixel),
// formed from sub-interval lengths so that a nearly vertical piece loses no
// precision; h times it is the piece's integral.
__device__ __forceinline__ float piece_mean(float a, float b) {
  const float w = __saturatef(a), v = __saturatef(b);  // clamp to [0, 1]
  const float in = fmaf(0.5f * (v - w), v + w, fmaxf(b - fmaxf(a, 1.f), 0.f));
  const float len = b - a;
  return len > 0.f ? in * rcp_approx_f(len) : w;
}

// Frame row r of J: each edge's piece inside the band r <= y <= r + 1
// (x-range [a, b] and signed height h, all zero when it misses the band),
// the columns [c0, c1] the band meets (widened by a small margin; extra
// columns get zero area) and the fully covered run [fa, fb] (empty when
// fa > fb), whose columns have all four corners in T (T convex): fa >= both
// left ends and fb + 1 <= both right ends of T's chords on the lines y = r
// and y = r + 1, which are the pieces' ends on those lines.
__device__ __forceinline__ void row_pieces(const TriJob &J, int r, float (&a)[3], float (&b)[3],
                                           float (&h)[3], int &c0, int &c1, int &fa, int &fb) {
  const float y0 = (float)r, y1 = (float)(r + 1);
  float lo = 3.0e38f, hi = -3.0e38f;
  float l0 = 3.0e38f, h0 = -3.0e38f, l1 = 3.0e38f, h1 = -3.0e38f;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const float px = J.t[2 * e], py = J.t[2 * e + 1];
    const float qx = J.t[(2 * e + 2) % 6], qy = J.t[(2 * e + 3) % 6];
    const float ys = fminf(fmaxf(py, y0), y1), ye = fminf(fmaxf(qy, y0), y1);
    const float xs = edge_x_at(ys, px, py, qx, qy, J.k[e]);
    const float xe = edge_x_at(ye, px, py, qx, qy, J.k[e]);
    const bool cross = ye != ys;
    a[e] = cross ? fminf(xs, xe) : 0.f;
    b[e] = cross ? fmaxf(xs, xe) : 0.f;
    h[e] = cross ? ye - ys : 0.f;
    if (cross) lo = fminf(lo, a[e]), hi = fmaxf(hi, b[e]);
    const float ylo = fminf(py, qy), yhi = fmaxf(py, qy);
    if (ylo < yhi) {
      if (ylo <= y0 && y0 <= yhi) {
        const float x = ys == y0 ? xs : xe;
        l0 = fminf(l0, x);
        h0 = fmaxf(h0, x);
      }
      if (ylo <= y1 && y1 <= yhi) {
        const float x = ys == y1 ? xs : xe;
        l1 = fminf(l1, x);
        h1 = fmaxf(h1, x);
      }
    }
  }
  const float eps = 1e-3f, lim = 1.0e9f;
  c0 = (int)floorf(fminf(fmaxf(lo - eps, -lim), lim));
  c1 = (int)floorf(fminf(fmaxf(hi + eps, -lim), lim));
  fa = 1;
  fb = 0;
  if (h0 >= l0 && h1 >= l1) {
    fa = (int)ceilf(fminf(fmaxf(fmaxf(l0, l1) + eps, -lim), lim));
    fb = (int)floorf(fminf(fmaxf(fminf(h0, h1) - eps, -lim), lim)) - 1;
  }
}

// Dealing tasks from a warp's lanes: lane j owns n_j tasks, numbered
// [ex_j, ex_j + n_j) in lane order (ex the exclusive scan), and the lanes
// with n_j > 0 are ranked by slot = their rank among them.  For the 32 tasks
// [base, base + 32), the owner of task base + l has slot
//   i0 + |{starts ex_j in (base, base + l]}|,  i0 = |{n_j > 0, ex_j <= base}| - 1,
// found with one ballot, one OR-reduction of start bits and a popcount:
// no chain of shuffles.
__device__ __forceinline__ int deal_owner_slot(int n, int ex, int base, int lane) {
  const int i0 = __popc(__ballot_sync(0xffffffffu, n > 0 && ex <= base)) - 1;
  const int d = ex - base;
  const unsigned bit = (n > 0 && d > 0 && d < 32) ? (1u << d) : 0u;
  const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
  return i0 + __popc(starts & ((2u << lane) - 1u));
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

// The pixel rows of one round of a larger-triangle batch, by slot (rank
// among the rows with partially covered pixels),
// shared by the lanes that measure their partially covered pixels: for each
// edge its piece in the row band, x relative to column c0, with height
// times 2/area (so the weighted sum of piece means is the pixel's share);
// the global column of c0, the global row, and the fully covered run
// [fa, fb] relative to c0 (none if fa > fb).  Stored as arrays over lanes,
// so lanes reading different rows hit different banks.
// One row's record as five 16-byte words (four used, one of padding so that
// eight consecutive records fall on distinct banks): the pixel lanes read it
// with four 16-byte loads.
struct __align__(16) RowRec {
  float4 p0;  // a0, b0, h0, a1
  float4 p1;  // b1, h1, a2, b2
  float4 p2;  // h2, gx0, gy, fa  (the last three as int bits)
  float4 p3;  // fb, st, -, -     (int bits)
  float4 pad;
};
struct RowRecs {
  RowRec r[32];
  int tk[32], trl[32], tex[32];  // triangles with rows: lane, first row, first row task
};

// Partially covered pixel number `task` of a round's rows, owned by the row
// in slot o.
__device__ __forceinline__ void pixel_task(const MapAcc &M, const RowRecs *rr, int o, int task,
                                           int ptotal) {
  if (task < ptotal) {
    const RowRec &R = rr->r[o];
    const float4 p0 = R.p0, p1 = R.p1, p2 = R.p2, p3 = R.p3;
    const int fa = __float_as_int(p2.w), fb = __float_as_int(p3.x);
    int c = task - __float_as_int(p3.y);
    if (fa <= fb && c >= fa) c += fb - fa + 1;
    const float cl = (float)c;
    float sh = p0.z * piece_mean(p0.x - cl, p0.y - cl);
    sh = fmaf(p1.y, piece_mean(p0.w - cl, p1.x - cl), sh);
    sh = fmaf(p2.x, piece_mean(p1.z - cl, p1.w - cl), sh);
    // the row and its columns lie in the map (clamped when the row was set up)
    const unsigned long long v = frac_to_fixed(sh);
    const long long idx =
        (long long)__float_as_int(p2.z) * M.npix + __float_as_int(p2.y) + c;
    if (v && MM_INDEX_OK(M.err, idx, (long long)M.npix * M.npix_y)) atomicAdd(&M.acc[idx], v);
  }
}

// The nb (<= 32) triangles q[0..nb) (warp shared memory) spanning more than
// 2 x 2 pixels.  Their pixel rows within the map are dealt out to the lanes,
// 32 at a time; a row adds 1/|area| to its fully covered run through the
// row difference array and records its edge pieces in rr[lane]; the
// partially covered pixels of those 32 rows are then dealt out one per lane.
// Work is proportional to the perimeter, and the lanes stay busy however
// the rows differ.  Call with all 32 lanes.
__device__ __forceinline__ void warp_tri_jobs(unsigned long long *acc,
                                                  unsigned long long *span, int npix,
                                                  int npix_y, unsigned *err,
                                                  const TriJob *q, int nb, RowRecs *rr,
                                                  int lane) {
  const MapAcc M = {acc, span, npix, npix_y, err};
  int rl = 0, nrows = 0;
  if (lane < nb) {
    const TriJob &J = q[lane];
    const float ymin = fminf(J.t[1], fminf(J.t[3], J.t[5]));
    const float ymax = fmaxf(J.t[1], fmaxf(J.t[3], J.t[5]));
    const int r0 = max((int)floorf(fmaxf(ymin, -1.0e9f)), -J.oy);
    const int r1 = min((int)floorf(fminf(ymax, 1.0e9f)), M.npix_y - 1 - J.oy);
    rl = r0;
    nrows = r1 >= r0 ? r1 - r0 + 1 : 0;
  }
  const int incl = warp_incl_scan(nrows, lane);
  const int excl = incl - nrows;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const unsigned with_rows = __ballot_sync(0xffffffffu, nrows > 0);
  if (nrows > 0) {
    const int slot = __popc(with_rows & ((1u << lane) - 1u));
    rr->tk[slot] = lane;
    rr->trl[slot] = rl;
    rr->tex[slot] = excl;
  }
  __syncwarp();
  for (int base = 0; base < total; base += 32) {
    const int task = base + lane;
    const int o = deal_owner_slot(nrows, excl, base, lane);
    int np = 0, r = 0, c0 = 0, fa = 1, fb = 0, k = 0;
    float pa[3], pb[3], ph[3];
    if (task < total) {
      k = rr->tk[o];
      r = rr->trl[o] + task - rr->tex[o];
      const TriJob &J = q[k];
      int c1;
      row_pieces(J, r, pa, pb, ph, c0, c1, fa, fb);
      c0 = max(c0, -J.ox);
      c1 = min(c1, M.npix - 1 - J.ox);
      fa = max(fa, c0);
      fb = min(fb, c1);
      if (c0 <= c1) {
        np = c1 - c0 + 1;
        if (fa <= fb) {
          np -= fb - fa + 1;
          // a fully covered pixel holds 1/|area| of the triangle (< 1 when any does)
          const unsigned long long full = frac_to_fixed(fabsf(J.inv2));
          const long long row = (long long)(J.oy + r) * (M.npix + 1);
          const long long sn = (long long)M.npix_y * (M.npix + 1);
          if (MM_INDEX_OK(M.err, row + J.ox + fa, sn) &&
              MM_INDEX_OK(M.err, row + J.ox + fb + 1, sn)) {
            atomicAdd(&M.span[row + J.ox + fa], full);
            atomicAdd(&M.span[row + J.ox + fb + 1], 0ull - full);
          }
        }
      }
    }
    // the partially covered pixels of these 32 rows: records by slot
    const int pincl = warp_incl_scan(np, lane);
    const int pexcl = pincl - np;
    const int ptotal = __shfl_sync(0xffffffffu, pincl, 31);
    const int slot = __popc(__ballot_sync(0xffffffffu, np > 0) & ((1u << lane) - 1u));
    __syncwarp();  // the previous round's readers are done with the records
    if (np > 0) {
      const TriJob &J = q[k];
      const float fc0 = (float)c0;
      float a[3], b[3], hh[3];
#pragma unroll
      for (int e = 0; e < 3; e++) {
        // x relative to column c0 (zero-height pieces stay zero)
        a[e] = ph[e] != 0.f ? pa[e] - fc0 : 0.f;
        b[e] = ph[e] != 0.f ? pb[e] - fc0 : 0.f;
        hh[e] = ph[e] * J.inv2;
      }
      RowRec &R = rr->r[slot];
      R.p0 = make_float4(a[0], b[0], hh[0], a[1]);
      R.p1 = make_float4(b[1], hh[1], a[2], b[2]);
      R.p2 = make_float4(hh[2], __int_as_float(J.ox + c0), __int_as_float(J.oy + r),
                         __int_as_float(fa - c0));
      R.p3 = make_float4(__int_as_float(fb - c0), __int_as_float(pexcl), 0.f, 0.f);
    }
    __syncwarp();
    for (int pbase = 0; pbase < ptotal; pbase += 32)
      pixel_task(M, rr, deal_owner_slot(np, pexcl, pbase, lane), pbase + lane, ptotal);
  }
  __syncwarp();
}

// Per-warp queue of larger triangles in shared memory (capacity 64 >=
// 31 + 31 + 2).  A full batch of 32 is shared out at once, so the lanes stay
// busy and the dealing overhead is amortised.
struct JobQueue {
  TriJob *q;
  RowRecs *rr;
  int n;
};

// Shared memory of one warp: the two queues and the row records.
struct WarpSmem {
  LineTri line[64];
  SmallTri quad[64];
  TriJob big[64];
  RowRecs rows;
};
#define MM_SHOOT_SMEM_BYTES (8 * sizeof(WarpSmem))  // 8 warps per block

// A queue entry with no pixel rows (frame far below any map).
__device__ __forceinline__ TriJob empty_job_impl() {
  TriJob e;
  e.ox = e.oy = -(1 << 30);
#pragma unroll
  for (int k = 0; k < 6; k++) e.t[k] = 0.f;
  e.inv2 = 0.f;
  e.k[0] = e.k[1] = e.k[2] = 0.f;
  return e;
}

// Queue the lanes' larger triangles (no processing).
__device__ __forceinline__ void jq_add(JobQueue &jq, bool want, const TriJob &job, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int pos = jq.n + __popc(m & ((1u << lane) - 1u));
  if (want) jq.q[pos] = job;
  jq.n += __popc(m);
  __syncwarp();
}

// Full batches of 32 queued triangles (with `flush` also the rest) go to
// the map's device queue for the larger-triangle kernel (k_big_ipm), which
// deals them out at a higher occupancy than this kernel's; a batch that
// does not fit is dealt out here, its reserved queue slots filled with
// empty jobs.
__device__ __forceinline__ void jq_share(const MapDev &M, JobQueue &jq, bool flush, int lane) {
  while (jq.n >= 32 || (flush && jq.n > 0)) {
    const int nb = min(jq.n, 32);
    jq.n -= nb;
    unsigned long long base = 0;
    if (M.bigq_cap > 0) {
      if (lane == 0) base = atomicAdd(M.bigq_n, (unsigned long long)nb);
      base = __shfl_sync(0xffffffffu, base, 0);
    }
    if (M.bigq_cap > 0 && base + nb <= (unsigned long long)M.bigq_cap) {
      if (lane < nb) M.bigq[base + lane] = jq.q[jq.n + lane];
      __syncwarp();
    } else {
      if (M.bigq_cap > 0 && lane < nb && base + lane < (unsigned long long)M.bigq_cap)
        M.bigq[base + lane] = empty_job_impl();
      warp_tri_jobs(M.acc, M.span, M.npix, M.npix_y, M.err, jq.q + jq.n, nb, jq.rr, lane);
    }
  }
}


}  // namespace mm
