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
// covering a 2 x 2 pixel box.  This computes exactly the areas that the
// column-then-row Sutherland-Hodgman clipping of Fig. 3 produces.
//
// Paths:
//   * the triangle lies inside one pixel (the common case at ~100 rays per
//     pixel): that pixel gains exactly 2^32;
//   * it spans at most 2 x 2 pixels: queued per warp in shared memory and
//     apportioned 32 at a time from three quadrant areas by
//     inclusion-exclusion;
//   * its box holds at most MM_MED_PIXELS pixels of the map: the pixels of
//     all such triangles of a warp are dealt out to its lanes, one pixel
//     (one box area) per lane at a time;
//   * larger (cells next to a star map to triangles hundreds of pixels
//     wide): the pixel rows of all such triangles of a warp are dealt out to
//     its lanes; each row adds the constant 1/|area| to its run of fully
//     covered pixels through a per-row difference array and computes only
//     the partially covered ones, so the work is proportional to the
//     perimeter, not the area.
#pragma once
#include <climits>

#include "mm_common.cuh"

namespace mm {

#define MM_VTX_INVALID INT_MIN
#define MM_FAR 1.0e30f
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
  f = fminf(fmaxf(f, 0.0f), 1.0f);
  return (unsigned long long)__float2uint_rn(f * 16777216.0f) << 8;
}

// ---------------------------------------------------------------------------
// accumulation
// ---------------------------------------------------------------------------

// Add v fixed-point units to map pixel (gx, gy) if it lies in the map.
__device__ __forceinline__ void deposit(const MapDev &M, long long gx, long long gy,
                                        unsigned long long v) {
  if (v && gx >= 0 && gx < M.npix && gy >= 0 && gy < M.npix)
    atomicAdd(&M.acc[gy * M.npix + gx], v);
}

// Lane-private run accumulator: consecutive one-pixel triangles of a lane's
// column usually hit the same pixel; they are summed in a register.
struct RunAcc {
  long long idx;  // map index of the pixel being summed, -1 for none
  unsigned long long val;
};

__device__ __forceinline__ void run_flush(const MapDev &M, RunAcc &a) {
  if (a.idx >= 0) atomicAdd(&M.acc[a.idx], a.val);
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
  if (a.idx >= 0) atomicAdd(&M.acc[a.idx], a.val);
  a.idx = idx;
  a.val = v;
}

// ---------------------------------------------------------------------------
// areas
// ---------------------------------------------------------------------------

// Signed area of T n [0,1]^2 (orientation of T), T = (x_k, y_k) given
// relative to the box corner.
__device__ __forceinline__ float unit_box_area(const float *t) {
  float s = 0.f;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const float px = t[2 * e], py = t[2 * e + 1];
    const float qx = t[(2 * e + 2) % 6], qy = t[(2 * e + 3) % 6];
    const float dx = qx - px, dy = qy - py;
    const float rx = rcp_approx_f(dx), ry = rcp_approx_f(dy);
    float a0 = -px * rx, a1 = (1.f - px) * rx, a2 = -py * ry, a3 = (1.f - py) * ry;
    a0 = fminf(fmaxf(a0, 0.f), 1.f);
    a1 = fminf(fmaxf(a1, 0.f), 1.f);
    a2 = fminf(fmaxf(a2, 0.f), 1.f);
    a3 = fminf(fmaxf(a3, 0.f), 1.f);
    // sort the four cut parameters
    const float l0 = fminf(a0, a1), h0 = fmaxf(a0, a1), l1 = fminf(a2, a3), h1 = fmaxf(a2, a3);
    const float s0 = fminf(l0, l1), s3 = fmaxf(h0, h1);
    const float m0 = fmaxf(l0, l1), m1 = fminf(h0, h1);
    const float s1 = fminf(m0, m1), s2 = fmaxf(m0, m1);
    const float ts[6] = {0.f, s0, s1, s2, s3, 1.f};
    float cx = fminf(fmaxf(px, 0.f), 1.f), cy = fminf(fmaxf(py, 0.f), 1.f);
#pragma unroll
    for (int k = 1; k < 6; k++) {
      const float nx = fminf(fmaxf(fmaf(ts[k], dx, px), 0.f), 1.f);
      const float ny = fminf(fmaxf(fmaf(ts[k], dy, py), 0.f), 1.f);
      s = fmaf(cx, ny, fmaf(-nx, cy, s));
      cx = nx;
      cy = ny;
    }
  }
  return 0.5f * s;
}

// Signed area of T n {x < X, y < Y} for T = (0,0), d1, d2.
__device__ __forceinline__ float quad_area(float d1x, float d1y, float d2x, float d2y, float X,
                                           float Y) {
  const float vx[3] = {0.f, d1x, d2x}, vy[3] = {0.f, d1y, d2y};
  float s = 0.f;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const float px = vx[e], py = vy[e];
    const float qx = vx[(e + 1) % 3], qy = vy[(e + 1) % 3];
    const float dx = qx - px, dy = qy - py;
    const float tx = (X - px) * rcp_approx_f(dx);
    const float ty = (Y - py) * rcp_approx_f(dy);
    float t1 = fminf(tx, ty), t2 = fmaxf(tx, ty);
    t1 = fminf(fmaxf(t1, 0.f), 1.f);
    t2 = fminf(fmaxf(t2, 0.f), 1.f);
    const float p0x = fminf(px, X), p0y = fminf(py, Y);
    const float p1x = fminf(fmaf(t1, dx, px), X), p1y = fminf(fmaf(t1, dy, py), Y);
    const float p2x = fminf(fmaf(t2, dx, px), X), p2y = fminf(fmaf(t2, dy, py), Y);
    const float p3x = fminf(qx, X), p3y = fminf(qy, Y);
    s = fmaf(p0x, p1y, fmaf(-p1x, p0y, s));
    s = fmaf(p1x, p2y, fmaf(-p2x, p1y, s));
    s = fmaf(p2x, p3y, fmaf(-p3x, p2y, s));
  }
  return 0.5f * s;
}

// Fraction of T (frame coordinates t, 2/signed area inv2) in frame pixel (c, r).
__device__ __forceinline__ float pixel_fraction(const float *t, int c, int r, float inv2) {
  const float fc = (float)c, fr = (float)r;
  const float u[6] = {t[0] - fc, t[1] - fr, t[2] - fc, t[3] - fr, t[4] - fc, t[5] - fr};
  return unit_box_area(u) * inv2;
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

__device__ __forceinline__ void small_tri_apportion(const MapDev &M, const SmallTri &e) {
  const float xmin = e.x0 + fminf(0.f, fminf(e.d1x, e.d2x));
  const float xmax = e.x0 + fmaxf(0.f, fmaxf(e.d1x, e.d2x));
  const float ymin = e.y0 + fminf(0.f, fminf(e.d1y, e.d2y));
  const float ymax = e.y0 + fmaxf(0.f, fmaxf(e.d1y, e.d2y));
  const int c0 = (int)floorf(xmin), c1 = (int)floorf(xmax);
  const int r0 = (int)floorf(ymin), r1 = (int)floorf(ymax);
  // dividing lines relative to the first vertex (MM_FAR when not crossed)
  const float X = (c1 > c0) ? (float)(c0 + 1) - e.x0 : MM_FAR;
  const float Y = (r1 > r0) ? (float)(r0 + 1) - e.y0 : MM_FAR;
  const float A = 0.5f * (e.d1x * e.d2y - e.d2x * e.d1y);
  const float L = quad_area(e.d1x, e.d1y, e.d2x, e.d2y, X, MM_FAR);
  const float B = quad_area(e.d1x, e.d1y, e.d2x, e.d2y, MM_FAR, Y);
  const float LB = quad_area(e.d1x, e.d1y, e.d2x, e.d2y, X, Y);
  const float inv = 1.0f / A;
  const long long gx = (long long)e.ox + c0, gy = (long long)e.oy + r0;
  deposit(M, gx, gy, frac_to_fixed(LB * inv));
  if (r1 > r0) deposit(M, gx, gy + 1, frac_to_fixed((L - LB) * inv));
  if (c1 > c0) deposit(M, gx + 1, gy, frac_to_fixed((B - LB) * inv));
  if (c1 > c0 && r1 > r0) deposit(M, gx + 1, gy + 1, frac_to_fixed((A - L - B + LB) * inv));
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
// [0] dropped, [1] multi-pixel (clipped) in the map, [2] within a 2 x 2 box,
// [3] box of at most MM_MED_PIXELS pixels (pixel jobs), [4] larger (row jobs).
struct IpmCounters {
  unsigned dropped, clipped, small, strip, big;
};

// A triangle shared out to the whole warp: frame pixel and frame coordinates.
struct __align__(16) TriJob {
  int ox, oy;
  float t[6];
  float inv2;  // 2 / signed area
  int pad[3];
};

enum { TRI_DONE = 0, TRI_SMALL = 1, TRI_PIX = 2, TRI_ROWS = 3 };

// Apportion one triangle (a, b, c).  One-pixel triangles are finished here;
// returns TRI_SMALL (se filled) for a triangle within a 2 x 2 pixel box, to be
// pushed on the warp queue, TRI_PIX (job filled) when its box within the map
// holds at most MM_MED_PIXELS pixels, which the warp deals out one pixel per
// lane (warp_pixel_jobs), and TRI_ROWS (job filled) for a larger one, whose
// pixel rows the warp deals out (warp_row_jobs).
__device__ __forceinline__ int ipm_triangle(const MapDev &M, const Vtx &a,
                                            const Vtx &b, const Vtx &c, RunAcc &ra,
                                            IpmCounters &cnt, SmallTri &se, TriJob &job) {
  if (a.px == MM_VTX_INVALID || b.px == MM_VTX_INVALID || c.px == MM_VTX_INVALID) {
    cnt.dropped++;
    return TRI_DONE;
  }
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
  const float xmin = fminf(t[0], fminf(t[2], t[4])), xmax = fmaxf(t[0], fmaxf(t[2], t[4]));
  const float ymin = fminf(t[1], fminf(t[3], t[5])), ymax = fmaxf(t[1], fmaxf(t[3], t[5]));
  // pixel range in frame coordinates (clamped well inside int range)
  const float lim = 1.0e9f;
  const int cx0 = (int)floorf(fmaxf(xmin, -lim)), cx1 = (int)floorf(fminf(xmax, lim));
  const int cy0 = (int)floorf(fmaxf(ymin, -lim)), cy1 = (int)floorf(fminf(ymax, lim));
  if (cx0 == cx1 && cy0 == cy1) {
    // whole triangle inside one pixel
    const long long gx = (long long)ox + cx0, gy = (long long)oy + cy0;
    if (gx >= 0 && gx < M.npix && gy >= 0 && gy < M.npix) run_add(M, ra, gy * M.npix + gx, MM_FIX_ONE);
    return TRI_DONE;
  }
  // restrict to the map: frame columns [-ox, npix-1-ox]
  const long long mcl = -(long long)ox, mch = (long long)M.npix - 1 - ox;
  const long long mrl = -(long long)oy, mrh = (long long)M.npix - 1 - oy;
  const long long cl = cx0 > mcl ? cx0 : mcl, ch = cx1 < mch ? cx1 : mch;
  const long long rl = cy0 > mrl ? cy0 : mrl, rh = cy1 < mrh ? cy1 : mrh;
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
  job.inv2 = 2.0f / area2;
  if ((ch - cl + 1) * (rh - rl + 1) <= MM_MED_PIXELS) {
    cnt.strip++;
    return TRI_PIX;
  }
  cnt.big++;
  return TRI_ROWS;
}

// ---------------------------------------------------------------------------
// big triangles: the whole warp, lanes over pixel rows
// ---------------------------------------------------------------------------

// x-interval of the intersection of the horizontal line y = Y with triangle
// t; returns false when the line misses it.
__device__ __forceinline__ bool line_span(const float *t, float Y, float &lo, float &hi) {
  lo = 3.0e38f;
  hi = -3.0e38f;
  bool any = false;
#pragma unroll
  for (int e = 0; e < 3; e++) {
    const float x0 = t[2 * e], y0 = t[2 * e + 1];
    const float x1 = t[(2 * e + 2) % 6], y1 = t[(2 * e + 3) % 6];
    if (y0 == y1) {
      if (y0 == Y) {
        lo = fminf(lo, fminf(x0, x1));
        hi = fmaxf(hi, fmaxf(x0, x1));
        any = true;
      }
    } else if ((y0 <= Y && Y <= y1) || (y1 <= Y && Y <= y0)) {
      const float x = x0 + (Y - y0) * (x1 - x0) / (y1 - y0);
      lo = fminf(lo, x);
      hi = fmaxf(hi, x);
      any = true;
    }
  }
  return any;
}

// Pixel row r (frame coordinates) of a big triangle.  The fully covered
// columns are those whose four corners lie in T (T convex):
// [max(l0, l1), min(r0, r1)] with [l0, r0] and [l1, r1] the spans of T on
// the lines y = r and y = r + 1; they receive 2^32/|area| through the row
// difference array.  The row's x-extent is the union of those spans and of
// the vertices inside the band; the remaining columns are computed exactly.
__device__ __forceinline__ void span_row(const MapDev &M, const TriJob &J,
                                         long long r, long long cl, long long ch,
                                         unsigned long long full) {
  const float y0 = (float)r, y1 = (float)(r + 1);
  float l0, r0, l1, r1;
  const bool s0 = line_span(J.t, y0, l0, r0);
  const bool s1 = line_span(J.t, y1, l1, r1);
  float bx0 = 3.0e38f, bx1 = -3.0e38f;
  if (s0) bx0 = fminf(bx0, l0), bx1 = fmaxf(bx1, r0);
  if (s1) bx0 = fminf(bx0, l1), bx1 = fmaxf(bx1, r1);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float vy = J.t[2 * k + 1];
    if (vy >= y0 && vy <= y1) bx0 = fminf(bx0, J.t[2 * k]), bx1 = fmaxf(bx1, J.t[2 * k]);
  }
  if (!(bx0 <= bx1)) return;
  long long c0 = (int)floorf(fmaxf(bx0, -1.0e9f));
  long long c1 = (int)floorf(fminf(bx1, 1.0e9f));
  if (c0 < cl) c0 = cl;
  if (c1 > ch) c1 = ch;
  if (c0 > c1) return;
  long long fa = 1, fb = 0;  // fully covered columns [fa, fb]
  if (s0 && s1) {
    const float eps = 1e-3f;
    fa = (int)ceilf(fminf(fmaxf(l0, l1) + eps, 1.0e9f));
    fb = (long long)(int)floorf(fmaxf(fminf(r0, r1) - eps, -1.0e9f)) - 1;
    if (fa < c0) fa = c0;
    if (fb > c1) fb = c1;
  }
  const long long row = (long long)J.oy + r;
  for (long long c = c0; c <= c1; c++) {
    if (fa <= fb && c == fa) {
      c = fb;  // skip the fully covered run
      continue;
    }
    deposit(M, (long long)J.ox + c, row,
            frac_to_fixed(pixel_fraction(J.t, (int)c, (int)r, J.inv2)));
  }
  if (fa <= fb) {
    unsigned long long *sp = M.span + row * (M.npix + 1);
    atomicAdd(&sp[J.ox + fa], full);
    atomicAdd(&sp[J.ox + fb + 1], 0ull - full);
  }
}

// Lanes whose `have` is set hold a triangle spanning more than a 2 x 2 box;
// the pixel rows of all of them (within the map) are dealt out to the 32
// lanes, one row per lane at a time.  A lane finds the triangle owning its
// row by binary search over the warp's inclusive scan of row counts and
// takes that triangle from its owner by shuffles.  Call with all 32 lanes.
static __device__ __noinline__ void warp_row_jobs(const MapDev &M, bool have, const TriJob &job,
                                           int lane) {
  if (!__any_sync(0xffffffffu, have)) return;
  int rl = 0, nrows = 0, cl = 0, ch = -1;
  if (have) {
    const float ymin = fminf(job.t[1], fminf(job.t[3], job.t[5]));
    const float ymax = fmaxf(job.t[1], fmaxf(job.t[3], job.t[5]));
    const float xmin = fminf(job.t[0], fminf(job.t[2], job.t[4]));
    const float xmax = fmaxf(job.t[0], fmaxf(job.t[2], job.t[4]));
    long long r0 = (int)floorf(fmaxf(ymin, -1.0e9f));
    long long r1 = (int)floorf(fminf(ymax, 1.0e9f));
    long long c0 = (int)floorf(fmaxf(xmin, -1.0e9f));
    long long c1 = (int)floorf(fminf(xmax, 1.0e9f));
    if (r0 < -(long long)job.oy) r0 = -(long long)job.oy;
    if (r1 > (long long)M.npix - 1 - job.oy) r1 = (long long)M.npix - 1 - job.oy;
    if (c0 < -(long long)job.ox) c0 = -(long long)job.ox;
    if (c1 > (long long)M.npix - 1 - job.ox) c1 = (long long)M.npix - 1 - job.ox;
    rl = (int)r0;
    cl = (int)c0;
    ch = (int)c1;
    nrows = r1 >= r0 ? (int)(r1 - r0 + 1) : 0;
  }
  int incl = nrows;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int task = base + lane;
    // owner: the first lane whose inclusive count exceeds task
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; it++) {
      const int mid = (lo + hi) >> 1;
      const int v = __shfl_sync(0xffffffffu, incl, mid);
      if (v > task)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int k = lo;
    TriJob J;
    J.ox = __shfl_sync(0xffffffffu, job.ox, k);
    J.oy = __shfl_sync(0xffffffffu, job.oy, k);
#pragma unroll
    for (int q = 0; q < 6; q++) J.t[q] = __shfl_sync(0xffffffffu, job.t[q], k);
    J.inv2 = __shfl_sync(0xffffffffu, job.inv2, k);
    const int krl = __shfl_sync(0xffffffffu, rl, k);
    const int kcl = __shfl_sync(0xffffffffu, cl, k);
    const int kch = __shfl_sync(0xffffffffu, ch, k);
    const int kn = __shfl_sync(0xffffffffu, nrows, k);
    const int kincl = __shfl_sync(0xffffffffu, incl, k);
    if (task < total) {
      // a fully covered pixel holds 1/|area| of the triangle (< 1 when any does)
      const unsigned long long full = frac_to_fixed(fabsf(J.inv2));
      span_row(M, J, krl + (task - (kincl - kn)), kcl, kch, full);
    }
  }
}

// Lanes whose `have` is set hold a triangle whose box (within the map) holds
// at most MM_MED_PIXELS pixels; all those pixels are dealt out to the 32
// lanes, one per lane at a time, and each lane adds its pixel's share.
static __device__ __noinline__ void warp_pixel_jobs(const MapDev &M, bool have, const TriJob &job,
                                             int lane) {
  if (!__any_sync(0xffffffffu, have)) return;
  int c0 = 0, r0 = 0, w = 1, npx = 0;
  if (have) {
    const float xmin = fminf(job.t[0], fminf(job.t[2], job.t[4]));
    const float xmax = fmaxf(job.t[0], fmaxf(job.t[2], job.t[4]));
    const float ymin = fminf(job.t[1], fminf(job.t[3], job.t[5]));
    const float ymax = fmaxf(job.t[1], fmaxf(job.t[3], job.t[5]));
    int cl = (int)floorf(xmin), ch = (int)floorf(xmax);
    int rl = (int)floorf(ymin), rh = (int)floorf(ymax);
    cl = max(cl, -job.ox);
    ch = min(ch, M.npix - 1 - job.ox);
    rl = max(rl, -job.oy);
    rh = min(rh, M.npix - 1 - job.oy);
    c0 = cl;
    r0 = rl;
    w = ch - cl + 1;
    npx = (ch >= cl && rh >= rl) ? w * (rh - rl + 1) : 0;
  }
  int incl = npx;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int task = base + lane;
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; it++) {
      const int mid = (lo + hi) >> 1;
      if (__shfl_sync(0xffffffffu, incl, mid) > task)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int k = lo;
    float t[6];
#pragma unroll
    for (int q = 0; q < 6; q++) t[q] = __shfl_sync(0xffffffffu, job.t[q], k);
    const int kox = __shfl_sync(0xffffffffu, job.ox, k);
    const int koy = __shfl_sync(0xffffffffu, job.oy, k);
    const float kinv = __shfl_sync(0xffffffffu, job.inv2, k);
    const int kc0 = __shfl_sync(0xffffffffu, c0, k);
    const int kr0 = __shfl_sync(0xffffffffu, r0, k);
    const int kw = __shfl_sync(0xffffffffu, w, k);
    const int kstart = __shfl_sync(0xffffffffu, incl - npx, k);
    if (task < total) {
      const int q = task - kstart;
      const int c = kc0 + q % kw, r = kr0 + q / kw;
      deposit(M, (long long)kox + c, (long long)koy + r,
              frac_to_fixed(pixel_fraction(t, c, r, kinv)));
    }
  }
}

// Per-warp queue of triangles for the pixel (PIX) or row (ROWS) jobs, in
// shared memory (capacity 64 >= 31 + 31 + 2).  A full batch of 32 is shared
// out at once, so the lanes stay busy and the dealing overhead is amortised.
struct JobQueue {
  TriJob *q;
  int n;
};

// Shared memory of one warp: the three queues.
struct WarpSmem {
  SmallTri quad[64];
  TriJob pix[64];
  TriJob rows[64];
};
#define MM_SHOOT_SMEM_BYTES (8 * sizeof(WarpSmem))  // 8 warps per block

template <bool ROWS>
__device__ __forceinline__ void jq_push(const MapDev &M, JobQueue &jq, bool want,
                                        const TriJob &job, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return;
  const int pos = jq.n + __popc(m & ((1u << lane) - 1u));
  if (want) jq.q[pos] = job;
  jq.n += __popc(m);
  __syncwarp();
  while (jq.n >= 32) {
    const TriJob t = jq.q[jq.n - 32 + lane];
    __syncwarp();
    jq.n -= 32;
    if (ROWS)
      warp_row_jobs(M, true, t, lane);
    else
      warp_pixel_jobs(M, true, t, lane);
  }
}

template <bool ROWS>
__device__ __forceinline__ void jq_drain(const MapDev &M, JobQueue &jq, int lane) {
  if (jq.n > 0) {
    const bool have = lane < jq.n;
    TriJob t;
    if (have) t = jq.q[lane];
    __syncwarp();
    jq.n = 0;
    if (ROWS)
      warp_row_jobs(M, have, t, lane);
    else
      warp_pixel_jobs(M, have, t, lane);
  }
  __syncwarp();
}

}  // namespace mm
