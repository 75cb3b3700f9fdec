// Plain FP64 path: the lens equation of Sec. 2.2 (sheet of Sec. 3.1, or of
// App. B for a rectangular star region)
// summed directly over every star in FP64 for each ray vertex (no tree), then
// the same inverse polygon mapping as the FMM path, reading the mapped
// vertices back from a buffer.  This is the baseline the FMM path's speed-up
// is measured against on the same GPU.
#include "ipm.cuh"
#include "mm_kernels.h"

namespace mm {

// 1/x: hardware approximation refined by two Newton-Raphson steps
// y <- y + y (1 - x y), each doubling the number of correct bits.
__device__ __forceinline__ double rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  return y;
}

#define D64_TILE 256

// alpha_star at (x, y) from all stars, staged through shared memory.
__device__ __forceinline__ void direct_sum(const double *__restrict__ sx,
                                           const double *__restrict__ sy,
                                           const double *__restrict__ sm, int64_t n_stars,
                                           double x, double y, double &ax, double &ay) {
  __shared__ double tx[D64_TILE], ty[D64_TILE], tm[D64_TILE];
  ax = 0.0;
  ay = 0.0;
  for (int64_t base = 0; base < n_stars; base += D64_TILE) {
    const int cnt = (int)min((int64_t)D64_TILE, n_stars - base);
    __syncthreads();
    if (threadIdx.x < cnt) {
      tx[threadIdx.x] = sx[base + threadIdx.x];
      ty[threadIdx.x] = sy[base + threadIdx.x];
      tm[threadIdx.x] = sm[base + threadIdx.x];
    }
    __syncthreads();
    for (int k = 0; k < cnt; k++) {
      const double dx = x - tx[k], dy = y - ty[k];
      const double r2 = fma(dx, dx, dy * dy);
      const double q = tm[k] * rcp64(r2);
      ax = fma(q, dx, ax);
      ay = fma(q, dy, ay);
    }
  }
}

__device__ __forceinline__ void lens64(const DirectConst &C, double x, double y, double ax,
                                       double ay, double &wx, double &wy) {
  const double ak = 1.0 - C.kappa + C.kappa_star;
  wx = (ak + C.gamma) * x - ax;
  wy = (ak - C.gamma) * y - ay;
  if (C.rect_c1 > 0.0) {  // rectangular sheet (App. B): alpha_s = -kappa_star z + conj(At)
    const double2 t = rect_sheet_At(C.kappa_star, C.rect_c1, C.rect_c2, x, y);
    wx -= t.x;
    wy += t.y;
  }
}

__global__ void __launch_bounds__(D64_TILE) k_direct64_vertices(
    const double *__restrict__ sx, const double *__restrict__ sy, const double *__restrict__ sm,
    int64_t n_stars, DirectConst C, int64_t col0, int64_t width, int64_t row_lo, int64_t row_hi,
    Vtx *out) {
  const int64_t nv = width * (row_hi - row_lo + 1);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tt = t < nv ? t : nv - 1;
  const int64_t i = col0 + tt % width, j = row_lo + tt / width;
  const double x = __dadd_rn(C.x0, __dmul_rn((double)i, C.hx));
  const double y = __dadd_rn(C.y0, __dmul_rn((double)j, C.hy));
  double ax, ay, wx, wy;
  direct_sum(sx, sy, sm, n_stars, x, y, ax, ay);
  if (t >= nv) return;
  lens64(C, x, y, ax, ay, wx, wy);
  double u = (wx - C.lox) / C.delta, v = (wy - C.loy) / C.delta;
  Vtx o;
  if (!isfinite(u) || !isfinite(v)) {
    o.px = o.py = MM_VTX_INVALID;
    o.fx = o.fy = 0.f;
  } else {
    u = fmin(fmax(u, -536870912.0), 536870912.0);  // pixel indices within +-2^29
    v = fmin(fmax(v, -536870912.0), 536870912.0);
    const double fu = floor(u), fv = floor(v);
    o.px = (int)fu;
    o.py = (int)fv;
    o.fx = fminf((float)(u - fu), 0.99999994f);
    o.fy = fminf((float)(v - fv), 0.99999994f);
  }
  out[t] = o;
}

__global__ void __launch_bounds__(D64_TILE) k_direct64_points(
    const double *__restrict__ sx, const double *__restrict__ sy, const double *__restrict__ sm,
    int64_t n_stars, DirectConst C, int64_t n, const double *z, double *w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tt = t < n ? t : n - 1;
  const double x = z[2 * tt], y = z[2 * tt + 1];
  double ax, ay, wx, wy;
  direct_sum(sx, sy, sm, n_stars, x, y, ax, ay);
  if (t >= n) return;
  lens64(C, x, y, ax, ay, wx, wy);
  w[2 * t] = wx;
  w[2 * t + 1] = wy;
}

__device__ __forceinline__ Vtx load_vtx(const Vtx *verts, int64_t n0, int64_t row_lo, int64_t i,
                                       int64_t j, bool valid) {
  if (valid) return verts[(j - row_lo) * n0 + i];
  Vtx v;
  v.px = v.py = MM_VTX_INVALID;
  v.fx = v.fy = 0.f;
  return v;
}

// Inverse polygon mapping of stored vertices, same warp-strip decomposition
// and triangle split as the fused FMM kernel.
__global__ void __launch_bounds__(256) k_ipm_vertices(const MapDev *__restrict__ maps,
                                                      const Vtx *__restrict__ verts, int64_t n0,
                                                      int64_t row_lo, int64_t row_hi,
                                                      unsigned long long *work_counter,
                                                      unsigned *err) {
  const int lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  WarpSmem *ws = reinterpret_cast<WarpSmem *>(s_dyn) + (threadIdx.x >> 5);
  WarpQueue wq = {ws->quad, 0};
  JobQueue jq = {ws->big, &ws->rows, 0};
  const MapDev &M = maps[0];
  const int64_t strips = (n0 - 1 + MM_STRIP - 1) / MM_STRIP;
  const int64_t rows = row_hi - row_lo;  // cell rows
  const int64_t rpi = M.rows_per_item;
  const int64_t total = strips * ((rows + rpi - 1) / rpi);
  IpmCounters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  while (true) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(work_counter, 1ull);
    w = __shfl_sync(0xffffffffu, w, 0);
    if ((int64_t)w >= total) break;
    const int64_t s = (int64_t)w % strips, b = (int64_t)w / strips;
    const int64_t i = s * MM_STRIP + lane;
    const int64_t jb = row_lo + b * rpi;
    int64_t je = jb + rpi;
    if (je > row_hi) je = row_hi;
    const bool vvalid = i < n0;
    const bool cell_col = (lane < MM_STRIP) && (i + 1 < n0);
    RunAcc ra = {-1, 0ull};
    Vtx prev = load_vtx(verts, n0, row_lo, i, jb, vvalid);
    for (int64_t j = jb + 1; j <= je; j++) {
      const Vtx cur = load_vtx(verts, n0, row_lo, i, j, vvalid);
      Vtx cur_r, prev_r;
      cur_r.px = __shfl_down_sync(0xffffffffu, cur.px, 1);
      cur_r.py = __shfl_down_sync(0xffffffffu, cur.py, 1);
      cur_r.fx = __shfl_down_sync(0xffffffffu, cur.fx, 1);
      cur_r.fy = __shfl_down_sync(0xffffffffu, cur.fy, 1);
      prev_r.px = __shfl_down_sync(0xffffffffu, prev.px, 1);
      prev_r.py = __shfl_down_sync(0xffffffffu, prev.py, 1);
      prev_r.fx = __shfl_down_sync(0xffffffffu, prev.fx, 1);
      prev_r.fy = __shfl_down_sync(0xffffffffu, prev.fy, 1);
#pragma unroll 1
      for (int tri = 0; tri < 2; tri++) {
        TriJob job;
        SmallTri se;
        LineTri le;  // (unused: two-pixel triangles are apportioned in place)
        const int code = cell_col ? ipm_triangle<false>(M, prev, tri ? cur_r : prev_r,
                                                        tri ? cur : cur_r, ra, cnt, se, job, le)
                                  : TRI_DONE;
        wq_push(M, wq, code == TRI_SMALL, se, lane);
        jq_add(jq, code == TRI_BIG, job, lane);
        jq_share(M, jq, false, lane);
      }
      prev = cur;
    }
    run_flush(M, ra);
    wq_drain(M, wq, lane);
    jq_share(M, jq, true, lane);
  }
  unsigned v[MM_N_COUNTERS] = {cnt.dropped, cnt.clipped, cnt.small,  cnt.strip,
                               cnt.big,     cnt.line,    cnt.culled, cnt.critical};
#pragma unroll
  for (int k = 0; k < MM_N_COUNTERS; k++) {
    for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], d);
    if (lane == 0 && v[k]) atomicAdd(&M.stat[k], (unsigned long long)v[k]);
  }
}

cudaError_t launch_direct64_vertices(const double *sx, const double *sy, const double *sm,
                                     int64_t n_stars, const DirectConst &C, int64_t col0,
                                     int64_t width, int64_t row_lo, int64_t row_hi, Vtx *out,
                                     cudaStream_t st) {
  const int64_t nv = width * (row_hi - row_lo + 1);
  if (nv <= 0) return cudaSuccess;
  k_direct64_vertices<<<(unsigned)((nv + D64_TILE - 1) / D64_TILE), D64_TILE, 0, st>>>(
      sx, sy, sm, n_stars, C, col0, width, row_lo, row_hi, out);
  return cudaGetLastError();
}

cudaError_t launch_direct64_points(const double *sx, const double *sy, const double *sm,
                                   int64_t n_stars, const DirectConst &C, int64_t n,
                                   const double *z, double *w, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_direct64_points<<<(unsigned)((n + D64_TILE - 1) / D64_TILE), D64_TILE, 0, st>>>(
      sx, sy, sm, n_stars, C, n, z, w);
  return cudaGetLastError();
}

cudaError_t launch_ipm_vertices(const MapDev *d_map, const Vtx *verts, int64_t n0,
                                int64_t row_lo, int64_t row_hi, unsigned long long *counter,
                                unsigned *err, int grid, cudaStream_t st) {
  if (row_hi <= row_lo || n0 < 2) return cudaSuccess;
  const int smem = (int)MM_SHOOT_SMEM_BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_ipm_vertices, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  k_ipm_vertices<<<grid, 256, smem, st>>>(d_map, verts, n0, row_lo, row_hi, counter, err);
  return cudaGetLastError();
}

}  // namespace mm
