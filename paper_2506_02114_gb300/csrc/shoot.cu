// Fused ray deflection + inverse polygon mapping (the hot kernel), the
// normalisation kernel and the deflection probe.
//
// Per ray vertex (Sec. 3.3, App. C): the vertex's leaf supplies
//   - the near-field stars (the leaf and its neighbours, at most leaf_size):
//     direct sum of m / conj(z - z_i);
//   - the local (Taylor) expansion of the far field about the leaf centre:
//     alpha_far = conj(dpsi/dz), dpsi/dz = (1/L) sum_l l c_l zeta^(l-1);
//   - the FP64 image of the leaf centre W_c (macro model + sheet + far field
//     at the centre), so that only small, centre-relative quantities are
//     evaluated in FP32 per ray.
// The lens equation (Sec. 2.2, circular sheet of Sec. 3.1) then gives
//   w - W_c = (1-kappa+kappa_*) d + gamma conj(d) - alpha_near
//             - conj(sum_{l>=2} l c_l zeta^(l-1) / L),   d = z - z_c.
#include <algorithm>

#include "ipm.cuh"
#include "mm_kernels.h"

namespace mm {

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Record of the sub-cell of the active leaf containing finest-level cell
// (cx, cy); -1 if none.
__device__ __forceinline__ int lookup_leaf(const MapDev &M, int cx, int cy) {
  int gx = (cx >> M.gshift) - M.gx0, gy = (cy >> M.gshift) - M.gy0;
  if (gx < 0 || gy < 0 || gx >= M.gw || gy >= M.gh) return -1;
  int e = __ldg(&M.grid[(int64_t)gy * M.gw + gx]);
  if (e >= 0) return e;
  int node = -e - 1;
  for (int lvl = M.glevel + 1; lvl <= MM_DMAX; lvl++) {
    int fc = __ldg(&M.first_child[node]);
    if (fc < 0) break;
    int sh = MM_DMAX - lvl;
    node = fc + (((cx >> sh) & 1) | (((cy >> sh) & 1) << 1));
  }
  const int a = __ldg(&M.node_active[node]);
  if (a < 0) return -1;
  // the host keeps every leaf level + sub <= MM_DMAX
  const int sh = MM_DMAX - __ldg(&M.node_level[node]) - M.sub, mask = (1 << M.sub) - 1;
  return (a << (2 * M.sub)) + (((cy >> sh) & mask) << M.sub) + ((cx >> sh) & mask);
}

// lookup_leaf with a per-lane cache keyed by the lookup-grid row: a grid
// entry that names a record directly holds for every finest-level row of
// that grid row (the lane's column is fixed), so consecutive vertex rows
// skip the grid read until they leave it
__device__ __forceinline__ int lookup_leaf_cached(const MapDev &M, int cx, int cy, int &c_gy,
                                                  int &c_leaf, bool &c_cull) {
  const int gy = (cy >> M.gshift) - M.gy0;
  if (gy == c_gy) return c_leaf;
  const int gx = (cx >> M.gshift) - M.gx0;
  int e = -1;
  if (gx >= 0 && gy >= 0 && gx < M.gw && gy < M.gh) {
    e = __ldg(&M.grid[(int64_t)gy * M.gw + gx]);
    if (e >= 0) {
      c_gy = gy;
      c_leaf = e;
    } else {
      c_gy = INT_MIN;  // a tree walk: not cached
      e = lookup_leaf(M, cx, cy);
    }
  } else {
    c_gy = INT_MIN;
  }
  // whether the record can prove a vertex beyond the map at all
  c_cull = e >= 0 && __ldg(&M.leaf[e].cull_side) != MM_CULL_NONE;
  return e;
}

// One Horner step of the two far-field chains: E <- E w + (c.x, c.y) and
// O <- O w + (c.z, c.w) in complex arithmetic, w = (wx, wy).
__device__ __forceinline__ void horner_pair(const float4 c, float wx, float wy, float &Er,
                                            float &Ei, float &Or, float &Oi) {
  const float er = fmaf(Er, wx, fmaf(-Ei, wy, c.x));
  const float ei = fmaf(Er, wy, fmaf(Ei, wx, c.y));
  const float orr = fmaf(Or, wx, fmaf(-Oi, wy, c.z));
  const float oi = fmaf(Or, wy, fmaf(Oi, wx, c.w));
  Er = er;
  Ei = ei;
  Or = orr;
  Oi = oi;
}

// Source-plane position of grid point (i + ti, j + tj) in pixel units:
// returns the integer pixel and the fraction.  ti = tj = 0 for ray vertices.
// PRELOAD: the far-field coefficient pairs are loaded ahead of the Horner
// steps (all six of the usual 15-term case at once, other orders four at a
// time); else each where it is used, which holds fewer registers across the
// steps (better in the polygon-mapping kernel of a map without a
// second-pass queue, which deals every larger triangle itself).
template <bool SQUARE, bool FRAC, bool PRELOAD = true>
__device__ __forceinline__ Vtx shoot_point(const MapDev &M, int leaf, int i, int j,
                                           float ti, float tj, bool valid) {
  const int4 *rp = reinterpret_cast<const int4 *>(M.leaf + (leaf < 0 ? 0 : leaf));
  int4 q0 = __ldg(rp), q1 = __ldg(rp + 1), q2 = __ldg(rp + 2), q3 = __ldg(rp + 3);
  const int i_ref = q0.x, j_ref = q0.y;
  const float fcx = __int_as_float(q0.z), fcy = __int_as_float(q0.w);
  const int Ui = q1.x, Vi = q1.y;
  const float Uf = __int_as_float(q1.z), Vf = __int_as_float(q1.w);
  const float zsx = __int_as_float(q2.x), zsy = __int_as_float(q2.y);
  const int near_off = q2.z, near_cnt = (leaf < 0) ? 0 : q2.w;
  const int coef_off = q3.x;

  // vertex position relative to the reference vertex, in grid units (exact
  // integers), and relative to the leaf centre
  const float fi = (float)(i - i_ref), fj = (float)(j - j_ref);
  float gx = fi - fcx, gy = fj - fcy;
  if (FRAC) {
    gx += ti;
    gy += tj;
  }

  // near field: S = sum m g / |g|^2 in grid units (|g|^2 = gx^2 + rho gy^2)
  // two stars per iteration into two accumulator pairs (independent chains)
  float Sx = 0.f, Sy = 0.f, Sx2 = 0.f, Sy2 = 0.f;
  const int maxcnt = __reduce_max_sync(0xffffffffu, near_cnt);
  const float4 *np_ = reinterpret_cast<const float4 *>(M.near_pos) + near_off;
  const float *nm_ = M.near_m + near_off;
  // a lane with fewer stars than the warp's most runs stand-ins whose
  // contribution is selected away after the reciprocal (a stand-in on a
  // vertex would otherwise give 0 x 1/0 = NaN there)
  int k = 0;
  for (; k + 1 < maxcnt; k += 2) {
    const bool a0 = k < near_cnt, a1 = k + 1 < near_cnt;
    const float4 s0 = a0 ? __ldg(np_ + k) : make_float4(0.f, 1.f, 0.f, 0.f);
    const float4 s1 = a1 ? __ldg(np_ + k + 1) : make_float4(0.f, 1.f, 0.f, 0.f);
    const float m0 = a0 ? __ldg(nm_ + k) : 0.f, m1 = a1 ? __ldg(nm_ + k + 1) : 0.f;
    float dx0 = (fi - s0.x) - s0.y, dy0 = (fj - s0.z) - s0.w;
    float dx1 = (fi - s1.x) - s1.y, dy1 = (fj - s1.z) - s1.w;
    if (FRAC) {
      dx0 += ti;
      dy0 += tj;
      dx1 += ti;
      dy1 += tj;
    }
    const float r0 = SQUARE ? fmaf(dx0, dx0, dy0 * dy0) : fmaf(dx0, dx0, M.rho * dy0 * dy0);
    const float r1 = SQUARE ? fmaf(dx1, dx1, dy1 * dy1) : fmaf(dx1, dx1, M.rho * dy1 * dy1);
    const float q0 = a0 ? m0 * rcp_approx(r0) : 0.f, q1 = a1 ? m1 * rcp_approx(r1) : 0.f;
    Sx = fmaf(q0, dx0, Sx);
    Sy = fmaf(q0, dy0, Sy);
    Sx2 = fmaf(q1, dx1, Sx2);
    Sy2 = fmaf(q1, dy1, Sy2);
  }
  if (k < maxcnt && k < near_cnt) {
    const float4 s0 = __ldg(np_ + k);
    const float m0 = __ldg(nm_ + k);
    float dx0 = (fi - s0.x) - s0.y, dy0 = (fj - s0.z) - s0.w;
    if (FRAC) {
      dx0 += ti;
      dy0 += tj;
    }
    const float r0 = SQUARE ? fmaf(dx0, dx0, dy0 * dy0) : fmaf(dx0, dx0, M.rho * dy0 * dy0);
    const float q0 = m0 * rcp_approx(r0);
    Sx = fmaf(q0, dx0, Sx);
    Sy = fmaf(q0, dy0, Sy);
  }
  Sx += Sx2;
  Sy += Sy2;

  // far field: f = sum_{k>=0} e_k zeta^(k+1), e_k = (k+2) c_(k+2) / (L delta),
  // as zeta E(w) + w O(w), w = zeta^2, E and O the even and odd k: two
  // independent Horner chains, one (e_2j, e_2j+1) pair per 16-byte load
  float fr = 0.f, fim = 0.f;
  const int npair = M.p >> 1;
  if (npair >= 1 && leaf >= 0) {
    const float zx = gx * zsx, zy = gy * zsy;
    const float wx = fmaf(zx, zx, -zy * zy), wy = 2.f * zx * zy;
    const float4 *e = reinterpret_cast<const float4 *>(M.coef + coef_off);
    const float4 c = __ldg(e + (npair - 1));
    float Er = c.x, Ei = c.y, Or = c.z, Oi = c.w;
    if (!PRELOAD) {
      for (int j = npair - 2; j >= 0; j--) horner_pair(__ldg(e + j), wx, wy, Er, Ei, Or, Oi);
    } else if (npair == 7) {
      // the usual case (15 terms): the other six pairs are all loaded before
      // the chains start, so their latencies overlap (a loop that loads each
      // pair where it is used waits on every load in turn)
      float4 cc[6];
#pragma unroll
      for (int j = 0; j < 6; j++) cc[j] = __ldg(e + j);
#pragma unroll
      for (int j = 5; j >= 0; j--) horner_pair(cc[j], wx, wy, Er, Ei, Or, Oi);
    } else {
      // other orders: four pairs loaded at a time
      int j = npair - 2;
      for (; j >= 3; j -= 4) {
        const float4 c0 = __ldg(e + j), c1 = __ldg(e + j - 1), c2 = __ldg(e + j - 2),
                     c3 = __ldg(e + j - 3);
        horner_pair(c0, wx, wy, Er, Ei, Or, Oi);
        horner_pair(c1, wx, wy, Er, Ei, Or, Oi);
        horner_pair(c2, wx, wy, Er, Ei, Or, Oi);
        horner_pair(c3, wx, wy, Er, Ei, Or, Oi);
      }
      for (; j >= 0; j--) horner_pair(__ldg(e + j), wx, wy, Er, Ei, Or, Oi);
    }
    fr = fmaf(zx, Er, fmaf(-zy, Ei, fmaf(wx, Or, -wy * Oi)));
    fim = fmaf(zx, Ei, fmaf(zy, Er, fmaf(wx, Oi, wy * Or)));
  }

  float u = Uf + (fmaf(M.A1, gx, -Sx * M.sx) - fr);
  float v = Vf + (fmaf(M.A2, gy, -Sy * M.sy) + fim);
  Vtx out;
  if (!valid || leaf < 0 || !isfinite(u) || !isfinite(v)) {
    out.px = MM_VTX_INVALID;
    out.py = MM_VTX_INVALID;
    out.fx = 0.f;
    out.fy = 0.f;
    return out;
  }
  const float lim = 268435456.0f;  // 2^28 pixels: far outside any map
  u = fminf(fmaxf(u, -lim), lim);
  v = fminf(fmaxf(v, -lim), lim);
  float flu = floorf(u), flv = floorf(v);
  out.px = Ui + (int)flu;
  out.py = Vi + (int)flv;
  out.fx = u - flu;
  out.fy = v - flv;
  return out;
}

// Map edge that vertex (i, j) of record `leaf` is proven to land beyond
// (MM_CULL_*), from the record's culling bound and the vertex's distances to
// the record's direct stars, measured as the near field measures them;
// MM_CULL_NONE when not proven.  `run` receives how many rows from j on
// (this one included) the proof holds for: the column's vertices stay in
// the sub-cell (below its upper edge, with a row to spare) and outside the
// culling radius of every direct star (a star above is approached by one
// row per row; one below or level only recedes).
template <bool SQUARE>
__device__ __forceinline__ int vertex_cull_side(const MapDev &M, int leaf, int i, int j,
                                                int &run) {
  run = 0;
  if (leaf < 0) return MM_CULL_NONE;
  const int4 *rp = reinterpret_cast<const int4 *>(M.leaf + leaf);
  const int4 q3 = __ldg(rp + 3);
  if (q3.z == MM_CULL_NONE) return MM_CULL_NONE;
  const int4 q0 = __ldg(rp), q2 = __ldg(rp + 2);
  const float r2 = __int_as_float(q3.w);
  const float fi = (float)(i - q0.x), fj = (float)(j - q0.y);
  // rows to the sub-cell's upper edge (centre + half-length, grid units)
  const float top = __int_as_float(q0.w) + 1.0f / __int_as_float(q2.y);
  int n = (int)floorf(fminf(top - fj, 1.0e6f)) - 1;
  const float rho = SQUARE ? 1.f : M.rho;
  const float4 *np_ = reinterpret_cast<const float4 *>(M.near_pos) + q2.z;
  for (int k = 0; k < q2.w; k++) {
    const float4 s = __ldg(np_ + k);
    const float dx = (fi - s.x) - s.y, dy = (fj - s.z) - s.w;
    const float dx2 = dx * dx;
    if (!(fmaf(rho * dy, dy, dx2) > r2)) return MM_CULL_NONE;
    if (dx2 > r2 || dy >= 0.f) continue;
    // rows until |dy| falls to sqrt((r2 - dx^2) / rho), less one to spare
    const float kin = -dy - sqrtf((r2 - dx2) / rho);
    n = min(n, (int)floorf(kin) - 1);
  }
  run = max(n, 1);
  return q3.z;
}

// The map edge a whole row of the warp's vertices is proven to lie beyond
// (lanes without a vertex agree with anything), and the rows from j on the
// proof holds for in every lane; MM_CULL_NONE otherwise.
template <bool SQUARE>
__device__ __forceinline__ int row_cull_side(const MapDev &M, int leaf, int i, int j,
                                             bool vvalid, int &run) {
  int r = 1 << 30;
  const int s = vvalid ? vertex_cull_side<SQUARE>(M, leaf, i, j, r) : -1;
  const int S = __reduce_max_sync(0xffffffffu, s);
  run = (int)__reduce_min_sync(0xffffffffu, (unsigned)r);
  return (S > 0 && __all_sync(0xffffffffu, s == S || s < 0)) ? S : MM_CULL_NONE;
}

// Whether both triangles of the cell (a, b, c, d) lie wholly beyond one
// edge of the map, from the vertices' pixels alone (false when a vertex is
// non-finite).
__device__ __forceinline__ bool cell_beyond_map(const MapDev &M, const Vtx &a, const Vtx &b,
                                                const Vtx &c, const Vtx &d) {
  const int x0 = min(min(a.px, b.px), min(c.px, d.px)), x1 = max(max(a.px, b.px), max(c.px, d.px));
  const int y0 = min(min(a.py, b.py), min(c.py, d.py)), y1 = max(max(a.py, b.py), max(c.py, d.py));
  return x0 != MM_VTX_INVALID && (x1 < 0 || x0 >= M.npix || y1 < 0 || y0 >= M.npix_y);
}

__device__ __forceinline__ Vtx shfl_down_vtx(const Vtx &v, int d) {
  Vtx r;
  r.px = __shfl_down_sync(0xffffffffu, v.px, d);
  r.py = __shfl_down_sync(0xffffffffu, v.py, d);
  r.fx = __shfl_down_sync(0xffffffffu, v.fx, d);
  r.fy = __shfl_down_sync(0xffffffffu, v.fy, d);
  return r;
}

// Warp-reduce the per-lane triangle counters into the map's statistics.
__device__ __forceinline__ void flush_counters(const MapDev &M, IpmCounters &cnt, int lane) {
  unsigned v[MM_N_COUNTERS] = {cnt.dropped, cnt.clipped, cnt.small,  cnt.strip,
                               cnt.big,     cnt.line,    cnt.culled, cnt.critical};
#pragma unroll
  for (int k = 0; k < MM_N_COUNTERS; k++) {
    for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], d);
    if (lane == 0 && v[k]) atomicAdd(&M.stat[k], (unsigned long long)v[k]);
  }
  cnt = IpmCounters{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
}

// Persistent warps; each work item is a strip of 31 cell columns by
// rows_per_item cell rows of one map.  Lane l computes vertex column
// 31*s + l for every vertex row of the item, keeps the previous row in
// registers and takes its right neighbour's vertices by shuffle; lanes 0..30
// then map cells (i, j-1) as the triangles {v00, v10, v11} and
// {v00, v11, v01} (diagonal from lower-left to upper-right).
#ifndef MM_SHOOT_MINB
#define MM_SHOOT_MINB 2  // resident 256-thread blocks per SM the register budget targets
#endif

// A single map (BATCH = false) arrives by value as a launch parameter, so
// its fields are read from the constant bank instead of held in registers;
// a batch reads its maps from the device array `maps`.
template <bool SQUARE, bool BATCH, bool PRELOAD>
__global__ void __launch_bounds__(256, MM_SHOOT_MINB)
    k_shoot_ipm(const MapDev *__restrict__ maps, const MapDev M1, int n_maps, int64_t total_work,
                unsigned long long *work_counter, unsigned *err) {
  const int lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  WarpSmem *ws = reinterpret_cast<WarpSmem *>(s_dyn) + (threadIdx.x >> 5);
  WarpQueue wq = {ws->quad, 0};
  LineQueue lq = {ws->line, 0};
  JobQueue jq = {ws->big, &ws->rows, 0};
  IpmCounters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  int last_map = -1;
  // A batch's current map, copied per warp into shared memory when the warp
  // moves to another map: its fields are then read there like a launch
  // parameter's, which leaves the registers to the per-ray work (reading
  // them from the descriptor array in global memory costs registers, and
  // spills, that the single-map kernel never pays).
  __shared__ MapDev s_md[8];
  MapDev &SM = s_md[threadIdx.x >> 5];
  while (true) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(work_counter, 1ull);
    w = __shfl_sync(0xffffffffu, w, 0);
    if ((int64_t)w >= total_work) break;
    int mi = 0;
    if (BATCH && n_maps > 1) {
      int lo = 0, hi = n_maps - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (maps[mid].work_begin <= (int64_t)w)
          lo = mid;
        else
          hi = mid - 1;
      }
      mi = lo;
    }
    if (BATCH && mi != last_map) {  // warp-uniform
      if (last_map >= 0) flush_counters(SM, cnt, lane);
      __syncwarp();
      const unsigned long long *src = reinterpret_cast<const unsigned long long *>(maps + mi);
      unsigned long long *dst = reinterpret_cast<unsigned long long *>(&SM);
      for (int k = lane; k < (int)(sizeof(MapDev) / 8); k += 32) dst[k] = src[k];
      __syncwarp();
      last_map = mi;
    }
    if (!BATCH) last_map = 0;
    const MapDev &M = BATCH ? SM : M1;
    const int64_t local = (int64_t)w - M.work_begin;
    const int64_t s = local % M.strips, b = (local / M.strips) * M.item_stride;
    // grid indices fit 32 bits (at most 2^31 - 1 rays per axis)
    const int i = (int)(M.col_begin + s * MM_STRIP) + lane;
    const int jb = (int)(M.row_begin + b * M.rows_per_item);
    const int je = (int)min((int64_t)jb + M.rows_per_item, M.row_end);
    const int col_end = (int)M.col_end;
    const bool vvalid = i <= col_end;  // vertex columns [col_begin, col_end]
    const int cx = __ldg(&M.col_cell[vvalid ? i : col_end]);
    const bool cell_col = (lane < MM_STRIP) && (i < col_end);
    RunAcc ra = {-1, 0ull};
    Vtx prev, prev_r;  // this lane's vertex of the previous row and its right neighbour's
    // culling state of the previous row (warp-uniform): the map edge it is
    // proven to lie beyond, and whether its vertices were computed
    int prev_side = MM_CULL_NONE;
    bool prev_exact = true;
    {
      const int leaf = lookup_leaf(M, cx, __ldg(&M.row_cell[jb]));
      if (leaf < 0 && vvalid) atomicOr(err, ERR_LOOKUP);
      prev = shoot_point<SQUARE, false, PRELOAD>(M, leaf, i, jb, 0.f, 0.f, vvalid);
      prev_r = shfl_down_vtx(prev, 1);
      int run;
      if (M.cull) prev_side = row_cull_side<SQUARE>(M, leaf, i, jb, vvalid, run);
    }
    // one pass more than there are cell rows: the last one maps nothing and
    // shares out what is left in the queue of larger triangles
    int c_gy = INT_MIN, c_leaf = -1;  // lookup cache of this lane's column
    bool c_cull = false;              // the cached record has a culling bound
    int cull_wait = 0, cull_pause = 0;  // rows left before the next culling test
    for (int j = jb + 1;; j++) {
      const bool fin = j > je;  // warp-uniform
      Vtx cur = prev, cur_r = prev_r;
      int side = MM_CULL_NONE;
      if (!fin) {
        const int cy = __ldg(&M.row_cell[j]);
        const int leaf = lookup_leaf_cached(M, cx, cy, c_gy, c_leaf, c_cull);
        if (leaf < 0 && vvalid) atomicOr(err, ERR_LOOKUP);
        // a row is provably beyond the map only if every lane's record has a
        // culling bound; otherwise the per-vertex test cannot succeed
        if (M.cull) {
          int run = 0;
          if (cull_wait > 0) {
            cull_wait--;
          } else if (!__any_sync(0xffffffffu, vvalid && !c_cull)) {
            side = row_cull_side<SQUARE>(M, leaf, i, j, vvalid, run);
            // a failed test pauses the tests of the next rows (1, 3, ... up to 8)
            cull_pause = side == MM_CULL_NONE ? min(2 * cull_pause + 1, 8) : 0;
            cull_wait = cull_pause;
          }
          if (side != MM_CULL_NONE && side == prev_side) {
            // rows j .. j + run - 1 and the one below lie beyond the same map
            // edge: the cells between them map nothing, and none of those
            // rows is computed
            const int skip = min(run, je - j + 1);
            prev_exact = false;
            if (lane == 0) cnt.culled += (unsigned)skip;
            j += skip - 1;
            continue;
          }
          if (!prev_exact) {
            // the row below was not computed; its cells with this row are needed
            const int lp = lookup_leaf(M, cx, __ldg(&M.row_cell[j - 1]));
            prev = shoot_point<SQUARE, false, PRELOAD>(M, lp, i, j - 1, 0.f, 0.f, vvalid);
            prev_r = shfl_down_vtx(prev, 1);
            prev_exact = true;
          }
        }
        cur = shoot_point<SQUARE, false, PRELOAD>(M, leaf, i, j, 0.f, 0.f, vvalid);
        cur_r = shfl_down_vtx(cur, 1);
        // a row of cells all beyond the map (and none with a non-finite
        // vertex, which must be counted) has nothing to map
        if (__all_sync(0xffffffffu, !cell_col || cell_beyond_map(M, prev, prev_r, cur, cur_r))) {
          prev = cur;
          prev_r = cur_r;
          prev_side = side;
          continue;
        }
      }
#pragma unroll 1
      for (int tri = 0; tri < 2; tri++) {
        TriJob job;
        SmallTri se;
        LineTri le;
        // triangle 0: (v00, v10, v11); triangle 1: (v00, v11, v01)
        Vtx vb, vc;
        vb.px = tri ? cur_r.px : prev_r.px;
        vb.py = tri ? cur_r.py : prev_r.py;
        vb.fx = tri ? cur_r.fx : prev_r.fx;
        vb.fy = tri ? cur_r.fy : prev_r.fy;
        vc.px = tri ? cur.px : cur_r.px;
        vc.py = tri ? cur.py : cur_r.py;
        vc.fx = tri ? cur.fx : cur_r.fx;
        vc.fy = tri ? cur.fy : cur_r.fy;
        const int code =
            (cell_col && !fin) ? ipm_triangle<!BATCH>(M, prev, vb, vc, ra, cnt, se, job, le)
                               : TRI_DONE;
        // (the batch kernel, which reads its maps from memory, has no
        // registers to spare for the line queue's state)
        if (!BATCH) lq_push(M, lq, code == TRI_LINE, le, lane);
        wq_push(M, wq, code == TRI_SMALL, se, lane);
        jq_add(jq, code == TRI_BIG, job, lane);
        jq_share(M, jq, fin && tri == 1, lane);
      }
      if (fin) break;
      prev = cur;
      prev_r = cur_r;
      prev_side = side;
    }
    run_flush(M, ra);
    if (!BATCH) lq_drain(M, lq, lane);
    wq_drain(M, wq, lane);
  }
  if (last_map >= 0) flush_counters(BATCH ? SM : M1, cnt, lane);
}

// Inverse ray shooting (Sec. 3.2; the IRS column of Table 1): every grid
// vertex is one ray, and the pixel it lands in gains one count.  The work
// items, deflection and culling are k_shoot_ipm's; lane l < 31 owns vertex
// column 31 s + l (lane 31 only the grid's last column) and a work item owns
// its vertex rows [jb, je) (the map's last item also je), so every ray is
// counted once.  Rows proven to land beyond a map edge are skipped: none of
// their rays can count, and a culled vertex is never non-finite (a ray on a
// star lies inside that star's culling radius).
// 4 blocks of 8 warps per SM (64 registers, no spills): the deflection
// alone gains from the occupancy that k_shoot_ipm's mapping code cannot
// afford (on the 2000^2 grid 3 blocks were 17 % faster than 2, and 4 are
// 8 % faster than 3; 5 spill and are slower).
#define MM_IRS_MINB 4
template <bool SQUARE>
__global__ void __launch_bounds__(256, MM_IRS_MINB)
    k_shoot_irs(const MapDev M, int64_t total_work, unsigned long long *work_counter,
                unsigned *err) {
  const int lane = threadIdx.x & 31;
  IpmCounters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  while (true) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(work_counter, 1ull);
    w = __shfl_sync(0xffffffffu, w, 0);
    if ((int64_t)w >= total_work) break;
    const int64_t local = (int64_t)w - M.work_begin;
    const int64_t s = local % M.strips, b = (local / M.strips) * M.item_stride;
    const int i = (int)(M.col_begin + s * MM_STRIP) + lane;
    const int jb = (int)(M.row_begin + b * M.rows_per_item);
    const int je = (int)min((int64_t)jb + M.rows_per_item, M.row_end);
    const int jl = je == (int)M.row_end ? je : je - 1;  // last vertex row owned
    const int col_end = (int)M.col_end;
    const bool vvalid = i <= col_end;
    const bool owner = vvalid && (lane < MM_STRIP || i == col_end);
    const int cx = __ldg(&M.col_cell[vvalid ? i : col_end]);
    RunAcc ra = {-1, 0ull};
    int c_gy = INT_MIN, c_leaf = -1;  // lookup cache of this lane's column
    bool c_cull = false;              // the cached record has a culling bound
    int cull_wait = 0, cull_pause = 0;  // rows left before the next culling test
    for (int j = jb; j <= jl; j++) {
      const int leaf = lookup_leaf_cached(M, cx, __ldg(&M.row_cell[j]), c_gy, c_leaf, c_cull);
      if (leaf < 0 && vvalid) atomicOr(err, ERR_LOOKUP);
      if (M.cull && cull_wait > 0) {
        cull_wait--;
      } else if (M.cull && !__any_sync(0xffffffffu, vvalid && !c_cull)) {
        int run;
        if (row_cull_side<SQUARE>(M, leaf, i, j, vvalid, run) != MM_CULL_NONE) {
          const int skip = min(run, jl - j + 1);
          if (lane == 0) cnt.culled += (unsigned)skip;
          j += skip - 1;
          cull_pause = 0;
          continue;
        }
        // a failed test pauses the tests of the next rows (1, 3, ... up to 8)
        cull_pause = min(2 * cull_pause + 1, 8);
        cull_wait = cull_pause;
      }
      const Vtx v = shoot_point<SQUARE, false>(M, leaf, i, j, 0.f, 0.f, vvalid);
      if (owner) {
        if (v.px == MM_VTX_INVALID)
          cnt.dropped++;
        else if (v.px >= 0 && v.px < M.npix && v.py >= 0 && v.py < M.npix_y)
          run_add(M, ra, (long long)v.py * M.npix + v.px, 1ull);
      }
    }
    run_flush(M, ra);
  }
  flush_counters(M, cnt, lane);
}

// Second pass over the larger triangles k_shoot_ipm (or k_ipm_vertices)
// queued for the map: each warp takes batches of 32 from the device queue
// and deals out their pixel rows and partially covered pixels
// (warp_tri_jobs), at 5 blocks per SM where the first kernel runs 2 (48
// registers allow 5 without spills: 3 % faster than 4; 6 forces spills)
#define MM_BIG_MINB 5
__global__ void __launch_bounds__(256, MM_BIG_MINB) k_big_ipm(const MapDev M) {
  __shared__ TriJob q[8][32];
  __shared__ RowRecs rr[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned long long cap = (unsigned long long)M.bigq_cap;
  const unsigned long long qn = *M.bigq_n;
  const long long n = (long long)(qn < cap ? qn : cap);
  while (true) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(M.bigq_n + 1, 1ull);
    b = __shfl_sync(0xffffffffu, b, 0);
    const long long base = (long long)b * 32;
    if (base >= n) break;
    const int nb = (int)min(32ll, n - base);
    if (lane < nb) q[w][lane] = M.bigq[base + lane];
    __syncwarp();
    warp_tri_jobs(M.acc, M.span, M.npix, M.npix_y, M.err, q[w], nb, &rr[w], lane);
  }
}

// mu = (acc + row-prefix(span)) * 2^-32 * (h_x h_y / 2) / delta^2; one block
// per map row.
__global__ void __launch_bounds__(256) k_normalize(const unsigned long long *__restrict__ acc,
                                                   const unsigned long long *__restrict__ span,
                                                   int npix, double scale, float *out) {
  __shared__ unsigned long long part[256];
  const int row = blockIdx.x;
  const int t = threadIdx.x;
  const int chunk = (npix + 255) / 256;
  const int c0 = t * chunk, c1 = min(npix, c0 + chunk);
  const unsigned long long *sp = span + (int64_t)row * (npix + 1);
  unsigned long long s = 0;
  for (int c = c0; c < c1; c++) s += sp[c];
  part[t] = s;
  __syncthreads();
  // inclusive scan of the 256 partial sums (Hillis-Steele)
  for (int d = 1; d < 256; d <<= 1) {
    unsigned long long v = (t >= d) ? part[t - d] : 0ull;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned long long run = (t > 0) ? part[t - 1] : 0ull;
  const unsigned long long *ar = acc + (int64_t)row * npix;
  float *o = out + (int64_t)row * npix;
  for (int c = c0; c < c1; c++) {
    run += sp[c];
    unsigned long long tot = ar[c] + run;
    o[c] = (float)((double)tot * scale);
  }
}

// mu = acc * scale for an accumulator already folded with its difference
// array (the same arithmetic as k_normalize, so a folded map normalises to
// the same floats)
__global__ void __launch_bounds__(256) k_scale_fixed(const unsigned long long *__restrict__ acc,
                                                     int64_t n, double scale, float *out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (float)((double)acc[k] * scale);
}

// acc += row-prefix(span): folds the difference array into the accumulator so
// the raw fixed-point map can be read back.
__global__ void k_fold_span(unsigned long long *acc, const unsigned long long *span, int npix,
                            int npix_y, unsigned long long *out) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= npix_y) return;
  const unsigned long long *sp = span + (int64_t)row * (npix + 1);
  unsigned long long run = 0;
  for (int c = 0; c < npix; c++) {
    run += sp[c];
    out[(int64_t)row * npix + c] = acc[(int64_t)row * npix + c] + run;
  }
}

// Deflection probe: w (FP64) at arbitrary image-plane points, through the
// same per-vertex code as the map kernel.
template <bool SQUARE>
__global__ void k_probe(const MapDev *maps, int64_t n, const double *z, double *w, double x0,
                        double y0, double hx, double hy, double R0, double lox, double loy,
                        double delta, unsigned *err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = t < n;
  const MapDev &M = maps[0];
  double zx = ok ? z[2 * t] : x0, zy = ok ? z[2 * t + 1] : y0;
  double gi = (zx - x0) / hx, gj = (zy - y0) / hy;
  double fi = floor(gi), fj = floor(gj);
  int64_t i = (int64_t)fi, j = (int64_t)fj;
  float ti = (float)(gi - fi), tj = (float)(gj - fj);
  const double scale = (double)(1 << MM_DMAX) / (2.0 * R0);
  double cxd = floor((zx + R0) * scale), cyd = floor((zy + R0) * scale);
  int cx = (int)fmin(fmax(cxd, 0.0), (double)((1 << MM_DMAX) - 1));
  int cy = (int)fmin(fmax(cyd, 0.0), (double)((1 << MM_DMAX) - 1));
  int leaf = ok ? lookup_leaf(M, cx, cy) : -1;
  Vtx v = shoot_point<SQUARE, true>(M, leaf, (int)i, (int)j, ti, tj, ok && leaf >= 0);
  if (!ok) return;
  if (v.px == MM_VTX_INVALID) {
    w[2 * t] = nan("");
    w[2 * t + 1] = nan("");
    return;
  }
  w[2 * t] = lox + ((double)v.px + (double)v.fx) * delta;
  w[2 * t + 1] = loy + ((double)v.py + (double)v.fy) * delta;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

template <bool SQUARE, bool BATCH, bool PRELOAD>
static cudaError_t launch_shoot_t(const MapDev *d_maps, const MapDev &m1, int n_maps,
                                  int64_t total_work, unsigned long long *counter, unsigned *err,
                                  int grid, cudaStream_t st) {
  const int smem = (int)MM_SHOOT_SMEM_BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_shoot_ipm<SQUARE, BATCH, PRELOAD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_shoot_ipm<SQUARE, BATCH, PRELOAD><<<grid, 256, smem, st>>>(d_maps, m1, n_maps, total_work,
                                                               counter, err);
  return cudaGetLastError();
}

cudaError_t launch_shoot_ipm(const MapDev *d_maps, const MapDev *h_single, int n_maps,
                             int64_t total_work, bool square, unsigned long long *counter,
                             unsigned *err, int grid, cudaStream_t st) {
  if (total_work <= 0) return cudaSuccess;
  if (n_maps == 1 && h_single) {
    // a map without a second-pass queue deals every larger triangle in this
    // kernel, which then runs faster with the far field's loads in place
    // (3-4 % on 10000^2 and 10000 x 1000 maps); with a queue the loads
    // ahead win (2-3 %)
    const MapDev &m = *h_single;
    if (m.bigq_cap > 0)
      return square ? launch_shoot_t<true, false, true>(nullptr, m, 1, total_work, counter, err,
                                                        grid, st)
                    : launch_shoot_t<false, false, true>(nullptr, m, 1, total_work, counter,
                                                         err, grid, st);
    return square ? launch_shoot_t<true, false, false>(nullptr, m, 1, total_work, counter, err,
                                                       grid, st)
                  : launch_shoot_t<false, false, false>(nullptr, m, 1, total_work, counter, err,
                                                        grid, st);
  }
  const MapDev none{};
  return square ? launch_shoot_t<true, true, true>(d_maps, none, n_maps, total_work, counter, err,
                                                   grid, st)
                : launch_shoot_t<false, true, true>(d_maps, none, n_maps, total_work, counter,
                                                    err, grid, st);
}

// Device-side assembly of a batch's descriptor array from the handles' own
// device copies (no host staging, so a batch can be captured in a CUDA
// graph): block i copies map i's descriptor and sets its first work item.
#define MM_GATHER_MAX 64
struct BatchGather {
  const MapDev *src[MM_GATHER_MAX];
  int64_t work_begin[MM_GATHER_MAX];
  int n;
};
static_assert(sizeof(MapDev) % 8 == 0, "MapDev copied in 8-byte words");

__global__ void k_batch_gather(const BatchGather g, MapDev *dst) {
  const int i = blockIdx.x;
  if (i >= g.n) return;
  const unsigned long long *s = reinterpret_cast<const unsigned long long *>(g.src[i]);
  unsigned long long *d = reinterpret_cast<unsigned long long *>(dst + i);
  for (int k = threadIdx.x; k < (int)(sizeof(MapDev) / 8); k += blockDim.x) d[k] = s[k];
  __syncthreads();
  if (threadIdx.x == 0) dst[i].work_begin = g.work_begin[i];
}

cudaError_t launch_batch_gather(const MapDev *const *src, const int64_t *work_begin, int n,
                                MapDev *dst, int &launches, cudaStream_t st) {
  for (int b = 0; b < n; b += MM_GATHER_MAX) {
    BatchGather g;
    g.n = min(MM_GATHER_MAX, n - b);
    for (int k = 0; k < g.n; k++) {
      g.src[k] = src[b + k];
      g.work_begin[k] = work_begin[b + k];
    }
    k_batch_gather<<<g.n, 64, 0, st>>>(g, dst + b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launches++;
  }
  return cudaSuccess;
}

cudaError_t launch_shoot_irs(const MapDev &m, int64_t total_work, bool square,
                             unsigned long long *counter, unsigned *err, cudaStream_t st) {
  if (total_work <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * MM_IRS_MINB;
  if (square)
    k_shoot_irs<true><<<grid, 256, 0, st>>>(m, total_work, counter, err);
  else
    k_shoot_irs<false><<<grid, 256, 0, st>>>(m, total_work, counter, err);
  return cudaGetLastError();
}

cudaError_t launch_big_ipm(const MapDev &m, cudaStream_t st) {
  if (m.bigq_cap <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_big_ipm<<<sms * MM_BIG_MINB, 256, 0, st>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_normalize(const unsigned long long *acc, const unsigned long long *span,
                             int npix, int npix_y, double scale, float *out, cudaStream_t st) {
  k_normalize<<<npix_y, 256, 0, st>>>(acc, span, npix, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_fixed(const unsigned long long *acc, int64_t n, double scale,
                               float *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)std::max(sms, 1) * 8);
  k_scale_fixed<<<(unsigned)blocks, 256, 0, st>>>(acc, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_fold_span(unsigned long long *acc, const unsigned long long *span, int npix,
                             int npix_y, unsigned long long *out, cudaStream_t st) {
  k_fold_span<<<(npix_y + 127) / 128, 128, 0, st>>>(acc, span, npix, npix_y, out);
  return cudaGetLastError();
}

cudaError_t launch_probe(const MapDev *d_maps, bool square, int64_t n, const double *z,
                         double *w, double x0, double y0, double hx, double hy, double R0,
                         double lox, double loy, double delta, unsigned *err,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (square)
    k_probe<true><<<(unsigned)blocks, 256, 0, st>>>(d_maps, n, z, w, x0, y0, hx, hy, R0, lox,
                                                    loy, delta, err);
  else
    k_probe<false><<<(unsigned)blocks, 256, 0, st>>>(d_maps, n, z, w, x0, y0, hx, hy, R0, lox,
                                                     loy, delta, err);
  return cudaGetLastError();
}

}  // namespace mm
