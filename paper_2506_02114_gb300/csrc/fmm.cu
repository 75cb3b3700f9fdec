// Multipole and local expansions of the quadtree FMM (App. C.2), FP64.
//
// Coefficients are complex and normalised to the node half-length L about
// the node centre, as in App. C.2:
//   multipole  psi(z) = a_0 log(zeta) + sum_{k=1..p} a_k zeta^-k
//   local      psi(z) = sum_{l=0..p} c_l zeta^l,      zeta = (z - z_node)/L.
// The three shift operators depend only on the relative position of the two
// nodes in units of L, so they are fixed (p+1)x(p+1) complex matrices built
// once on the host: 4 for M2M (child quadrant), 49 slots (40 used) for M2L
// (same-level offsets in [-3, 3]^2 with Chebyshev distance >= 2) and 4 for
// L2L.  Each is stored as [op][k][l] so that threads indexed by the output
// coefficient l read consecutive entries.
//
// The l = 0 (logarithmic) terms of the locals are not formed: the deflection
// needs only dpsi/dz (Sec. 3.3), so c_0 never reaches a ray.
#include <cmath>
#include <vector>

#include "mm_kernels.h"

namespace mm {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// z^k by repeated squaring (k >= 0)
__device__ __forceinline__ double2 cpow(double2 z, int k) {
  double2 r = make_double2(1.0, 0.0);
  while (k > 0) {
    if (k & 1) r = cmul(r, z);
    z = cmul(z, z);
    k >>= 1;
  }
  return r;
}

__device__ __forceinline__ void node_geom(const TreeDev &T, int64_t node, int &level, int &cx,
                                          int &cy, double &zx, double &zy, double &L) {
  level = T.lvl[node];
  uint32_t x, y;
  morton_decode(T.code[node], x, y);
  cx = (int)x;
  cy = (int)y;
  const double side = 2.0 * T.R0 / (double)(1ll << level);
  zx = -T.R0 + ((double)cx + 0.5) * side;
  zy = -T.R0 + ((double)cy + 0.5) * side;
  L = 0.5 * side;
}

// Node id of the level-`level` cell (x, y), or -1 if that cell is not a node.
__device__ __forceinline__ int64_t find_node(const TreeDev &T, int level, int x, int y) {
  const int side = 1 << level;
  if (x < 0 || y < 0 || x >= side || y >= side) return -1;
  const uint64_t c = morton2((uint32_t)x, (uint32_t)y);
  int64_t lo = T.level_off[level], hi = T.level_off[level + 1];
  int64_t k = lower_bound_u64(T.code, lo, hi, c);
  return (k < hi && T.code[k] == c) ? k : -1;
}

// ---------------------------------------------------------------------------
// P2M: a_0 = sum m_i, a_k = -(1/k) sum m_i zeta_i^k  (leaves only)
// ---------------------------------------------------------------------------
__global__ void k_p2m(TreeDev T, int64_t n_nodes, int p, double2 *mp) {
  const int64_t node = blockIdx.x;
  if (node >= n_nodes || T.first_child[node] >= 0) return;
  const int k = threadIdx.x;
  if (k > p) return;
  int level, cx, cy;
  double zx, zy, L;
  node_geom(T, node, level, cx, cy, zx, zy, L);
  const double invL = 1.0 / L;
  double2 s = make_double2(0.0, 0.0);
  for (int64_t i = T.sbeg[node]; i < T.send[node]; i++) {
    const double m = T.sm[i];
    if (k == 0) {
      s.x += m;
    } else {
      double2 zeta = make_double2((T.sx[i] - zx) * invL, (T.sy[i] - zy) * invL);
      double2 zk = cpow(zeta, k);
      s.x = fma(m, zk.x, s.x);
      s.y = fma(m, zk.y, s.y);
    }
  }
  if (k > 0) s = make_double2(-s.x / k, -s.y / k);
  mp[node * (p + 1) + k] = s;
}

// ---------------------------------------------------------------------------
// M2M: parent b = sum over the four children of MM[q] a_child (App. C.2)
// ---------------------------------------------------------------------------
__global__ void k_m2m(TreeDev T, int level, int64_t n, int p, const double2 *__restrict__ MMop,
                      double2 *mp) {
  const int64_t node = T.level_off[level] + blockIdx.x;
  if ((int64_t)blockIdx.x >= n) return;
  const int fc = T.first_child[node];
  if (fc < 0) return;
  __shared__ double2 a[4][MM_PMAX + 1];
  const int P1 = p + 1;
  // factored M2M: b_k = z0^-k a_k per child, then
  // c_l = sum_q (z0/2)^l (-a_0 / l + sum_{k<=l} C(l-1, k-1) b_k), c_0 = sum_q a_0
  for (int idx = threadIdx.x; idx < 4 * P1; idx += blockDim.x) {
    const int q = idx / P1, k = idx % P1;
    const double2 v = mp[(int64_t)(fc + q) * P1 + k];
    a[q][k] = k ? cfma(MMop[(int64_t)P1 * P1 + q * 2 * P1 + k], v, make_double2(0.0, 0.0)) : v;
  }
  __syncthreads();
  const int l = threadIdx.x;
  if (l > p) return;
  double2 s = make_double2(0.0, 0.0);
  if (l == 0) {
    for (int q = 0; q < 4; q++) s = make_double2(s.x + a[q][0].x, s.y + a[q][0].y);
  } else {
    const double2 *bl = MMop + (int64_t)l * P1;  // binomials of row l, 1/l at k = 0
    for (int q = 0; q < 4; q++) {
      double tx = -a[q][0].x * bl[0].x, ty = -a[q][0].y * bl[0].x;
      for (int k = 1; k <= l; k++) {
        const double b = bl[k].x;
        tx = fma(b, a[q][k].x, tx);
        ty = fma(b, a[q][k].y, ty);
      }
      s = cfma(MMop[(int64_t)P1 * P1 + q * 2 * P1 + P1 + l], make_double2(tx, ty), s);
    }
  }
  mp[node * P1 + l] = s;
}

// ---------------------------------------------------------------------------
// Locals of an active node at level >= 2 (App. C.2):
//   L2L from the parent, M2L from the parent's neighbours' children that are
//   not adjacent (<= 27), P2L from the parent's unsplit neighbours that are
//   not adjacent (<= 5).
// ---------------------------------------------------------------------------
__global__ void k_local(TreeDev T, int level, int64_t n, int p, const int32_t *node_act,
                        const double2 *__restrict__ MLop, const double2 *__restrict__ LLop,
                        const double2 *__restrict__ mp, double2 *loc, unsigned *err) {
  if ((int64_t)blockIdx.x >= n) return;
  const int64_t node = T.level_off[level] + blockIdx.x;
  if (!node_act[node]) return;
  __shared__ double2 src[MM_PMAX + 1];
  const int P1 = p + 1;
  const int l = threadIdx.x;
  const bool on = l <= p && l >= 1;
  int lv, nx, ny;
  double zx, zy, L;
  node_geom(T, node, lv, nx, ny, zx, zy, L);
  const int px = nx >> 1, py = ny >> 1;
  double2 acc = make_double2(0.0, 0.0);

  // L2L from the parent
  const int64_t parent = find_node(T, level - 1, px, py);
  if (parent >= 0) {
    for (int k = threadIdx.x; k < P1; k += blockDim.x) src[k] = loc[parent * P1 + k];
    __syncthreads();
    const int q = (nx & 1) | ((ny & 1) << 1);
    const double2 *op = LLop + (int64_t)q * P1 * P1;
    if (on)
      for (int k = l; k <= p; k++) acc = cfma(op[k * P1 + l], src[k], acc);
    __syncthreads();
  }

  const double invL = 1.0 / L;
  for (int dy = -1; dy <= 1; dy++)
    for (int dx = -1; dx <= 1; dx++) {
      if (dx == 0 && dy == 0) continue;
      const int qx = px + dx, qy = py + dy;
      const int side = 1 << (level - 1);
      if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
      const int64_t qid = find_node(T, level - 1, qx, qy);
      if (qid < 0) {
        if (threadIdx.x == 0) atomicOr(err, ERR_TREE_INVARIANT);
        continue;
      }
      const int fc = T.first_child[qid];
      if (fc >= 0) {
        for (int c = 0; c < 4; c++) {
          const int ox = 2 * qx + (c & 1) - nx, oy = 2 * qy + (c >> 1) - ny;
          if (abs(ox) <= 1 && abs(oy) <= 1) continue;  // neighbour: near field
          // factored M2L: b_k = (-1/z0)^k a_k, then
          // c_l += (1/z0)^l (-a_0 / l + sum_k C(l+k-1, k-1) b_k)
          const double2 *pw =
              MLop + (int64_t)P1 * P1 + (int64_t)((oy + 3) * 7 + (ox + 3)) * 2 * P1;
          for (int k = threadIdx.x; k < P1; k += blockDim.x) {
            const double2 a = mp[(int64_t)(fc + c) * P1 + k];
            src[k] = k ? cfma(pw[k], a, make_double2(0.0, 0.0)) : a;
          }
          __syncthreads();
          if (on) {
            const double2 *bl = MLop + (int64_t)l * P1;  // binomials of row l, 1/l at k = 0
            double tx = -src[0].x * bl[0].x, ty = -src[0].y * bl[0].x;
            for (int k = 1; k <= p; k++) {
              const double b = bl[k].x;
              tx = fma(b, src[k].x, tx);
              ty = fma(b, src[k].y, ty);
            }
            acc = cfma(pw[P1 + l], make_double2(tx, ty), acc);
          }
          __syncthreads();
        }
      } else {
        // unsplit parent-neighbour: adjacent to the node unless its 2x2
        // level cells all lie at Chebyshev distance >= 2
        const int x0 = 2 * qx, y0 = 2 * qy;
        const bool adj = (x0 + 1 >= nx - 1 && x0 <= nx + 1) && (y0 + 1 >= ny - 1 && y0 <= ny + 1);
        if (adj) continue;
        if (on) {
          for (int64_t i = T.sbeg[qid]; i < T.send[qid]; i++) {
            double2 zeta = make_double2((T.sx[i] - zx) * invL, (T.sy[i] - zy) * invL);
            const double d = zeta.x * zeta.x + zeta.y * zeta.y;
            double2 inv = make_double2(zeta.x / d, -zeta.y / d);
            double2 zl = cpow(inv, l);
            const double f = -T.sm[i] / (double)l;
            acc.x = fma(f, zl.x, acc.x);
            acc.y = fma(f, zl.y, acc.y);
          }
        }
      }
    }
  if (l <= p) loc[node * P1 + l] = on ? acc : make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------------------
// Near field of an active leaf: the leaf, its same-level neighbour cells that
// are nodes (with all their descendants), and the unsplit nodes one level up
// covering the missing neighbour cells.
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ int for_each_near_range(const TreeDev &T, int64_t node, F &&f,
                                                   unsigned *err) {
  int level, nx, ny;
  double zx, zy, L;
  node_geom(T, node, level, nx, ny, zx, zy, L);
  if (level == 0) {
    f(T.sbeg[node], T.send[node]);
    return 0;
  }
  int64_t seen[9];
  int nseen = 0;
  for (int dy = -1; dy <= 1; dy++)
    for (int dx = -1; dx <= 1; dx++) {
      const int x = nx + dx, y = ny + dy;
      const int side = 1 << level;
      if (x < 0 || y < 0 || x >= side || y >= side) continue;
      int64_t id = find_node(T, level, x, y);
      if (id >= 0) {
        f(T.sbeg[id], T.send[id]);
        continue;
      }
      int64_t pid = find_node(T, level - 1, x >> 1, y >> 1);
      if (pid < 0) {
        atomicOr(err, ERR_TREE_INVARIANT);
        continue;
      }
      bool dup = false;
      for (int s = 0; s < nseen; s++) dup |= (seen[s] == pid);
      if (dup) continue;
      seen[nseen++] = pid;
      f(T.sbeg[pid], T.send[pid]);
    }
  return 0;
}

// Sub-cell q of active leaf t (records are numbered g = 4^s t + q, q
// row-major with y major): its centre and half-length.
__device__ __forceinline__ void sub_cell_geom(const TreeDev &T, const FmmConst &C,
                                              const int32_t *active_list, int64_t g,
                                              int64_t &node, double &zx, double &zy,
                                              double &L, double &cx, double &cy, double &Lq) {
  const int ns = 1 << C.sub, NS = ns * ns;
  const int64_t t = g / NS;
  const int q = (int)(g % NS), qx = q & (ns - 1), qy = q >> C.sub;
  node = active_list[t];
  int level, nx, ny;
  node_geom(T, node, level, nx, ny, zx, zy, L);
  Lq = L / ns;
  cx = zx + (double)(2 * qx + 1 - ns) * Lq;
  cy = zy + (double)(2 * qy + 1 - ns) * Lq;
}

// Whether a star of the leaf's near field stays in the sub-cell's direct
// sum: without sub-cells every one does; with them, those within the
// (2 MM_NEAR_K + 1)^2 block of sub-cells around it (L-inf distance below
// (2 MM_NEAR_K + 1) L_q from its centre).  The others join its local
// expansion (P2L), which they leave converging at least as fast as the
// ratio sqrt(2) / (2 MM_NEAR_K + 1).
__device__ __forceinline__ bool stays_direct(const FmmConst &C, double dx, double dy,
                                             double Lq) {
  if (C.sub == 0) return true;
  const double hw = (2 * MM_NEAR_K + 1) * Lq;
  return fabs(dx) < hw && fabs(dy) < hw;
}

// Direct-sum stars per sub-cell record.
__global__ void k_near_count(TreeDev T, FmmConst C, int64_t n_rec, const int32_t *active_list,
                             int32_t *near_cnt, unsigned *err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_rec) return;
  int64_t node;
  double zx, zy, L, cx, cy, Lq;
  sub_cell_geom(T, C, active_list, g, node, zx, zy, L, cx, cy, Lq);
  int64_t total = 0;
  for_each_near_range(
      T, node,
      [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; i++) total += stays_direct(C, T.sx[i] - cx, T.sy[i] - cy, Lq);
      },
      err);
  near_cnt[g] = (int32_t)total;
}

// One thread per sub-cell record g (active leaf t, sub-cell q).  The leaf's
// local expansion psi = sum_l c_l zeta^l, zeta = (z - z_c)/L, is re-centred
// exactly on the sub-cell centre z_q (an L2L translation to a descendant of
// the leaf, which receives no further M2L terms: its far field is the
// leaf's):
//   d_n = (L_q/L)^n sum_{l>=n} C(l, n) c_l u^(l-n),  u = (z_q - z_c)/L;
// the leaf's near-field stars that leave the direct sum (stays_direct) add
// their own expansion about z_q (P2L): m log(z - z_i) contributes
//   d_n += -m / (n w^n),  w = (z_i - z_q)/L_q,  n >= 1,
// and the result is kept to n <= p_eval.  A record's coefficients
// e_n = n d_n / (L_q delta), n = 2..p_eval, take coef_stride(p_eval) slots
// (an even count, zero-padded) so the kernel loads them in pairs; its
// direct stars are stored in its own grid frame.
// NB >= p_eval bounds the coefficients at compile time, so they stay in
// registers.
template <int NB>
__global__ void __launch_bounds__(64) k_leaf_finalize(TreeDev T, FmmConst C, int64_t n_rec,
                                const int32_t *active_list, const int32_t *near_off,
                                const int32_t *near_cnt, const double2 *__restrict__ loc,
                                LeafRec *leaf, NearPos *near_pos, float *near_m, float2 *coef,
                                unsigned *err) {
  __shared__ float2 s_cf[64][MM_PMAX + 1];  // per thread: FP32 copy of the leaf's coefficients
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_rec) return;
  int64_t node;
  double zx, zy, L, cx, cy, Lq;
  sub_cell_geom(T, C, active_list, g, node, zx, zy, L, cx, cy, Lq);
  const int p = C.p, P1 = p + 1, pe = min(C.p_eval, NB), cs = coef_stride(pe);

  // the grid vertex nearest the sub-cell centre
  const double gi = rint((cx - C.x0) / C.hx), gj = rint((cy - C.y0) / C.hy);
  const double xr = C.x0 + gi * C.hx, yr = C.y0 + gj * C.hy;
  LeafRec R;
  R.i_ref = (int32_t)gi;
  R.j_ref = (int32_t)gj;
  R.fcx = (float)((cx - xr) / C.hx);
  R.fcy = (float)((cy - yr) / C.hy);
  R.cull_side = MM_CULL_NONE;
  R.cull_r2 = -1.f;

  // re-centred leaf expansion.  d_1 sets the FP64 image of the centre and is
  // formed in FP64; d_2..d_pe are stored as FP32 coefficients, scaled to the
  // sub-cell (terms decay like the convergence ratio), and are formed in
  // FP32 from FP32 copies of the leaf's coefficients (GB300's FP64 rate is
  // 1/64 of its FP32 rate).
  const double2 *c = loc + node * P1;
  const double ux = (cx - zx) / L, uy = (cy - zy) / L, r = Lq / L;
  double2 d1 = make_double2(0.0, 0.0);
  if (pe >= 1) {
    double sx = 0.0, sy = 0.0, px = 1.0, py = 0.0;  // u^(l-1); C(l, 1) = l
    for (int l = 1; l <= p; l++) {
      const double2 cl = c[l];
      sx += l * (cl.x * px - cl.y * py);
      sy += l * (cl.x * py + cl.y * px);
      const double npx = px * ux - py * uy;
      py = px * uy + py * ux;
      px = npx;
    }
    d1 = make_double2(sx * r, sy * r);
  }
  float2 *cf = s_cf[threadIdx.x];
  for (int l = 0; l <= p; l++) cf[l] = make_float2((float)c[l].x, (float)c[l].y);
  const float fux = (float)ux, fuy = (float)uy, fr = (float)r;
  float2 d[NB + 1];
  float rn = fr;
#pragma unroll
  for (int n = 2; n <= NB; n++) {
    d[n] = make_float2(0.f, 0.f);
    if (n > pe) continue;
    rn *= fr;
    float sx = 0.f, sy = 0.f, px = 1.f, py = 0.f, binom = 1.f;  // u^(l-n), C(l, n)
#pragma unroll 1
    for (int l = n; l <= p; l++) {
      const float2 cl = cf[l];
      sx = fmaf(binom, cl.x * px - cl.y * py, sx);
      sy = fmaf(binom, cl.x * py + cl.y * px, sy);
      const float npx = px * fux - py * fuy;
      py = px * fuy + py * fux;
      px = npx;
      binom = binom * (float)(l + 1) / (float)(l + 1 - n);
    }
    d[n] = make_float2(sx * rn, sy * rn);
  }

  // near-field stars: direct (in this record's frame) or into the expansion;
  // the direct ones never exceed the slots k_near_count reserved
  int64_t k = near_off[g];
  const int64_t kend = k + near_cnt[g];
  double m_direct = 0.0;
  for_each_near_range(
      T, node,
      [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; i++) {
          const double dxs = T.sx[i] - cx, dys = T.sy[i] - cy;
          if (stays_direct(C, dxs, dys, Lq) && k < kend) {
            const double sxg = (T.sx[i] - xr) / C.hx, syg = (T.sy[i] - yr) / C.hy;
            const double Kx = rint(sxg), Ky = rint(syg);
            NearPos np;
            np.Kx = (float)Kx;
            np.fx = (float)(sxg - Kx);
            np.Ky = (float)Ky;
            np.fy = (float)(syg - Ky);
            near_pos[k] = np;
            near_m[k] = (float)T.sm[i];
            m_direct += T.sm[i];
            k++;
          } else {
            // 1/w = L_q / (z_i - z_q); d_1 in FP64, the rest in FP32
            const double den = dxs * dxs + dys * dys;
            const double ix = Lq * dxs / den, iy = -Lq * dys / den;
            const double m = T.sm[i];
            d1.x -= m * ix;
            d1.y -= m * iy;
            const float fix = (float)ix, fiy = (float)iy, fm = (float)m;
            float tx = fix * fix - fiy * fiy, ty = 2.f * fix * fiy;  // w^-2
#pragma unroll
            for (int n = 2; n <= NB; n++) {
              if (n <= pe) {
                d[n].x -= fm * tx / n;
                d[n].y -= fm * ty / n;
              }
              const float ntx = tx * fix - ty * fiy;
              ty = tx * fiy + ty * fix;
              tx = ntx;
            }
          }
        }
      },
      err);

  // Rectangular star region: the sheet's part beyond -kappa_star z is the
  // conjugate of At, analytic inside the rectangle, so its potential joins
  // the expansion like a far source: d_n += At^(n-1)(z_q) L_q^n / n!, with
  //   At'    = (kappa_star i / pi) sum_a s_a (-log(a - z)) - kappa_star,
  //   At^(k) = (kappa_star i / pi) sum_a s_a (k - 2)! / (a - z)^(k - 1), k >= 2,
  // i.e. d_n += (kappa_star i / pi) L_q^2 sum_a s_a r_a^(n-2) / (n (n-1) (n-2))
  // for n >= 3, r_a = L_q / (a - z_q).  No per-ray cost.
  if (C.rect_c1 > 0.0) {
    const double2 t0 = rect_sheet_At(C.kappa_star, C.rect_c1, C.rect_c2, cx, cy);
    d1.x += t0.x * Lq;
    d1.y += t0.y * Lq;
    const double f = C.kappa_star / 3.14159265358979323846;
    double lx = 0.0, ly = 0.0, rx[4], ry[4], px[4], py[4], sg[4], dmin2 = 1e300;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      double ax, ay;
      rect_corner(C.rect_c1, C.rect_c2, k, ax, ay, sg[k]);
      const double dx = ax - cx, dy = ay - cy, q = Lq / (dx * dx + dy * dy);
      dmin2 = fmin(dmin2, dx * dx + dy * dy);
      const double2 l = clog64(dx, dy);
      lx -= sg[k] * l.x;
      ly -= sg[k] * l.y;
      rx[k] = dx * q;   // L_q / (a - z_q)
      ry[k] = -dy * q;
      px[k] = 1.0;      // r_a^(n-2)
      py[k] = 0.0;
    }
    // the series converges like sqrt(2) L_q / (distance to the nearest
    // corner) over the record; beyond 1/2 its truncation is not negligible
    // (only sub-cells meeting the ray grid are ever evaluated)
    const bool on_grid = cx + Lq >= C.x0 && cx - Lq <= C.x1 && cy + Lq >= C.y0 && cy - Lq <= C.y1;
    if (on_grid && 2.0 * Lq * Lq > 0.25 * dmin2) atomicOr(err, ERR_RECT_CORNER);
    const double l2 = Lq * Lq;
    if (pe >= 2) {
      d[2].x += (float)((-f * ly - C.kappa_star) * l2 * 0.5);
      d[2].y += (float)(f * lx * l2 * 0.5);
    }
#pragma unroll
    for (int n = 3; n <= NB; n++) {
      double sx = 0.0, sy = 0.0;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const double t = px[k] * rx[k] - py[k] * ry[k];
        py[k] = px[k] * ry[k] + py[k] * rx[k];
        px[k] = t;
        sx += sg[k] * px[k];
        sy += sg[k] * py[k];
      }
      if (n <= pe) {
        const double w = f * l2 / ((double)n * (n - 1) * (n - 2));  // times i
        d[n].x += (float)(-w * sy);
        d[n].y += (float)(w * sx);
      }
    }
  }
  R.near_off = near_off[g];
  R.near_cnt = (int32_t)(k - R.near_off);

  const double s = 1.0 / (Lq * C.delta);
  const float fs = (float)s;
#pragma unroll
  for (int n = 2; n <= NB; n++)
    if (n <= pe) coef[g * cs + (n - 2)] = make_float2(n * d[n].x * fs, n * d[n].y * fs);
  for (int kk = pe - 1; kk < cs; kk++) coef[g * cs + kk] = make_float2(0.f, 0.f);

  // FP64 image of the sub-cell centre: macro model + sheet - far field there
  const double ak = 1.0 - C.kappa + C.kappa_star;
  const double Wx = (ak + C.gamma) * cx - d1.x / Lq;
  const double Wy = (ak - C.gamma) * cy + d1.y / Lq;  // - conj(d1/L_q)
  double U = (Wx - C.lox) / C.delta, V = (Wy - C.loy) / C.delta;
  // |Ui|, |Vi| < 2^28 keeps vertex pixel indices within +-2^29
  U = fmin(fmax(U, -2.0e8), 2.0e8);
  V = fmin(fmax(V, -2.0e8), 2.0e8);
  const double Ui = floor(U), Vi = floor(V);
  R.Ui = (int32_t)Ui;
  R.Vi = (int32_t)Vi;
  R.Uf = (float)(U - Ui);
  R.Vf = (float)(V - Vi);
  R.zsx = (float)(C.hx / Lq);
  R.zsy = (float)(C.hy / Lq);
  R.coef_off = (int32_t)(g * cs);
  R.node = (int32_t)node;

  // Culling bounds.  A vertex of this sub-cell (grid offset within
  // L_s + h of its centre) lands at the centre's image plus the macro term,
  // the evaluated far-field series and the direct stars' deflection, all in
  // pixels.  The first two stay within a box of half-widths B about (U, V):
  // |macro| <= |1 - kappa + kappa_* +- gamma| (L_s + h)/delta and
  // |series| <= sum_n |e_n| zeta_max^(n-1) over the stored coefficients.  If
  // that box lies D pixels beyond a map edge, a vertex whose direct stars
  // are all farther than M_direct / (delta (D - margin)) is deflected by
  // them less than D - margin, so it lands beyond that edge too.
  if (C.cull) {
    const double ak = 1.0 - C.kappa + C.kappa_star;
    const double hmax = fmax(C.hx, C.hy);
    const double zmax = sqrt(2.0) * (Lq + hmax) / Lq;
    double F = 0.0, zp = 1.0;
#pragma unroll
    for (int n = 2; n <= NB; n++) {
      zp *= zmax;  // zeta_max^(n-1)
      if (n <= pe) F += hypot((double)(n * d[n].x * fs), (double)(n * d[n].y * fs)) * zp;
    }
    F *= 1.01;
    const double Bu = fabs(ak + C.gamma) * (Lq + hmax) / C.delta + F;
    const double Bv = fabs(ak - C.gamma) * (Lq + hmax) / C.delta + F;
    const double Uc = U, Vc = V, n = (double)C.npix, ny = (double)C.npix_y, margin = 2.0;
    const double Dl = -(Uc + Bu), Dr = (Uc - Bu) - n, Db = -(Vc + Bv), Dt = (Vc - Bv) - ny;
    double D = Dl;
    int side = MM_CULL_LEFT;
    if (Dr > D) D = Dr, side = MM_CULL_RIGHT;
    if (Db > D) D = Db, side = MM_CULL_BOTTOM;
    if (Dt > D) D = Dt, side = MM_CULL_TOP;
    if (D > 2.0 * margin && U > -1.9e8 && U < 1.9e8 && V > -1.9e8 && V < 1.9e8) {
      const double rc = m_direct / (C.delta * (D - margin) * C.hx);  // grid units of h_x
      R.cull_side = side;
      R.cull_r2 = (float)(rc * rc * 1.01);
    }
  }
  leaf[g] = R;
}

// ---------------------------------------------------------------------------
// host: operator tables and launchers
// ---------------------------------------------------------------------------

struct cplx {
  double x, y;
};
static inline cplx cm(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
static inline cplx cpw(cplx z, int k) {
  cplx r{1.0, 0.0};
  for (int i = 0; i < k; i++) r = cm(r, z);
  return r;
}
static inline cplx cinv(cplx z) {
  double d = z.x * z.x + z.y * z.y;
  return {z.x / d, -z.y / d};
}

// binomial coefficients C(n, k) for n <= 2 p (Pascal's triangle, FP64)
static std::vector<std::vector<double>> binomials(int nmax) {
  std::vector<std::vector<double>> C(nmax + 1, std::vector<double>(nmax + 1, 0.0));
  for (int n = 0; n <= nmax; n++) {
    C[n][0] = 1.0;
    for (int k = 1; k <= n; k++) C[n][k] = C[n - 1][k - 1] + (k <= n - 1 ? C[n - 1][k] : 0.0);
  }
  return C;
}

void build_operator_tables(int p, std::vector<double2> &MM, std::vector<double2> &ML,
                           std::vector<double2> &LL) {
  const int P1 = p + 1;
  auto C = binomials(2 * p + 1);
  // M2M factored like M2L below: op[k][l] = (z0/2)^l C(l-1, k-1) z0^-k for
  // 1 <= k <= l and op[0][l] = -(z0/2)^l / l: the real binomials ([l][k],
  // 1/l at k = 0), then per child quadrant the powers z0^-k and (z0/2)^l
  MM.assign((size_t)P1 * P1 + (size_t)4 * 2 * P1, make_double2(0.0, 0.0));
  for (int l = 1; l <= p; l++) {
    MM[(size_t)l * P1].x = 1.0 / l;
    for (int k = 1; k <= l; k++) MM[(size_t)l * P1 + k].x = C[l - 1][k - 1];
  }
  LL.assign((size_t)4 * P1 * P1, make_double2(0.0, 0.0));
  ML.assign((size_t)49 * P1 * P1, make_double2(0.0, 0.0));
  for (int q = 0; q < 4; q++) {
    // M2M: child centre relative to the parent, in child half-lengths
    cplx z0{(q & 1) ? 1.0 : -1.0, (q >> 1) ? 1.0 : -1.0};
    double2 *pw = &MM[(size_t)P1 * P1 + (size_t)q * 2 * P1];
    const cplx iz = cinv(z0), hz{0.5 * z0.x, 0.5 * z0.y};
    for (int k = 0; k <= p; k++) {
      const cplx a = cpw(iz, k), b = cpw(hz, k);
      pw[k] = make_double2(a.x, a.y);
      pw[P1 + k] = make_double2(b.x, b.y);
    }
    // L2L: child centre relative to the parent, in parent half-lengths
    cplx w0{(q & 1) ? 0.5 : -0.5, (q >> 1) ? 0.5 : -0.5};
    double2 *ol = &LL[(size_t)q * P1 * P1];
    for (int l = 0; l <= p; l++) {
      const double s = std::ldexp(1.0, -l);
      for (int k = l; k <= p; k++) {
        cplx zz = cpw(w0, k - l);
        double b = C[k][l] * s;
        ol[k * P1 + l] = make_double2(zz.x * b, zz.y * b);
      }
    }
  }
  // M2L: source centre relative to the target, z0 = 2 (dx + i dy).  The
  // operator factors as op[k][l] = (1/z0)^l C(l+k-1, k-1) (-1/z0)^k for
  // k >= 1 and op[0][l] = -(1/z0)^l / l, so the table holds the real
  // binomials once ([l][k], with 1/l in the unused k = 0 slot) and, per
  // offset, the powers of -1/z0 (scaling the multipoles) and of 1/z0
  // (scaling the sums): P1^2 + 49 x 2 P1 entries.
  ML.assign((size_t)P1 * P1 + (size_t)49 * 2 * P1, make_double2(0.0, 0.0));
  for (int l = 1; l <= p; l++) {
    ML[(size_t)l * P1].x = 1.0 / l;
    for (int k = 1; k <= p; k++) ML[(size_t)l * P1 + k].x = C[l + k - 1][k - 1];
  }
  for (int dy = -3; dy <= 3; dy++)
    for (int dx = -3; dx <= 3; dx++) {
      if (std::abs(dx) <= 1 && std::abs(dy) <= 1) continue;
      cplx z0{2.0 * dx, 2.0 * dy};
      cplx iz = cinv(z0);
      cplx imz = cinv(cplx{-z0.x, -z0.y});
      double2 *pw = &ML[(size_t)P1 * P1 + (size_t)((dy + 3) * 7 + (dx + 3)) * 2 * P1];
      for (int k = 0; k <= p; k++) {
        const cplx a = cpw(imz, k), b = cpw(iz, k);
        pw[k] = make_double2(a.x, a.y);
        pw[P1 + k] = make_double2(b.x, b.y);
      }
    }
}

static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
static inline int coef_threads(int p) { return 32 * ((p + 1 + 31) / 32); }

cudaError_t launch_p2m(const TreeDev &T, int64_t n_nodes, int p, double2 *mp, cudaStream_t st) {
  if (n_nodes <= 0) return cudaSuccess;
  k_p2m<<<(unsigned)n_nodes, coef_threads(p), 0, st>>>(T, n_nodes, p, mp);
  return cudaGetLastError();
}

cudaError_t launch_m2m(const TreeDev &T, int level, int64_t n, int p, const double2 *MMop,
                       double2 *mp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_m2m<<<(unsigned)n, coef_threads(p), 0, st>>>(T, level, n, p, MMop, mp);
  return cudaGetLastError();
}

cudaError_t launch_local(const TreeDev &T, int level, int64_t n, int p, const int32_t *node_act,
                         const double2 *MLop, const double2 *LLop, const double2 *mp,
                         double2 *loc, unsigned *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_local<<<(unsigned)n, coef_threads(p), 0, st>>>(T, level, n, p, node_act, MLop, LLop, mp,
                                                   loc, err);
  return cudaGetLastError();
}

cudaError_t launch_near_count(const TreeDev &T, const FmmConst &C, int64_t n_active,
                              const int32_t *active_list, int32_t *near_cnt, unsigned *err,
                              cudaStream_t st) {
  if (n_active <= 0) return cudaSuccess;
  const int64_t n = n_active << (2 * C.sub);
  k_near_count<<<blocks_for(n, 128), 128, 0, st>>>(T, C, n, active_list, near_cnt, err);
  return cudaGetLastError();
}

cudaError_t launch_leaf_finalize(const TreeDev &T, const FmmConst &C, int64_t n_active,
                                 const int32_t *active_list, const int32_t *near_off,
                                 const int32_t *near_cnt, const double2 *loc, LeafRec *leaf,
                                 NearPos *near_pos, float *near_m, float2 *coef, unsigned *err,
                                 cudaStream_t st) {
  if (n_active <= 0) return cudaSuccess;
  const int64_t n = n_active << (2 * C.sub);
  const unsigned nb = blocks_for(n, 64);
  if (C.p_eval <= 16)
    k_leaf_finalize<16><<<nb, 64, 0, st>>>(T, C, n, active_list, near_off, near_cnt, loc, leaf,
                                           near_pos, near_m, coef, err);
  else if (C.p_eval <= 32)
    k_leaf_finalize<32><<<nb, 64, 0, st>>>(T, C, n, active_list, near_off, near_cnt, loc, leaf,
                                           near_pos, near_m, coef, err);
  else
    k_leaf_finalize<MM_PMAX><<<nb, 64, 0, st>>>(T, C, n, active_list, near_off, near_cnt, loc,
                                                leaf, near_pos, near_m, coef, err);
  return cudaGetLastError();
}

}  // namespace mm
