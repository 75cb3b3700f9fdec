// libmm C ABI: parameter derivation, workspace planning and the stream-
// ordered pipeline of a magnification map (see include/mm.h).
//
// mm_create derives every scalar of the run (Sec. 2.1-2.3, App. A and C.3),
// uploads the stars, and builds the quadtree once with host read-backs of the
// per-level node counts ("plan").  Those counts size every buffer, so mm_run
// then rebuilds the same tree and runs the whole path with no host
// synchronisation: Morton sort, level-by-level split/scan/children, active
// region, P2M, M2M up-sweep, M2L + P2L + L2L down-sweep, leaf records, lookup
// grid, fused deflection + inverse polygon mapping, big-triangle spans,
// normalisation.
#include <cub/cub.cuh>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mm.h"
#include "mm_kernels.h"

#ifndef MM_SHOOT_MINB
#define MM_SHOOT_MINB 2
#endif
// streams a batch's per-map trees, expansions and second passes run on
#define MM_BATCH_STREAMS 8

using namespace mm;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_err;

static mm_status fail(mm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

namespace mm {
// Lets other translation units of the library report through mm_last_error.
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace mm

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      if (e_ == cudaErrorMemoryAllocation) {                                            \
        cudaGetLastError();                                                             \
        return fail(MM_ENOMEM, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                          \
      }                                                                                 \
      return fail(MM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                  __LINE__);                                                            \
    }                                                                                   \
  } while (0)

// a library kernel launch: checked and counted
#define LCH(call)                   \
  do {                              \
    CK(call);                       \
    h->launches++;                  \
  } while (0)

#define CKS(expr)                   \
  do {                              \
    mm_status s_ = (expr);          \
    if (s_ != MM_OK) return s_;     \
  } while (0)

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------

// stream on which DBuf allocates and frees (NULL: synchronous cudaMalloc/cudaFree)
static thread_local cudaStream_t g_alloc_stream = nullptr;

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  bool pooled = false;  // p came from cudaMallocAsync
  cudaError_t ensure(size_t count, bool keep = false) {
    if (count == 0) count = 1;
    if (count <= n) return cudaSuccess;
    T *q = nullptr;
    const cudaStream_t s = g_alloc_stream;
    cudaError_t e = s ? cudaMallocAsync(&q, count * sizeof(T), s) : cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) return e;
    if (keep && p && n) {
      e = s ? cudaMemcpyAsync(q, p, n * sizeof(T), cudaMemcpyDeviceToDevice, s)
            : cudaMemcpy(q, p, n * sizeof(T), cudaMemcpyDeviceToDevice);
      if (e != cudaSuccess) {
        free_buf(q, s != nullptr);
        return e;
      }
    }
    if (p) free_buf(p, pooled);
    p = q;
    n = count;
    pooled = s != nullptr;
    return cudaSuccess;
  }
  void release() {
    if (p) free_buf(p, pooled);
    p = nullptr;
    n = 0;
    pooled = false;
  }
  // stream-ordered free for pooled memory when an allocation stream is set;
  // otherwise (or for cudaMalloc memory) a synchronous cudaFree
  static void free_buf(T *q, bool from_pool) {
    if (from_pool && g_alloc_stream)
      cudaFreeAsync(q, g_alloc_stream);
    else
      cudaFree(q);
  }
};

// Buffers of a handle are allocated and freed in stream order on its plan
// stream, from the device's default memory pool, whose release threshold is
// raised so that the memory of a destroyed handle is reused by the next one
// instead of being returned to the CUDA driver (creating and destroying handles
// of the same size then costs no driver allocation).
struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStream() { g_alloc_stream = prev; }
};

static void keep_pool_memory(int dev) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t threshold = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  done[dev] = true;
}

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------

struct mm_map {
  int device = 0;
  mm_params P{};
  mm_options opt{};
  int mode = MM_FMM_FP32;
  int p = 0, leaf_size = 32;
  int sub = 0, p_eval = 0;         // sub-cell levels; terms evaluated per ray
  int64_t N = 0;
  double R0 = 1.0;
  int64_t row_lo = 0, row_hi = 0;  // cell rows [row_lo, row_hi)
  int64_t col_lo = 0, col_hi = 0;  // cell columns [col_lo, col_hi)
  int rows_per_item = 64;
  cudaStream_t plan_stream = nullptr;
  cudaStream_t last_stream = nullptr;

  // stars
  DBuf<double> pos_in, m_in, sx, sy, sm;
  DBuf<uint64_t> keys_in, keys;
  DBuf<int32_t> idx_in, idx;
  DBuf<char> cub_tmp;

  // tree
  int depth = 0;
  std::vector<int64_t> level_off, level_cnt;
  int64_t n_nodes = 0;
  DBuf<int64_t> d_level_off;
  DBuf<uint64_t> code;
  DBuf<int32_t> lvl, sbeg, send, first_child, split, scan;

  // active region
  DBuf<int32_t> col_cell, row_cell, node_act, leaf_flag, leaf_scan, node_active, active_list;
  int64_t n_active = 0;
  double min_leaf_L = 0.0;
  int max_leaf_level = 0;

  // expansions
  DBuf<double2> MMop, MLop, LLop, mp, loc;
  DBuf<int32_t> near_cnt, near_off;
  int64_t n_near = 0;
  DBuf<LeafRec> leaf;
  DBuf<NearPos> near_pos;
  DBuf<float> near_m;
  DBuf<float2> coef;

  // lookup grid
  int glevel = 0, gshift = 0, gx0 = 0, gy0 = 0, gw = 1, gh = 1;
  DBuf<int32_t> grid;

  // map
  DBuf<unsigned long long> acc, span, stat, counter, fixed_out;
  DBuf<char> bigq;                     // larger triangles for the second IPM pass
  DBuf<unsigned long long> bigq_n;     // [0] queued, [1] batches taken
  int64_t bigq_cap = 0;
  DBuf<unsigned> err;
  DBuf<float> map;
  DBuf<MapDev> d_md;
  MapDev md{};
  DBuf<Vtx> verts;

  // batch workspace (used when this handle leads an mm_run_batch call)
  DBuf<MapDev> batch_md;

  int64_t launches = 0;   // library kernels launched by the last run
  bool prepared = false;  // tree + expansions current for the stars
  bool fresh = false;     // mm_create's plan built them and no run has used them yet
  bool ran = false;
  bool timed_out = false;
  // stage events: start, tree, expansions, mapping done, normalised, first
  // mapping pass done
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool ev_recorded = false;

  // autotuner outcome (mm_stats.autotuned, ms_autotune) and the larger
  // triangles per 2^20 cells its sampled runs counted (-1: not measured),
  // which sizes the default second-pass queue
  int tuned = 0;
  double ms_tune = 0.0;
  int32_t jobs_pm = -1;

  // The first mapping pass runs in `segments` launches over consecutive work
  // items, each followed by the second pass, so that the queue of larger
  // triangles (est_jobs) fits its capacity.  Per segment k,
  // seg_ev[2k] marks the end of its first pass and seg_ev[2k + 1] the end of
  // its second (time_stages only).
  int64_t segments = 1, last_segments = 0;
  std::vector<cudaEvent_t> seg_ev;

  // set when this handle led the last mm_run_batch (time_stages): events
  // around the batch's one shared deflection + mapping launch
  bool led_batch = false;
  cudaEvent_t batch_ev[2] = {nullptr, nullptr};

  // streams on which this handle, leading an mm_run_batch, runs the maps'
  // trees and expansions and their second passes side by side (each map's
  // launches are small; one stream would run them one after another), with
  // the events that fork them from and join them to the caller's stream
  std::vector<cudaStream_t> fan;
  std::vector<cudaEvent_t> fan_join;
  cudaEvent_t fan_fork[2] = {nullptr, nullptr};

  // pinned host scratch for the plan's small reads and uploads: [0, 4) read
  // slots, [8, 8 + MM_DMAX + 2) the level offsets (pageable copies of a few
  // bytes would each wait for the stream)
  int64_t *pin = nullptr;
};

// ---------------------------------------------------------------------------
// parameters (Sec. 2.1-2.3, 3.1, 3.2, App. A)
// ---------------------------------------------------------------------------

static mm_status derive(double kappa, double gamma, double s, int64_t n_stars,
                        const double *masses, double half_length, int32_t npix, double rpp,
                        const mm_options &o, mm_params &P) {
  memset(&P, 0, sizeof P);
  if (!std::isfinite(kappa) || !std::isfinite(gamma) || !std::isfinite(s))
    return fail(MM_EINVAL, "kappa, gamma and s must be finite");
  if (!(s >= 0.0 && s <= 1.0)) return fail(MM_EINVAL, "smooth_fraction %g outside [0, 1]", s);
  if (!(half_length > 0.0)) return fail(MM_EINVAL, "half_length must be > 0");
  if (npix < 1) return fail(MM_EINVAL, "npix must be >= 1");
  if (o.npix_y < 0) return fail(MM_EINVAL, "npix_y must be >= 0");
  if (n_stars < 0) return fail(MM_EINVAL, "n_stars must be >= 0");
  if (n_stars > 0 && !masses) return fail(MM_EINVAL, "masses is NULL");
  const double detm = (1.0 - kappa) * (1.0 - kappa) - gamma * gamma;
  if (std::fabs(detm) < 1e-12)
    return fail(MM_EINVAL, "|(1-kappa)^2 - gamma^2| < 1e-12: the macro model is critical");
  P.kappa = kappa;
  P.gamma = gamma;
  P.smooth_fraction = s;
  P.kappa_star = kappa * (1.0 - s);
  P.a1 = 1.0 - kappa + gamma;
  P.a2 = 1.0 - kappa - gamma;
  P.mu_macro = 1.0 / detm;
  if (P.kappa_star > 0.0 && n_stars == 0)
    return fail(MM_EINVAL, "kappa_star > 0 needs stars");
  double msum = 0.0, m2sum = 0.0;
  for (int64_t i = 0; i < n_stars; i++) {
    const double m = masses[i];
    if (!(m > 0.0) || !std::isfinite(m)) return fail(MM_EINVAL, "mass %lld is not > 0", (long long)i);
    msum += m;
    m2sum += m * m;
  }
  P.mean_m = n_stars ? msum / (double)n_stars : 0.0;
  P.m2_over_m = msum > 0.0 ? m2sum / msum : 0.0;
  P.flux_fraction_f = o.flux_fraction_f > 0.0 ? o.flux_fraction_f : 1e-3;
  // App. A: fraction f of the deflection PDF outside r
  P.r_border = std::sqrt(P.kappa_star * P.m2_over_m / P.flux_fraction_f);
  P.half_length = half_length;
  P.npix = npix;
  P.npix_y = o.npix_y > 0 ? o.npix_y : npix;
  P.delta = 2.0 * half_length / (double)npix;
  // square pixels: the map is npix_y delta high
  P.half_length_y = P.npix_y == npix ? half_length : 0.5 * (double)P.npix_y * P.delta;
  P.center_y[0] = o.center_y[0];
  P.center_y[1] = o.center_y[1];
  // Sec. 2.3: the macro image of the map, widened by the border r
  const double a[2] = {P.a1, P.a2};
  for (int k = 0; k < 2; k++) {
    P.img_center[k] = P.center_y[k] / a[k];
    P.img_half[k] = (o.img_half[0] > 0.0 && o.img_half[1] > 0.0)
                        ? o.img_half[k]
                        : ((k ? P.half_length_y : half_length) + P.r_border) / std::fabs(a[k]);
  }
  const bool grid_given = o.ray_grid[0] >= 2 && o.ray_grid[1] >= 2;
  for (int k = 0; k < 2; k++) {
    if (grid_given) {
      P.n[k] = o.ray_grid[k];
      P.h[k] = 2.0 * P.img_half[k] / (double)(P.n[k] - 1);
      P.x0[k] = P.img_center[k] - P.img_half[k];
    } else {
      if (!(rpp > 0.0)) return fail(MM_EINVAL, "rays_per_pixel must be > 0");
      // rays per pixel without lensing: square cells of side delta/sqrt(rpp)
      const double hh = P.delta / std::sqrt(rpp);
      const double nn = std::ceil(2.0 * P.img_half[k] / hh) + 1.0;
      if (!(nn < 2147483647.0)) return fail(MM_EINVAL, "ray grid above 2^31 rays per axis");
      P.n[k] = (int64_t)nn;
      P.h[k] = hh;
      P.x0[k] = P.img_center[k] - 0.5 * (double)(P.n[k] - 1) * hh;
    }
    if (P.n[k] < 2 || P.n[k] > 2147483647LL)
      return fail(MM_EINVAL, "ray grid must have 2 .. 2^31-1 rays per axis");
  }
  return MM_OK;
}

// ---------------------------------------------------------------------------
// pipeline stages
// ---------------------------------------------------------------------------

static TreeDev tree_dev(const mm_map *h) {
  TreeDev T;
  T.keys = h->keys.p;
  T.sx = h->sx.p;
  T.sy = h->sy.p;
  T.sm = h->sm.p;
  T.n_stars = h->N;
  T.R0 = h->R0;
  T.code = h->code.p;
  T.lvl = h->lvl.p;
  T.sbeg = h->sbeg.p;
  T.send = h->send.p;
  T.first_child = h->first_child.p;
  T.level_off = h->d_level_off.p;
  T.depth = h->depth;
  return T;
}

template <class F>
static mm_status cub_call(mm_map *h, bool plan, F &&f) {
  size_t bytes = 0;
  CK(f((void *)nullptr, bytes));
  if (plan) CK(h->cub_tmp.ensure(bytes));
  if (bytes > h->cub_tmp.n) return fail(MM_ESTATE, "internal: CUB workspace too small");
  CK(f((void *)h->cub_tmp.p, bytes));
  return MM_OK;
}

// Host operator tables of order p (App. C.2), built once per process and
// shared by every handle of that order.
struct OpTables {
  std::vector<double2> MM, ML, LL;
};
static const OpTables &operator_tables(int p) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<OpTables>> cache;
  std::lock_guard<std::mutex> lock(mu);
  std::unique_ptr<OpTables> &t = cache[p];
  if (!t) {
    t.reset(new OpTables);
    build_operator_tables(p, t->MM, t->ML, t->LL);
  }
  return *t;
}

// Reads n (<= 4) int32 device values through the pinned scratch: the copies
// are enqueued together and one synchronisation waits for all of them.
static mm_status read_ints(mm_map *h, cudaStream_t st, int n, const int32_t *const *src,
                           int32_t *out) {
  int32_t *slot = reinterpret_cast<int32_t *>(h->pin);
  for (int k = 0; k < n; k++)
    CK(cudaMemcpyAsync(slot + k, src[k], sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < n; k++) out[k] = slot[k];
  return MM_OK;
}

// Uploads the host level offsets through the pinned scratch (the caller's
// next read_ints completes the copy before the scratch is rewritten).
static mm_status upload_level_off(mm_map *h, cudaStream_t st) {
  int64_t *lo = h->pin + 8;
  for (int k = 0; k < MM_DMAX + 2; k++) lo[k] = h->level_off[k];
  CK(cudaMemcpyAsync(h->d_level_off.p, lo, (MM_DMAX + 2) * sizeof(int64_t),
                     cudaMemcpyHostToDevice, st));
  return MM_OK;
}

// Morton sort + levels.  plan: learn and store the level counts (host reads).
static mm_status run_tree(mm_map *h, cudaStream_t st, bool plan) {
  const int64_t N = h->N;
  if (plan) {
    CK(h->keys_in.ensure(N));
    CK(h->keys.ensure(N));
    CK(h->idx_in.ensure(N));
    CK(h->idx.ensure(N));
    CK(h->sx.ensure(N));
    CK(h->sy.ensure(N));
    CK(h->sm.ensure(N));
  }
  LCH(launch_star_keys(h->pos_in.p, N, h->R0, h->keys_in.p, h->idx_in.p, st));
  if (N > 0) {
    CKS(cub_call(h, plan, [&](void *tmp, size_t &bytes) {
      return cub::DeviceRadixSort::SortPairs(tmp, bytes, h->keys_in.p, h->keys.p, h->idx_in.p,
                                             h->idx.p, (int)N, 0, 2 * MM_DMAX, st);
    }));
  }
  LCH(launch_gather_stars(h->pos_in.p, h->m_in.p, h->idx.p, N, h->sx.p, h->sy.p, h->sm.p, st));

  if (plan) {
    h->level_off.assign(MM_DMAX + 2, 0);
    h->level_cnt.assign(MM_DMAX + 2, 0);
    h->level_off[0] = 0;
    h->level_cnt[0] = 1;
    h->level_off[1] = 1;
    CK(h->d_level_off.ensure(MM_DMAX + 2));
    if (!h->pin) CK(cudaMallocHost(&h->pin, (8 + MM_DMAX + 2) * sizeof(int64_t)));
    CKS(upload_level_off(h, st));
    CK(h->code.ensure(5, true));
    CK(h->lvl.ensure(5, true));
    CK(h->sbeg.ensure(5, true));
    CK(h->send.ensure(5, true));
    CK(h->first_child.ensure(5, true));
  }
  LCH(launch_root_init(N, h->code.p, h->lvl.p, h->sbeg.p, h->send.p, st));
  for (int l = 0; l <= MM_DMAX; l++) {
    const int64_t n = h->level_cnt[l];
    if (plan) {
      CK(h->split.ensure(n));
      CK(h->scan.ensure(n));
    }
    TreeDev T = tree_dev(h);
    LCH(launch_level_split(T, l, n, h->leaf_size, h->split.p, st));
    CKS(cub_call(h, plan, [&](void *tmp, size_t &bytes) {
      return cub::DeviceScan::ExclusiveSum(tmp, bytes, h->split.p, h->scan.p, (int)n, st);
    }));
    if (plan) {
      const int32_t *src[2] = {h->scan.p + (n - 1), h->split.p + (n - 1)};
      int32_t ab[2];
      CKS(read_ints(h, st, 2, src, ab));
      const int64_t nxt = 4 * (int64_t)(ab[0] + ab[1]);
      h->level_cnt[l + 1] = nxt;
      h->level_off[l + 1] = h->level_off[l] + n;
      if (l + 2 <= MM_DMAX + 1) h->level_off[l + 2] = h->level_off[l + 1] + nxt;
      const int64_t need = h->level_off[l + 1] + nxt;
      CK(h->code.ensure(need, true));
      CK(h->lvl.ensure(need, true));
      CK(h->sbeg.ensure(need, true));
      CK(h->send.ensure(need, true));
      CK(h->first_child.ensure(need, true));
      CKS(upload_level_off(h, st));
      T = tree_dev(h);
    }
    LCH(launch_level_children(T, l, n, h->split.p, h->scan.p, h->code.p, h->lvl.p, h->sbeg.p,
                             h->send.p, h->first_child.p, st));
    if (h->level_cnt[l + 1] == 0) {
      if (plan) {
        h->depth = l;
        h->n_nodes = h->level_off[l + 1];
      }
      break;
    }
  }
  return MM_OK;
}

// Terms of a sub-cell's re-centred local expansion evaluated per ray.  The
// far-field stars of a leaf of half-length L lie outside its 3 x 3 block
// (L-inf distance >= 3L from the centre), so truncating the expansion about
// the leaf centre at order p errs by ~ (sqrt(2) L / 3L)^p at a corner.  About
// the centre of a sub-cell of half-length L/2^s the far field's ratio is
// sqrt(2) 2^-s / (2 + 2^-s), and the near stars moved into the sub-cell's
// expansion (outside its (2K+1)^2 block of sub-cells) add the ratio
// sqrt(2) / (2K+1); keep the fewest terms that do as well as order p at the
// leaf centre for the larger of the two.
static int eval_terms(int p, int s) {
  if (s <= 0 || p <= 2) return p;
  const double r0 = std::sqrt(2.0) / 3.0;
  const double q = std::ldexp(1.0, -s);
  const double rs = std::max(std::sqrt(2.0) * q / (2.0 + q), std::sqrt(2.0) / (2 * MM_NEAR_K + 1));
  const int pe = (int)std::ceil(p * std::log(r0) / std::log(rs) - 1e-9);
  return std::max(2, std::min(p, pe));
}

// Active region, expansions, leaf records and the lookup grid.
static mm_status run_fmm(mm_map *h, cudaStream_t st, bool plan) {
  const mm_params &P = h->P;
  const int64_t nn = h->n_nodes;
  TreeDev T = tree_dev(h);
  if (plan) {
    CK(h->col_cell.ensure(P.n[0]));
    CK(h->row_cell.ensure(P.n[1]));
    CK(h->node_act.ensure(nn));
    CK(h->leaf_flag.ensure(nn));
    CK(h->leaf_scan.ensure(nn));
    CK(h->node_active.ensure(nn));
  }
  LCH(launch_axis_cells(P.x0[0], P.h[0], P.n[0], h->R0, h->col_cell.p, st));
  LCH(launch_axis_cells(P.x0[1], P.h[1], P.n[1], h->R0, h->row_cell.p, st));
  LCH(launch_active_flags(T, nn, h->col_cell.p, h->col_lo, h->col_hi, h->row_cell.p, h->row_lo,
                          h->row_hi, h->node_act.p, h->leaf_flag.p, st));
  CKS(cub_call(h, plan, [&](void *tmp, size_t &bytes) {
    return cub::DeviceScan::ExclusiveSum(tmp, bytes, h->leaf_flag.p, h->leaf_scan.p, (int)nn, st);
  }));
  if (plan) {
    const int32_t *src[2] = {h->leaf_scan.p + (nn - 1), h->leaf_flag.p + (nn - 1)};
    int32_t ab[2];
    CKS(read_ints(h, st, 2, src, ab));
    h->n_active = (int64_t)ab[0] + ab[1];
    if (h->n_active <= 0) return fail(MM_ECUDA, "internal: no active leaf");
    CK(h->active_list.ensure(h->n_active));
  }
  LCH(launch_compact_leaves(nn, h->leaf_flag.p, h->leaf_scan.p, h->node_active.p,
                           h->active_list.p, st));

  if (plan) {
    // smallest active leaf and the deepest active level (plan-time analysis)
    std::vector<int32_t> al(h->n_active), lv(nn);
    CK(cudaMemcpyAsync(al.data(), h->active_list.p, h->n_active * sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lv.data(), h->lvl.p, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int ml = 0;
    for (int32_t id : al) ml = std::max(ml, (int)lv[id]);
    h->max_leaf_level = ml;
    h->min_leaf_L = h->R0 / (double)(1ll << ml);
    // sub-cells: finest-level cell indices must still resolve them
    h->sub = h->opt.sub_levels < 0 ? 0 : (h->opt.sub_levels == 0 ? MM_SUB_DEFAULT
                                                                  : h->opt.sub_levels);
    h->sub = std::max(0, std::min(h->sub, MM_DMAX - ml));
    // App. C.3: p > log2(<m^2>/<m> / (L |eps|)), eps = 1/10 of the pixel side
    if (h->p == 0) {
      double arg = (P.m2_over_m > 0.0) ? P.m2_over_m / (h->min_leaf_L * 0.1 * P.delta) : 1.0;
      int p = (int)std::floor(std::log2(std::max(arg, 1.0))) + 1;
      h->p = std::min(MM_PMAX, std::max(2, p));
    }
    h->p_eval = eval_terms(h->p, h->sub);
    const OpTables &ops = operator_tables(h->p);
    const std::vector<double2> &MMh = ops.MM, &MLh = ops.ML, &LLh = ops.LL;
    CK(h->MMop.ensure(MMh.size()));
    CK(h->MLop.ensure(MLh.size()));
    CK(h->LLop.ensure(LLh.size()));
    CK(cudaMemcpyAsync(h->MMop.p, MMh.data(), MMh.size() * sizeof(double2),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->MLop.p, MLh.data(), MLh.size() * sizeof(double2),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->LLop.p, LLh.data(), LLh.size() * sizeof(double2),
                       cudaMemcpyHostToDevice, st));  // (the cached tables outlive the copies)
    CK(h->mp.ensure((size_t)nn * (h->p + 1)));
    CK(h->loc.ensure((size_t)nn * (h->p + 1)));
    CK(h->near_cnt.ensure(h->n_active << (2 * h->sub)));
    CK(h->near_off.ensure(h->n_active << (2 * h->sub)));
    CK(h->err.ensure(1));
  }
  const int p = h->p, P1 = p + 1;
  CK(cudaMemsetAsync(h->err.p, 0, sizeof(unsigned), st));

  // up-sweep: P2M at every leaf, then M2M level by level towards the root
  LCH(launch_p2m(T, nn, p, h->mp.p, st));
  for (int l = h->depth - 1; l >= 0; l--)
    LCH(launch_m2m(T, l, h->level_cnt[l], p, h->MMop.p, h->mp.p, st));
  // down-sweep: levels 0 and 1 have no well-separated nodes
  CK(cudaMemsetAsync(h->loc.p, 0, (size_t)nn * P1 * sizeof(double2), st));
  for (int l = 2; l <= h->depth; l++)
    LCH(launch_local(T, l, h->level_cnt[l], p, h->node_act.p, h->MLop.p, h->LLop.p, h->mp.p,
                    h->loc.p, h->err.p, st));

  // near-field lists and leaf records, per sub-cell record
  FmmConst C;
  C.p = p;
  C.p_eval = h->p_eval;
  C.sub = h->sub;
  C.npix = P.npix;
  C.npix_y = P.npix_y;
  C.cull = h->opt.no_cull ? 0 : 1;
  C.kappa = P.kappa;
  C.gamma = P.gamma;
  C.kappa_star = P.kappa_star;
  C.x0 = P.x0[0];
  C.y0 = P.x0[1];
  C.hx = P.h[0];
  C.hy = P.h[1];
  C.lox = P.center_y[0] - P.half_length;
  C.loy = P.center_y[1] - P.half_length_y;
  C.delta = P.delta;
  C.x1 = P.x0[0] + (double)(P.n[0] - 1) * P.h[0];
  C.y1 = P.x0[1] + (double)(P.n[1] - 1) * P.h[1];
  C.rect_c1 = h->opt.star_rect[0];
  C.rect_c2 = h->opt.star_rect[1];
  const int64_t n_rec = h->n_active << (2 * h->sub);
  LCH(launch_near_count(T, C, h->n_active, h->active_list.p, h->near_cnt.p, h->err.p, st));
  CKS(cub_call(h, plan, [&](void *tmp, size_t &bytes) {
    return cub::DeviceScan::ExclusiveSum(tmp, bytes, h->near_cnt.p, h->near_off.p, (int)n_rec,
                                         st);
  }));
  if (plan) {
    const int32_t *src[2] = {h->near_off.p + (n_rec - 1), h->near_cnt.p + (n_rec - 1)};
    int32_t ab[2];
    CKS(read_ints(h, st, 2, src, ab));
    h->n_near = (int64_t)ab[0] + ab[1];
    CK(h->leaf.ensure(n_rec));
    CK(h->near_pos.ensure(h->n_near));
    CK(h->near_m.ensure(h->n_near));
    CK(h->coef.ensure((size_t)n_rec * coef_stride(h->p_eval)));
  }
  LCH(launch_leaf_finalize(T, C, h->n_active, h->active_list.p, h->near_off.p, h->near_cnt.p,
                          h->loc.p, h->leaf.p, h->near_pos.p, h->near_m.p, h->coef.p,
                          h->err.p, st));

  if (plan) {
    // lookup grid over the active cell rectangle, as deep as 4M entries allow
    const int32_t *src[4] = {h->col_cell.p + h->col_lo, h->col_cell.p + h->col_hi,
                             h->row_cell.p + h->row_lo, h->row_cell.p + h->row_hi};
    int32_t cr[4];
    CKS(read_ints(h, st, 4, src, cr));
    const int CX0 = cr[0], CX1 = cr[1], CY0 = cr[2], CY1 = cr[3];
    // (deep enough to resolve sub-cells where entries allow)
    int gl = std::min(MM_DMAX, h->max_leaf_level + h->sub);
    for (; gl > 0; gl--) {
      const int sh = MM_DMAX - gl;
      const int64_t w = (int64_t)(CX1 >> sh) - (CX0 >> sh) + 1;
      const int64_t hh = (int64_t)(CY1 >> sh) - (CY0 >> sh) + 1;
      if (w * hh <= (int64_t)1 << 22) break;
    }
    h->glevel = gl;
    h->gshift = MM_DMAX - gl;
    h->gx0 = CX0 >> h->gshift;
    h->gy0 = CY0 >> h->gshift;
    h->gw = (CX1 >> h->gshift) - h->gx0 + 1;
    h->gh = (CY1 >> h->gshift) - h->gy0 + 1;
    CK(h->grid.ensure((size_t)h->gw * h->gh));
  }
  LCH(launch_lookup_grid(T, h->node_active.p, h->glevel, h->sub, h->gx0, h->gy0, h->gw, h->gh,
                        h->grid.p, st));
  return MM_OK;
}

static int shoot_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  per_sm = MM_SHOOT_MINB;  // resident 256-thread blocks per SM
  return std::max(1, sms * per_sm);
}

static void fill_mapdev(mm_map *h) {
  const mm_params &P = h->P;
  MapDev &M = h->md;
  memset(&M, 0, sizeof M);
  M.n0 = P.n[0];
  M.n1 = P.n[1];
  M.row_begin = h->row_lo;
  M.row_end = h->row_hi;
  M.col_begin = h->col_lo;
  M.col_end = h->col_hi;
  M.strips = (int32_t)((h->col_hi - h->col_lo + MM_STRIP - 1) / MM_STRIP);
  if (h->opt.rows_per_item <= 0) {
    // longest items (fewest re-shot first rows) that still give every
    // resident warp >= 16 items to balance over
    const int64_t rows = h->row_hi - h->row_lo, want = 16 * 8 * (int64_t)shoot_grid();
    int rpi = 256;
    while (rpi > 16 && (int64_t)M.strips * ((rows + rpi - 1) / rpi) < want) rpi >>= 1;
    h->rows_per_item = rpi;
  }
  M.rows_per_item = h->rows_per_item;
  M.row_blocks = (h->row_hi - h->row_lo + h->rows_per_item - 1) / h->rows_per_item;
  M.item_stride = 1;
  M.work_begin = 0;
  M.col_cell = h->col_cell.p;
  M.row_cell = h->row_cell.p;
  M.grid = h->grid.p;
  M.glevel = h->glevel;
  M.gshift = h->gshift;
  M.gx0 = h->gx0;
  M.gy0 = h->gy0;
  M.gw = h->gw;
  M.gh = h->gh;
  M.first_child = h->first_child.p;
  M.node_active = h->node_active.p;
  M.leaf = h->leaf.p;
  M.near_pos = h->near_pos.p;
  M.near_m = h->near_m.p;
  M.coef = h->coef.p;
  M.p = h->p_eval;
  M.cull = h->opt.no_cull ? 0 : 1;
  M.sub = h->sub;
  M.node_level = h->lvl.p;
  M.square_cells = (P.h[0] == P.h[1]) ? 1 : 0;
  const double ak = 1.0 - P.kappa + P.kappa_star;
  M.A1 = (float)((ak + P.gamma) * P.h[0] / P.delta);
  M.A2 = (float)((ak - P.gamma) * P.h[1] / P.delta);
  M.sx = (float)(1.0 / (P.h[0] * P.delta));
  M.sy = (float)(P.h[1] / (P.h[0] * P.h[0] * P.delta));
  M.rho = (float)((P.h[1] / P.h[0]) * (P.h[1] / P.h[0]));
  // twice the image triangle's area in pixel units, over the threshold |mu|
  M.crit_area2 = (float)(P.h[0] * P.h[1] / (P.delta * P.delta) /
                         (h->opt.critical_mu > 0.0 ? h->opt.critical_mu : 1e3));
  M.npix = P.npix;
  M.npix_y = P.npix_y;
  M.err = h->err.p;
  M.acc = h->acc.p;
  M.span = h->span.p;
  M.stat = h->stat.p;
  M.bigq = reinterpret_cast<TriJob *>(h->bigq.p);
  M.bigq_n = h->bigq_n.p;
  M.bigq_cap = h->bigq_cap;
}

static mm_status clear_map(mm_map *h, cudaStream_t st) {
  const size_t np = (size_t)h->P.npix * h->P.npix_y;
  CK(cudaMemsetAsync(h->acc.p, 0, np * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(h->span.p, 0, (size_t)h->P.npix_y * (h->P.npix + 1) * sizeof(unsigned long long),
                     st));
  CK(cudaMemsetAsync(h->stat.p, 0, 8 * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(h->counter.p, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(h->bigq_n.p, 0, 2 * sizeof(unsigned long long), st));
  return MM_OK;
}

// mu per accumulator unit: a triangle's 2^32 units stand for its image
// area h_x h_y / 2 (IPM); a ray's one count for its cell's h_x h_y (IRS)
static double map_scale(const mm_map *h) {
  const mm_params &P = h->P;
  if (h->mode == MM_FMM_IRS) return P.h[0] * P.h[1] / (P.delta * P.delta);
  return std::ldexp(0.5 * P.h[0] * P.h[1] / (P.delta * P.delta), -32);
}

// Larger triangles (queued for the second pass) expected from `cells` cells:
// the autotuner's count scaled to them, else one per 12 cells.
static int64_t est_jobs(const mm_map *h, int64_t cells) {
  if (h->jobs_pm >= 0) return (int64_t)std::ceil((double)cells * h->jobs_pm / 1048576.0);
  return cells / 12;
}

static mm_status alloc_map_buffers(mm_map *h) {
  const size_t np = (size_t)h->P.npix * h->P.npix_y;
  CK(h->acc.ensure(np));
  CK(h->span.ensure((size_t)h->P.npix_y * (h->P.npix + 1)));
  CK(h->map.ensure(np));
  CK(h->stat.ensure(8));
  CK(h->counter.ensure(1));
  // Queue for the second IPM pass.  It pays while the map's accumulators
  // (acc + row-difference array, 16 B per pixel) stay in L2: the second pass
  // then finds their lines there.  A larger map's lines are gone by the time
  // the second pass reaches a triangle, whereas the first pass deals it where
  // the lines are hot (measured on 5000^2 and 10000^2 maps: no queue was 18 %
  // and 8 % faster than a queue, and first passes split into segments to fit
  // the queue were 17-44 % slower).  Default, for maps that fit half the L2
  // (else none): the larger triangles the autotuner's sampled runs counted,
  // with a quarter to spare, else 1 slot per 12 cells; 2^16 .. 2^27 slots
  // (48 B each).  When that much device memory is not to be had, 2^20 slots,
  // then none.  Batches that do not fit are dealt out by the first kernel.
  {
    const int64_t cells = (h->col_hi - h->col_lo) * (h->row_hi - h->row_lo);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device);
    const bool fits_l2 = 16.0 * (double)h->P.npix * (double)h->P.npix_y <= 0.5 * (double)l2;
    const int32_t want = h->mode == MM_FMM_IRS ? -1 : h->opt.big_queue_slots;
    const int64_t est = est_jobs(h, cells);
    const int64_t slots = h->jobs_pm >= 0 ? est + est / 4 + 4096 : est;
    h->bigq_cap = want < 0 ? 0
                  : want > 0 ? (int64_t)want
                  : fits_l2  ? std::min<int64_t>(int64_t(1) << 27,
                                                 std::max<int64_t>(int64_t(1) << 16, slots))
                             : 0;
    if (h->bigq_cap > 0) {
      cudaError_t e = h->bigq.ensure((size_t)h->bigq_cap * MM_TRIJOB_BYTES);
      if (e == cudaErrorMemoryAllocation && want == 0) {
        cudaGetLastError();  // (clears the failed allocation's error)
        h->bigq_cap = std::min<int64_t>(h->bigq_cap, int64_t(1) << 20);
        e = h->bigq.ensure((size_t)h->bigq_cap * MM_TRIJOB_BYTES);
        if (e == cudaErrorMemoryAllocation) {
          cudaGetLastError();
          h->bigq_cap = 0;
          e = cudaSuccess;
        }
      }
      CK(e);
    }
    CK(h->bigq_n.ensure(2));
    // a map that fits: the first pass runs in segments so that each
    // segment's larger triangles fit the queue
    h->segments = 1;
    if (h->bigq_cap > 0 && h->mode == MM_FMM_FP32 && fits_l2)
      h->segments = std::max<int64_t>(1, (est + h->bigq_cap - 1) / h->bigq_cap);
    if (h->opt.time_stages && (int64_t)h->seg_ev.size() < 2 * h->segments) {
      const size_t have = h->seg_ev.size();
      h->seg_ev.resize(2 * h->segments, nullptr);
      for (size_t k = have; k < h->seg_ev.size(); k++) CK(cudaEventCreate(&h->seg_ev[k]));
    }
  }
  CK(h->err.ensure(1));
  CK(cudaMemset(h->err.p, 0, sizeof(unsigned)));  // read after the plan in every mode
  CK(h->d_md.ensure(1));
  return MM_OK;
}

static mm_status record(mm_map *h, int k, cudaStream_t st) {
  if (h->opt.time_stages) CK(cudaEventRecord(h->ev[k], st));
  return MM_OK;
}

// The FMM pipeline up to (and including) the lookup grid.
static mm_status prepare(mm_map *h, cudaStream_t st) {
  CKS(run_tree(h, st, false));
  CKS(record(h, 1, st));
  CKS(run_fmm(h, st, false));
  h->prepared = true;
  return MM_OK;
}

// A rectangle of cells [r0, r1) x [c0, c1) of the ray grid.
struct CellRect {
  int64_t r0, r1, c0, c1;
};

// The handle's descriptor restricted to the cells of `r` (the plan -- tree,
// expansions, lookup, culling bounds, queue -- is unchanged).
static MapDev restrict_mapdev(const mm_map *h, const CellRect &r) {
  MapDev m = h->md;
  m.row_begin = r.r0;
  m.row_end = r.r1;
  m.col_begin = r.c0;
  m.col_end = r.c1;
  m.strips = (int32_t)((r.c1 - r.c0 + MM_STRIP - 1) / MM_STRIP);
  m.row_blocks = (r.r1 - r.r0 + h->rows_per_item - 1) / h->rows_per_item;
  return m;
}

// First-pass segments for `cells` cells: their larger triangles must fit
// the queue (maps that fit L2, polygon mapping only).
static int64_t segments_for(const mm_map *h, int64_t cells) {
  if (h->segments <= 1 || h->bigq_cap <= 0) return 1;
  return std::max<int64_t>(1, (est_jobs(h, cells) + h->bigq_cap - 1) / h->bigq_cap);
}

// One run of the handle's map over its cells, or over the rectangle `rect`
// of them (NULL: all).
static mm_status run_one(mm_map *h, cudaStream_t st, const CellRect *rect = nullptr) {
  const mm_params &P = h->P;
  const CellRect all = {h->row_lo, h->row_hi, h->col_lo, h->col_hi};
  const CellRect R = rect ? *rect : all;
  h->launches = 0;
  h->led_batch = false;
  CKS(record(h, 0, st));
  CKS(clear_map(h, st));
  if (h->mode == MM_PLAIN_FP64) {
    CKS(record(h, 1, st));
    CKS(record(h, 2, st));
    DirectConst C;
    C.kappa = P.kappa;
    C.gamma = P.gamma;
    C.kappa_star = P.kappa_star;
    C.x0 = P.x0[0];
    C.y0 = P.x0[1];
    C.hx = P.h[0];
    C.hy = P.h[1];
    C.lox = P.center_y[0] - P.half_length;
    C.loy = P.center_y[1] - P.half_length_y;
    C.delta = P.delta;
    C.rect_c1 = h->opt.star_rect[0];
    C.rect_c2 = h->opt.star_rect[1];
    LCH(launch_direct64_vertices(h->sx.p, h->sy.p, h->sm.p, h->N, C, R.c0, R.c1 - R.c0 + 1,
                                 R.r0, R.r1, h->verts.p, st));
    LCH(launch_ipm_vertices(h->d_md.p, h->verts.p, R.c1 - R.c0 + 1, R.r0, R.r1, h->counter.p,
                            h->err.p, shoot_grid(), st));
    CKS(record(h, 5, st));
    LCH(launch_big_ipm(h->md, st));
  } else {
    // The plan of mm_create ran the whole tree and expansion pipeline on the
    // same stars; the first run uses that result instead of repeating it.
    if (h->fresh) {
      h->fresh = false;
      CKS(record(h, 1, st));
    } else {
      CKS(prepare(h, st));
    }
    CKS(record(h, 2, st));
    const MapDev base = rect ? restrict_mapdev(h, R) : h->md;
    const int64_t work =
        (int64_t)base.strips * ((base.row_blocks + base.item_stride - 1) / base.item_stride);
    if (h->mode == MM_FMM_IRS) {
      LCH(launch_shoot_irs(base, work, base.square_cells != 0, h->counter.p, h->err.p, st));
      h->last_segments = 0;
      CKS(record(h, 5, st));
      CKS(record(h, 3, st));
      LCH(launch_normalize(h->acc.p, h->span.p, P.npix, P.npix_y, map_scale(h), h->map.p, st));
      CKS(record(h, 4, st));
      h->ev_recorded = h->opt.time_stages != 0;
      h->last_stream = st;
      h->ran = true;
      return MM_OK;
    }
    const int64_t segs = rect ? segments_for(h, (R.r1 - R.r0) * (R.c1 - R.c0)) : h->segments;
    const int64_t nseg = std::max<int64_t>(1, std::min(segs, work));
    const int64_t per = (work + nseg - 1) / nseg;
    int64_t k = 0;
    for (int64_t w0 = 0; w0 < work; w0 += per, k++) {
      if (w0 > 0) {  // the previous segment's second pass has drained the queue
        CK(cudaMemsetAsync(h->counter.p, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(h->bigq_n.p, 0, 2 * sizeof(unsigned long long), st));
      }
      MapDev ms = base;
      ms.work_begin = -w0;  // this launch's item w is item w0 + w of the map
      LCH(launch_shoot_ipm(h->d_md.p, &ms, 1, std::min(per, work - w0), base.square_cells != 0,
                          h->counter.p, h->err.p, shoot_grid(), st));
      if (h->opt.time_stages) CK(cudaEventRecord(h->seg_ev[2 * k], st));
      LCH(launch_big_ipm(ms, st));
      if (h->opt.time_stages) CK(cudaEventRecord(h->seg_ev[2 * k + 1], st));
    }
    h->last_segments = k;
    CKS(record(h, 5, st));
  }
  CKS(record(h, 3, st));
  LCH(launch_normalize(h->acc.p, h->span.p, P.npix, P.npix_y, map_scale(h), h->map.p, st));
  CKS(record(h, 4, st));
  h->ev_recorded = h->opt.time_stages != 0;
  h->last_stream = st;
  h->ran = true;
  return MM_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *mm_last_error(void) { return g_err.c_str(); }

mm_status mm_derive_params(double kappa_tot, double shear, double smooth_fraction,
                           int64_t n_stars, const double *masses, double half_length,
                           int32_t npix, double rays_per_pixel, const mm_options *opt,
                           mm_params *out) {
  if (!out) return fail(MM_EINVAL, "out is NULL");
  mm_options o{};
  if (opt) o = *opt;
  return derive(kappa_tot, shear, smooth_fraction, n_stars, masses, half_length, npix,
                rays_per_pixel, o, *out);
}

static mm_status create_impl(mm_map *h, double kappa_tot, double shear, double smooth_fraction,
                             int64_t n_stars, const double *masses, const double *pos_xy,
                             double half_length, int32_t npix, double rays_per_pixel,
                             int32_t fmm_order, int32_t leaf_size) {
  mm_params &P = h->P;
  CKS(derive(kappa_tot, shear, smooth_fraction, n_stars, masses, half_length, npix,
             rays_per_pixel, h->opt, P));
  if (fmm_order < 0 || fmm_order > MM_PMAX)
    return fail(MM_EINVAL, "fmm_order %d outside [0, %d]", fmm_order, MM_PMAX);
  if (leaf_size < 0 || leaf_size > 1024)
    return fail(MM_EINVAL, "leaf_size %d outside [0, 1024]", leaf_size);
  if (h->opt.mode != MM_FMM_FP32 && h->opt.mode != MM_PLAIN_FP64 && h->opt.mode != MM_FMM_IRS)
    return fail(MM_EINVAL, "unknown mode %d", h->opt.mode);
  if (!(h->opt.critical_mu >= 0.0) || !std::isfinite(h->opt.critical_mu))
    return fail(MM_EINVAL, "critical_mu %g is negative or not finite", h->opt.critical_mu);
  if (h->opt.big_queue_slots < -1)
    return fail(MM_EINVAL, "big_queue_slots %d below -1", h->opt.big_queue_slots);
  if (h->opt.sub_levels < -1 || h->opt.sub_levels > MM_SUB_MAX)
    return fail(MM_EINVAL, "sub_levels %d outside [-1, %d]", h->opt.sub_levels, MM_SUB_MAX);
  if (n_stars > 0 && !pos_xy) return fail(MM_EINVAL, "pos_xy is NULL");
  if (n_stars > 2000000000LL) return fail(MM_EINVAL, "too many stars");
  h->mode = h->opt.mode;
  h->p = fmm_order;
  h->leaf_size = leaf_size ? leaf_size : 32;
  h->N = n_stars;
  h->rows_per_item = h->opt.rows_per_item > 0 ? std::min(h->opt.rows_per_item, 4096) : 256;

  // cell-row band
  const int64_t rows = P.n[1] - 1;
  h->row_lo = 0;
  h->row_hi = rows;
  if (h->opt.row_begin != 0 || h->opt.row_end != 0) {
    if (h->opt.row_begin < 0 || h->opt.row_end <= h->opt.row_begin || h->opt.row_end > rows)
      return fail(MM_EINVAL, "row band [%lld, %lld) outside [0, %lld)",
                  (long long)h->opt.row_begin, (long long)h->opt.row_end, (long long)rows);
    h->row_lo = h->opt.row_begin;
    h->row_hi = h->opt.row_end;
  }
  // cell-column band
  const int64_t cols = P.n[0] - 1;
  h->col_lo = 0;
  h->col_hi = cols;
  if (h->opt.col_begin != 0 || h->opt.col_end != 0) {
    if (h->opt.col_begin < 0 || h->opt.col_end <= h->opt.col_begin || h->opt.col_end > cols)
      return fail(MM_EINVAL, "column band [%lld, %lld) outside [0, %lld)",
                  (long long)h->opt.col_begin, (long long)h->opt.col_end, (long long)cols);
    h->col_lo = h->opt.col_begin;
    h->col_hi = h->opt.col_end;
  }

  // star extent, coverage and root square
  double ext = 0.0, bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
  for (int64_t i = 0; i < n_stars; i++) {
    const double x = pos_xy[2 * i], y = pos_xy[2 * i + 1];
    if (!std::isfinite(x) || !std::isfinite(y))
      return fail(MM_EINVAL, "star %lld has a non-finite position", (long long)i);
    ext = std::max(ext, std::max(std::fabs(x), std::fabs(y)));
    bx0 = std::min(bx0, x);
    bx1 = std::max(bx1, x);
    by0 = std::min(by0, y);
    by1 = std::max(by1, y);
  }
  const double gx0 = P.x0[0], gx1 = P.x0[0] + (double)(P.n[0] - 1) * P.h[0];
  const double gy0 = P.x0[1], gy1 = P.x0[1] + (double)(P.n[1] - 1) * P.h[1];
  const bool explicit_region = h->opt.img_half[0] > 0.0 && h->opt.img_half[1] > 0.0;
  const bool rect_region = h->opt.star_rect[0] != 0.0 || h->opt.star_rect[1] != 0.0;
  if (P.kappa_star > 0.0 && !explicit_region &&
      (gx0 < bx0 || gx1 > bx1 || gy0 < by0 || gy1 > by1))
    return fail(MM_EINVAL,
                "the stars' bounding box [%g, %g] x [%g, %g] does not cover the shooting "
                "region [%g, %g] x [%g, %g]",
                bx0, bx1, by0, by1, gx0, gx1, gy0, gy1);
  if (P.kappa_star > 0.0 && !explicit_region && !rect_region) {
    // Sec. 3.1: the circular sheet deflects by -kappa_star z only inside the
    // disk the stars fill (radius max |z_i| about the origin); every ray must
    // lie inside it, so each corner of the ray grid must
    double r2 = 0.0;
    for (int64_t i = 0; i < n_stars; i++)
      r2 = std::max(r2, pos_xy[2 * i] * pos_xy[2 * i] + pos_xy[2 * i + 1] * pos_xy[2 * i + 1]);
    const double cx[2] = {gx0, gx1}, cy[2] = {gy0, gy1};
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        if (cx[a] * cx[a] + cy[b] * cy[b] > r2)
          return fail(MM_EINVAL,
                      "ray-grid corner (%g, %g) lies outside the star disk (radius max |z_i| "
                      "= %g about the origin), where the circular sheet of Sec. 3.1 no "
                      "longer deflects by -kappa_star z: use a larger star disk",
                      cx[a], cy[b], std::sqrt(r2));
  }
  if (rect_region) {
    // App. B: rectangular star region centred on the origin
    const double c1 = h->opt.star_rect[0], c2 = h->opt.star_rect[1];
    if (!(c1 > 0.0 && c2 > 0.0 && std::isfinite(c1) && std::isfinite(c2)))
      return fail(MM_EINVAL, "star_rect (%g, %g) must be two positive half-widths", c1, c2);
    if (!(std::max(std::fabs(gx0), std::fabs(gx1)) < c1 &&
          std::max(std::fabs(gy0), std::fabs(gy1)) < c2))
      return fail(MM_EINVAL,
                  "the shooting region [%g, %g] x [%g, %g] is not inside the star rectangle "
                  "|x| < %g, |y| < %g",
                  gx0, gx1, gy0, gy1, c1, c2);
  }
  ext = std::max(ext, std::max(std::max(std::fabs(gx0), std::fabs(gx1)),
                               std::max(std::fabs(gy0), std::fabs(gy1))));
  h->R0 = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(ext * 1.0001, 1e-3))));
  if (h->R0 <= ext) h->R0 *= 2.0;

  CK(cudaGetDevice(&h->device));
  CK(cudaStreamCreateWithFlags(&h->plan_stream, cudaStreamNonBlocking));
  keep_pool_memory(h->device);
  AllocStream alloc_on(h->plan_stream);
  for (int k = 0; k < 6; k++) CK(cudaEventCreate(&h->ev[k]));
  cudaStream_t st = h->plan_stream;

  // stars to the device
  CK(h->pos_in.ensure(2 * n_stars));
  CK(h->m_in.ensure(n_stars));
  if (n_stars > 0) {
    CK(cudaMemcpyAsync(h->pos_in.p, pos_xy, 2 * n_stars * sizeof(double),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->m_in.p, masses, n_stars * sizeof(double), cudaMemcpyHostToDevice,
                       st));
  }
  CKS(alloc_map_buffers(h));
  if (h->mode == MM_PLAIN_FP64) {
    CK(h->sx.ensure(n_stars));
    CK(h->sy.ensure(n_stars));
    CK(h->sm.ensure(n_stars));
    // unsorted SoA copy
    CK(h->idx.ensure(n_stars));
    std::vector<int32_t> id(n_stars);
    for (int64_t i = 0; i < n_stars; i++) id[i] = (int32_t)i;
    if (n_stars > 0)
      CK(cudaMemcpyAsync(h->idx.p, id.data(), n_stars * sizeof(int32_t), cudaMemcpyHostToDevice,
                         st));
    LCH(launch_gather_stars(h->pos_in.p, h->m_in.p, h->idx.p, n_stars, h->sx.p, h->sy.p, h->sm.p,
                           st));
    CK(h->verts.ensure((size_t)(h->col_hi - h->col_lo + 1) * (h->row_hi - h->row_lo + 1)));
    CK(cudaStreamSynchronize(st));
  } else {
    CKS(run_tree(h, st, true));
    CKS(run_fmm(h, st, true));
    CK(cudaStreamSynchronize(st));
    h->prepared = true;
    h->fresh = true;
  }
  fill_mapdev(h);
  CK(cudaMemcpyAsync(h->d_md.p, &h->md, sizeof(MapDev), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  unsigned e = 0;
  CK(cudaMemcpy(&e, h->err.p, sizeof e, cudaMemcpyDeviceToHost));
  if (e & ERR_TREE_INVARIANT) return fail(MM_ECUDA, "internal: quadtree invariant violated");
  if (e & ERR_RECT_CORNER)
    return fail(MM_EINVAL,
                "a corner of star_rect lies within two half-diagonals of a ray-grid sub-cell: "
                "widen the rectangle or use sub-cells (sub_levels 1 or 2)");
  h->last_stream = st;
  return MM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: the settings that change the speed of a map but not what it
// computes (beyond the FMM tolerances), chosen by timing candidate plans.
// ---------------------------------------------------------------------------

// jobs_pm: the larger triangles per 2^20 cells that the chosen candidate's
// sampled run counted (-1: none recorded), for the second-pass queue's size
struct TuneChoice {
  int32_t leaf = 32, sub = 0, rpi = 0, jobs_pm = -1;
};

static bool tune_valid(const TuneChoice &c) {
  return c.leaf >= 1 && c.leaf <= 1024 && c.sub >= -1 && c.sub <= MM_SUB_MAX && c.rpi >= 0 &&
         c.rpi <= 4096 && c.jobs_pm >= -1 && c.jobs_pm <= (1 << 21);
}

static int log2_bucket(double v) { return v >= 1.0 ? (int)std::floor(std::log2(v)) : 0; }

static std::string tune_key(int dev, const mm_options &o, int32_t fmm_order, int32_t leaf_size,
                            int64_t n_stars, const mm_params &P) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  char b[256];
  snprintf(b, sizeof b, "sm_%d%d/p%d/leaf%d/sub%d/rpi%d/nstar%d/rays%d/npix%d", major, minor,
           fmm_order, leaf_size, o.sub_levels, o.rows_per_item, log2_bucket((double)n_stars),
           log2_bucket((double)P.n[0] * (double)P.n[1]),
           log2_bucket((double)P.npix * (double)P.npix_y) / 2);
  return b;
}

// integer value of "name": in one line of the cache
static bool json_int(const std::string &line, const char *name, int32_t &v) {
  const std::string pat = std::string("\"") + name + "\":";
  size_t k = line.find(pat);
  if (k == std::string::npos) return false;
  k += pat.size();
  while (k < line.size() && line[k] == ' ') k++;
  const char *s = line.c_str() + k;
  char *end = nullptr;
  const long x = strtol(s, &end, 10);
  if (end == s || x < -2147483647L || x > 2147483647L) return false;
  v = (int32_t)x;
  return true;
}

static bool tune_cache_lookup(const char *path, const std::string &key, TuneChoice &out) {
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  const std::string want = "\"key\": \"" + key + "\"";
  bool found = false;
  char buf[1024];
  while (fgets(buf, sizeof buf, f)) {
    const std::string line(buf);
    if (line.find(want) == std::string::npos) continue;
    TuneChoice c;
    if (!json_int(line, "jobs_per_mcell", c.jobs_pm)) c.jobs_pm = -1;  // (older lines)
    if (json_int(line, "leaf_size", c.leaf) && json_int(line, "sub_levels", c.sub) &&
        json_int(line, "rows_per_item", c.rpi) && tune_valid(c)) {
      out = c;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void tune_cache_store(const char *path, const std::string &key, const TuneChoice &c,
                             double ms) {
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f,
          "{\"key\": \"%s\", \"leaf_size\": %d, \"sub_levels\": %d, \"rows_per_item\": %d, "
          "\"jobs_per_mcell\": %d, \"ms_estimate\": %.4f}\n",
          key.c_str(), c.leaf, c.sub, c.rpi, c.jobs_pm, ms);
  fclose(f);
}

struct CreateArgs {
  double kappa, gamma, s;
  int64_t n_stars;
  const double *masses, *pos_xy;
  double half_length;
  int32_t npix;
  double rays_per_pixel;
  int32_t fmm_order;
};

// Device time of one sampled run of a trial handle, scaled to the whole grid:
// tree + expansions + stride x mapping + normalisation.
static mm_status trial_ms(mm_map *t, double scale, double &ms) {
  CKS(run_one(t, t->plan_stream));
  CK(cudaStreamSynchronize(t->plan_stream));
  unsigned e = 0;
  CK(cudaMemcpy(&e, t->err.p, sizeof e, cudaMemcpyDeviceToHost));
  if (e) return fail(MM_ECUDA, "internal: autotune trial run reported error 0x%x", e);
  float a = 0.f, b = 0.f, c = 0.f;
  CK(cudaEventElapsedTime(&a, t->ev[0], t->ev[2]));
  CK(cudaEventElapsedTime(&b, t->ev[2], t->ev[3]));
  CK(cudaEventElapsedTime(&c, t->ev[3], t->ev[4]));
  ms = (double)a + scale * (double)b + (double)c;
  return MM_OK;
}

// Times every candidate (leaf_size x sub_levels x rows_per_item over the
// settings left 0) and writes the fastest into o / leaf_size, and the
// larger triangles per 2^20 cells its sampled run counted into jobs_pm.
static mm_status autotune(const CreateArgs &a, mm_options &o, int32_t &leaf_size, int &tuned,
                          double &ms_tune, int32_t &jobs_pm) {
  tuned = 0;
  ms_tune = 0.0;
  jobs_pm = -1;
  if (!o.autotune || o.mode != MM_FMM_FP32) return MM_OK;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int32_t> leafs = {leaf_size}, subs = {o.sub_levels}, rpis = {o.rows_per_item};
  if (leaf_size == 0) leafs = {16, 32, 64};
  if (o.sub_levels == 0) subs = {1, 2};
  if (o.rows_per_item == 0) rpis = {0, 64, 512};
  if (leafs.size() * subs.size() * rpis.size() == 1) return MM_OK;
  mm_params P;
  CKS(derive(a.kappa, a.gamma, a.s, a.n_stars, a.masses, a.half_length, a.npix,
             a.rays_per_pixel, o, P));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const std::string key = tune_key(dev, o, a.fmm_order, leaf_size, a.n_stars, P);
  TuneChoice best;
  if (tune_cache_lookup(o.tune_cache, key, best)) {
    tuned = 2;
  } else {
    double best_ms = 1e300;
    bool any = false;
    mm_status last = MM_OK;
    std::string last_msg;
    for (int32_t leaf : leafs)
      for (int32_t sub : subs) {
        mm_map *t = new (std::nothrow) mm_map();
        if (!t) return fail(MM_ENOMEM, "host allocation failed");
        t->opt = o;
        t->opt.autotune = 0;
        t->opt.tune_cache = nullptr;
        t->opt.time_stages = 1;
        t->opt.sub_levels = sub;
        t->opt.rows_per_item = 0;
        mm_status s = create_impl(t, a.kappa, a.gamma, a.s, a.n_stars, a.masses, a.pos_xy,
                                  a.half_length, a.npix, a.rays_per_pixel, a.fmm_order, leaf);
        for (size_t r = 0; s == MM_OK && r < rpis.size(); r++) {
          t->opt.rows_per_item = rpis[r];
          t->rows_per_item = rpis[r] > 0 ? std::min(rpis[r], 4096) : 256;
          fill_mapdev(t);
          // every k-th row block: >= 4 work items per resident warp remain
          const int64_t items = (int64_t)t->md.strips * t->md.row_blocks;
          const int64_t k = std::max<int64_t>(
              1, std::min<int64_t>(16, items / (4 * 8 * (int64_t)shoot_grid())));
          t->md.item_stride = k;
          const int64_t sampled = (t->md.row_blocks + k - 1) / k;
          const double scale = (double)t->md.row_blocks / (double)sampled;
          cudaError_t ce = cudaMemcpy(t->d_md.p, &t->md, sizeof(MapDev), cudaMemcpyHostToDevice);
          if (ce != cudaSuccess) {
            s = fail(MM_ECUDA, "autotune: %s", cudaGetErrorString(ce));
            break;
          }
          double est = 1e300;
          for (int rep = 0; s == MM_OK && rep < 3; rep++) {
            double ms = 0.0;
            s = trial_ms(t, scale, ms);
            if (rep > 0) est = std::min(est, ms);  // the first run is a warm-up
          }
          if (s == MM_OK && est < best_ms) {
            best_ms = est;
            best.leaf = leaf;
            best.sub = sub;
            best.rpi = rpis[r];
            any = true;
            // the larger triangles of the sampled run (statistics 3 and 4),
            // scaled to the whole grid, per 2^20 cells
            unsigned long long st[8] = {};
            ce = cudaMemcpy(st, t->stat.p, sizeof st, cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) {
              s = fail(MM_ECUDA, "autotune: %s", cudaGetErrorString(ce));
              break;
            }
            const double cells = (double)(t->col_hi - t->col_lo) * (double)(t->row_hi - t->row_lo);
            const double pm = cells > 0.0 ? (double)(st[3] + st[4]) * scale * 1048576.0 / cells
                                          : 0.0;
            best.jobs_pm = (int32_t)std::min(std::ceil(pm), (double)(1 << 21));
          }
        }
        if (s != MM_OK) {
          last = s;
          last_msg = g_err;
        }
        mm_destroy(t);
        if (s == MM_ETIMEOUT || s == MM_ECUDA) {
          g_err = last_msg;
          return s;  // a device error is not a candidate's property
        }
      }
    if (!any) {
      g_err = last_msg;
      return last != MM_OK ? last : fail(MM_ESTATE, "autotune: no candidate ran");
    }
    g_err.clear();
    tuned = 1;
    tune_cache_store(o.tune_cache, key, best, best_ms);
  }
  leaf_size = best.leaf;
  o.sub_levels = best.sub;
  o.rows_per_item = best.rpi;
  jobs_pm = best.jobs_pm;
  ms_tune = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
  return MM_OK;
}

mm_status mm_create(double kappa_tot, double shear, double smooth_fraction, int64_t n_stars,
                    const double *masses, const double *pos_xy, double half_length,
                    int32_t npix, double rays_per_pixel, int32_t fmm_order, int32_t leaf_size,
                    const mm_options *opt, mm_map **out) {
  if (!out) return fail(MM_EINVAL, "out is NULL");
  *out = nullptr;
  mm_map *h = new (std::nothrow) mm_map();
  if (!h) return fail(MM_ENOMEM, "host allocation failed");
  if (opt) h->opt = *opt;
  const CreateArgs args = {kappa_tot, shear,        smooth_fraction, n_stars,  masses, pos_xy,
                           half_length, npix, rays_per_pixel,  fmm_order};
  mm_status s = MM_OK;
  if (h->opt.autotune && (leaf_size < 0 || leaf_size > 1024 || fmm_order < 0 ||
                          fmm_order > MM_PMAX || h->opt.sub_levels < -1 ||
                          h->opt.sub_levels > MM_SUB_MAX))
    h->opt.autotune = 0;  // create_impl reports the invalid argument
  if (h->opt.autotune)
    s = autotune(args, h->opt, leaf_size, h->tuned, h->ms_tune, h->jobs_pm);
  h->opt.autotune = 0;
  h->opt.tune_cache = nullptr;
  if (s == MM_OK)
    s = create_impl(h, kappa_tot, shear, smooth_fraction, n_stars, masses, pos_xy, half_length,
                    npix, rays_per_pixel, fmm_order, leaf_size);
  if (s != MM_OK) {
    std::string msg = g_err;
    mm_destroy(h);
    g_err = msg;
    return s;
  }
  g_err.clear();
  *out = h;
  return MM_OK;
}

mm_status mm_run(mm_map *h, void *stream) {
  if (!h) return fail(MM_EINVAL, "handle is NULL");
  if (h->timed_out) return fail(MM_ESTATE, "a previous run timed out");
  CK(cudaSetDevice(h->device));
  return run_one(h, (cudaStream_t)stream);
}

mm_status mm_run_cells(mm_map *h, int64_t row_begin, int64_t row_end, int64_t col_begin,
                       int64_t col_end, void *stream) {
  if (!h) return fail(MM_EINVAL, "handle is NULL");
  if (h->timed_out) return fail(MM_ESTATE, "a previous run timed out");
  if (row_begin < h->row_lo || row_end <= row_begin || row_end > h->row_hi ||
      col_begin < h->col_lo || col_end <= col_begin || col_end > h->col_hi)
    return fail(MM_EINVAL,
                "cell rectangle rows [%lld, %lld) x columns [%lld, %lld) is empty or outside "
                "the handle's rows [%lld, %lld) x columns [%lld, %lld)",
                (long long)row_begin, (long long)row_end, (long long)col_begin,
                (long long)col_end, (long long)h->row_lo, (long long)h->row_hi,
                (long long)h->col_lo, (long long)h->col_hi);
  CK(cudaSetDevice(h->device));
  const CellRect r = {row_begin, row_end, col_begin, col_end};
  return run_one(h, (cudaStream_t)stream, &r);
}

mm_status mm_normalize_fixed(const mm_map *hc, const uint64_t *acc, float *out, void *stream) {
  const mm_map *h = hc;
  if (!h || !acc || !out) return fail(MM_EINVAL, "NULL argument");
  CK(cudaSetDevice(h->device));
  CK(launch_scale_fixed(reinterpret_cast<const unsigned long long *>(acc),
                        (int64_t)h->P.npix * h->P.npix_y, map_scale(h), out,
                        (cudaStream_t)stream));
  return MM_OK;
}

mm_status mm_run_batch(mm_map *const *hs, int32_t n, void *stream) {
  if (!hs || n <= 0) return fail(MM_EINVAL, "empty batch");
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < n; i++) {
    if (!hs[i]) return fail(MM_EINVAL, "handle %d is NULL", i);
    if (hs[i]->mode != MM_FMM_FP32) return fail(MM_EINVAL, "batch needs MM_FMM_FP32 handles");
    if (hs[i]->device != hs[0]->device) return fail(MM_EINVAL, "batch spans devices");
    if (hs[i]->timed_out) return fail(MM_ESTATE, "handle %d timed out earlier", i);
  }
  CK(cudaSetDevice(hs[0]->device));
  mm_map *lead = hs[0];
  // the lead's fan-out streams (created by its first batch call)
  const int nfan = std::min<int>(n, MM_BATCH_STREAMS);
  while ((int)lead->fan.size() < nfan) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t e2 = nullptr;
    CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    lead->fan.push_back(s2);
    CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    lead->fan_join.push_back(e2);
  }
  for (auto &e : lead->fan_fork)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // fork: the fan streams start after the work the caller queued before
  CK(cudaEventRecord(lead->fan_fork[0], st));
  for (int k = 0; k < nfan; k++) CK(cudaStreamWaitEvent(lead->fan[k], lead->fan_fork[0], 0));
  std::vector<const MapDev *> src(n);
  std::vector<int64_t> wb(n);
  int64_t work = 0;
  bool all_square = true;
  for (int i = 0; i < n; i++) {
    mm_map *h = hs[i];
    cudaStream_t si = lead->fan[i % nfan];
    h->launches = 0;
    CKS(record(h, 0, si));
    CKS(clear_map(h, si));
    if (h->fresh) {
      h->fresh = false;
      CKS(record(h, 1, si));
    } else {
      CKS(prepare(h, si));
    }
    CKS(record(h, 2, si));
    src[i] = h->d_md.p;
    wb[i] = work;
    work += (int64_t)h->md.strips * h->md.row_blocks;
    all_square = all_square && h->md.square_cells;
  }
  // join: the shared launch waits for every map's tree and expansions
  for (int k = 0; k < nfan; k++) {
    CK(cudaEventRecord(lead->fan_join[k], lead->fan[k]));
    CK(cudaStreamWaitEvent(st, lead->fan_join[k], 0));
  }
  // the descriptor array is assembled on the device from the handles' own
  // copies: no host staging and no synchronisation, so the whole batch can
  // be captured in a CUDA graph (after one call has sized the array)
  CK(lead->batch_md.ensure(n));
  for (int i = 0; i < n; i++) hs[i]->led_batch = false;
  if (lead->opt.time_stages) {
    for (auto &e : lead->batch_ev)
      if (!e) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(lead->batch_ev[0], st));
  }
  int gl = 0;
  CK(launch_batch_gather(src.data(), wb.data(), n, lead->batch_md.p, gl, st));
  lead->launches += gl;
  CK(launch_shoot_ipm(lead->batch_md.p, nullptr, n, work, all_square, lead->counter.p, lead->err.p,
                      shoot_grid(), st));
  lead->launches++;
  if (lead->opt.time_stages) {
    CK(cudaEventRecord(lead->batch_ev[1], st));
    lead->led_batch = true;
  }
  // second passes and normalisation, fanned out again and joined back
  CK(cudaEventRecord(lead->fan_fork[1], st));
  for (int k = 0; k < nfan; k++) CK(cudaStreamWaitEvent(lead->fan[k], lead->fan_fork[1], 0));
  for (int i = 0; i < n; i++) {
    mm_map *h = hs[i];
    cudaStream_t si = lead->fan[i % nfan];
    h->last_segments = 0;  // one first pass for the whole batch
    CKS(record(h, 5, si));
    LCH(launch_big_ipm(h->md, si));
    CKS(record(h, 3, si));
    LCH(launch_normalize(h->acc.p, h->span.p, h->P.npix, h->P.npix_y, map_scale(h), h->map.p, si));
    CKS(record(h, 4, si));
    h->ev_recorded = h->opt.time_stages != 0;
    h->last_stream = st;
    h->ran = true;
  }
  for (int k = 0; k < nfan; k++) {
    CK(cudaEventRecord(lead->fan_join[k], lead->fan[k]));
    CK(cudaStreamWaitEvent(st, lead->fan_join[k], 0));
  }
  return MM_OK;
}

mm_status mm_get_map(const mm_map *hc, float *out, int32_t on_device) {
  mm_map *h = const_cast<mm_map *>(hc);
  if (!h || !out) return fail(MM_EINVAL, "NULL argument");
  if (!h->ran) return fail(MM_ESTATE, "mm_run has not been called");
  CK(cudaSetDevice(h->device));
  const size_t bytes = (size_t)h->P.npix * h->P.npix_y * sizeof(float);
  if (on_device) {
    CK(cudaMemcpyAsync(out, h->map.p, bytes, cudaMemcpyDeviceToDevice, h->last_stream));
  } else {
    CK(cudaMemcpyAsync(out, h->map.p, bytes, cudaMemcpyDeviceToHost, h->last_stream));
    CK(cudaStreamSynchronize(h->last_stream));
  }
  return MM_OK;
}

mm_status mm_get_map_fixed(const mm_map *hc, uint64_t *out, int32_t on_device) {
  mm_map *h = const_cast<mm_map *>(hc);
  if (!h || !out) return fail(MM_EINVAL, "NULL argument");
  if (!h->ran) return fail(MM_ESTATE, "mm_run has not been called");
  CK(cudaSetDevice(h->device));
  const size_t np = (size_t)h->P.npix * h->P.npix_y;
  CK(h->fixed_out.ensure(np));
  LCH(launch_fold_span(h->acc.p, h->span.p, h->P.npix, h->P.npix_y, h->fixed_out.p,
                       h->last_stream));
  if (on_device) {
    CK(cudaMemcpyAsync(out, h->fixed_out.p, np * 8, cudaMemcpyDeviceToDevice, h->last_stream));
  } else {
    CK(cudaMemcpyAsync(out, h->fixed_out.p, np * 8, cudaMemcpyDeviceToHost, h->last_stream));
    CK(cudaStreamSynchronize(h->last_stream));
  }
  return MM_OK;
}

mm_status mm_shoot_points(mm_map *h, int64_t n, const double *z_xy, double *w_xy) {
  if (!h) return fail(MM_EINVAL, "handle is NULL");
  if (n < 0 || (n > 0 && (!z_xy || !w_xy))) return fail(MM_EINVAL, "bad point arrays");
  if (n == 0) return MM_OK;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->plan_stream;
  CK(cudaStreamSynchronize(h->last_stream));
  double *dz = nullptr, *dw = nullptr;
  CK(cudaMalloc(&dz, 2 * n * sizeof(double)));
  cudaError_t e = cudaMalloc(&dw, 2 * n * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(dz);
    CK(e);
  }
  mm_status s = MM_OK;
  do {
    const mm_params &P = h->P;
    if (cudaMemcpyAsync(dz, z_xy, 2 * n * sizeof(double), cudaMemcpyHostToDevice, st)) {
      s = fail(MM_ECUDA, "copy of probe points failed");
      break;
    }
    if (h->mode == MM_PLAIN_FP64) {
      DirectConst C;
      C.kappa = P.kappa;
      C.gamma = P.gamma;
      C.kappa_star = P.kappa_star;
      C.x0 = P.x0[0];
      C.y0 = P.x0[1];
      C.hx = P.h[0];
      C.hy = P.h[1];
      C.lox = P.center_y[0] - P.half_length;
      C.loy = P.center_y[1] - P.half_length_y;
      C.delta = P.delta;
      C.rect_c1 = h->opt.star_rect[0];
      C.rect_c2 = h->opt.star_rect[1];
      e = launch_direct64_points(h->sx.p, h->sy.p, h->sm.p, h->N, C, n, dz, dw, st);
    } else {
      if (!h->prepared) {
        s = prepare(h, st);
        if (s != MM_OK) break;
      }
      e = launch_probe(h->d_md.p, h->md.square_cells != 0, n, dz, dw, P.x0[0], P.x0[1], P.h[0],
                       P.h[1], h->R0, P.center_y[0] - P.half_length,
                       P.center_y[1] - P.half_length_y, P.delta, h->err.p, st);
    }
    if (e != cudaSuccess) {
      s = fail(MM_ECUDA, "probe launch: %s", cudaGetErrorString(e));
      break;
    }
    e = cudaMemcpyAsync(w_xy, dw, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = fail(MM_ECUDA, "probe: %s", cudaGetErrorString(e));
  } while (0);
  cudaFree(dz);
  cudaFree(dw);
  return s;
}

mm_status mm_get_stats(const mm_map *hc, mm_stats *out) {
  mm_map *h = const_cast<mm_map *>(hc);
  if (!h || !out) return fail(MM_EINVAL, "NULL argument");
  CK(cudaSetDevice(h->device));
  memset(out, 0, sizeof *out);
  out->params = h->P;
  out->mode = h->mode;
  out->fmm_order = h->mode != MM_PLAIN_FP64 ? h->p : 0;
  out->eval_order = h->mode != MM_PLAIN_FP64 ? h->p_eval : 0;
  out->sub_levels = h->mode != MM_PLAIN_FP64 ? h->sub : 0;
  out->leaf_size = h->leaf_size;
  out->depth = h->depth;
  out->n_stars = h->N;
  out->nodes = h->n_nodes;
  out->active_leaves = h->n_active;
  out->root_half_length = h->R0;
  out->min_leaf_half_length = h->min_leaf_L;
  out->rays = (h->col_hi - h->col_lo + 1) * (h->row_hi - h->row_lo + 1);
  out->cells = (h->col_hi - h->col_lo) * (h->row_hi - h->row_lo);
  out->ms_tree = out->ms_expansions = out->ms_shoot = out->ms_normalize = out->ms_total = -1.0;
  out->ms_first_pass = out->ms_second_pass = -1.0;
  out->queue_slots = (int32_t)std::min<int64_t>(h->bigq_cap, INT32_MAX);
  if (h->last_stream || h->ran) CK(cudaStreamSynchronize(h->last_stream));
  if (h->err.p)
    CK(cudaMemcpy(&out->error_bits, h->err.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (h->mode != MM_PLAIN_FP64 && h->n_nodes > 0) {
    std::vector<int32_t> fc(h->n_nodes);
    CK(cudaMemcpy(fc.data(), h->first_child.p, h->n_nodes * sizeof(int32_t),
                  cudaMemcpyDeviceToHost));
    int64_t leaves = 0;
    for (int32_t c : fc) leaves += (c < 0);
    out->leaves = leaves;
    // vertex-weighted mean near-field size over active leaves
    std::vector<LeafRec> lr(h->n_active << (2 * h->sub));
    CK(cudaMemcpy(lr.data(), h->leaf.p, lr.size() * sizeof(LeafRec), cudaMemcpyDeviceToHost));
    double sw = 0.0, swn = 0.0;
    std::vector<int32_t> lv(h->n_nodes);
    CK(cudaMemcpy(lv.data(), h->lvl.p, h->n_nodes * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (const LeafRec &r : lr) {
      const double side = 2.0 * h->R0 / (double)(1ll << lv[r.node]);
      const double w = side * side;  // vertices per leaf scale with its area
      sw += w;
      swn += w * r.near_cnt;
    }
    out->mean_near_stars = sw > 0 ? swn / sw : 0.0;
  }
  if (h->ran) {
    unsigned long long st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpy(st, h->stat.p, sizeof st, cudaMemcpyDeviceToHost));
    out->triangles_dropped = (int64_t)st[0];
    out->triangles_clipped = (int64_t)st[1];
    out->triangles_quad = (int64_t)st[2];
    out->triangles_box = (int64_t)st[3];
    out->triangles_rows = (int64_t)st[4];
    out->triangles_line = (int64_t)st[5];
    out->rows_culled = (int64_t)st[6];
    out->triangles_near_critical = (int64_t)st[7];
  }
  out->kernel_launches = h->launches;
  out->rows_per_item = h->rows_per_item;
  out->autotuned = h->tuned;
  out->ms_autotune = h->ms_tune;
  if (h->ev_recorded) {
    float a = 0, b = 0, c = 0, d = 0;
    CK(cudaEventElapsedTime(&a, h->ev[0], h->ev[4]));
    out->ms_total = a;
    if (h->mode != MM_PLAIN_FP64) {
      CK(cudaEventElapsedTime(&b, h->ev[0], h->ev[1]));
      CK(cudaEventElapsedTime(&c, h->ev[1], h->ev[2]));
      out->ms_tree = b;
      out->ms_expansions = c;
    }
    CK(cudaEventElapsedTime(&d, h->ev[2], h->ev[3]));
    out->ms_shoot = d;
    if (h->mode == MM_FMM_FP32 && h->last_segments > 0) {
      double f = 0.0, g = 0.0;
      for (int64_t k = 0; k < h->last_segments; k++) {
        CK(cudaEventElapsedTime(&d, k ? h->seg_ev[2 * k - 1] : h->ev[2], h->seg_ev[2 * k]));
        f += d;
        CK(cudaEventElapsedTime(&d, h->seg_ev[2 * k], h->seg_ev[2 * k + 1]));
        g += d;
      }
      out->ms_first_pass = f;
      out->ms_second_pass = g;
    } else if (h->led_batch) {
      // the lead of a batch: the batch's one shared first-pass launch
      CK(cudaEventElapsedTime(&d, h->batch_ev[0], h->batch_ev[1]));
      out->ms_first_pass = d;
      CK(cudaEventElapsedTime(&d, h->ev[5], h->ev[3]));
      out->ms_second_pass = d;
    } else {
      CK(cudaEventElapsedTime(&d, h->ev[2], h->ev[5]));
      out->ms_first_pass = d;
      CK(cudaEventElapsedTime(&d, h->ev[5], h->ev[3]));
      out->ms_second_pass = d;
    }
    CK(cudaEventElapsedTime(&a, h->ev[3], h->ev[4]));
    out->ms_normalize = a;
  }
  return MM_OK;
}

void mm_destroy(mm_map *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->last_stream) cudaStreamSynchronize(h->last_stream);
  // frees in stream order on the plan stream (synchronised below)
  AllocStream free_on(h->plan_stream);
  DBuf<double> *dbs[] = {&h->pos_in, &h->m_in, &h->sx, &h->sy, &h->sm};
  for (auto *b : dbs) b->release();
  h->keys_in.release();
  h->keys.release();
  h->bigq.release();
  h->bigq_n.release();
  h->idx_in.release();
  h->idx.release();
  h->cub_tmp.release();
  h->d_level_off.release();
  h->code.release();
  DBuf<int32_t> *ibs[] = {&h->lvl,       &h->sbeg,      &h->send,      &h->first_child,
                          &h->split,     &h->scan,      &h->col_cell,  &h->row_cell,
                          &h->node_act,  &h->leaf_flag, &h->leaf_scan, &h->node_active,
                          &h->active_list, &h->near_cnt, &h->near_off, &h->grid};
  for (auto *b : ibs) b->release();
  DBuf<double2> *cbs[] = {&h->MMop, &h->MLop, &h->LLop, &h->mp, &h->loc};
  for (auto *b : cbs) b->release();
  h->leaf.release();
  h->near_pos.release();
  h->near_m.release();
  h->coef.release();
  h->acc.release();
  h->span.release();
  h->stat.release();
  h->counter.release();
  h->fixed_out.release();
  h->err.release();
  h->map.release();
  h->d_md.release();
  h->verts.release();
  h->batch_md.release();
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : h->seg_ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : h->batch_ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t f : h->fan) {
    cudaStreamSynchronize(f);
    cudaStreamDestroy(f);
  }
  for (cudaEvent_t e : h->fan_join) cudaEventDestroy(e);
  for (auto &e : h->fan_fork)
    if (e) cudaEventDestroy(e);
  if (h->plan_stream) {
    cudaStreamSynchronize(h->plan_stream);
    cudaStreamDestroy(h->plan_stream);
  }
  if (h->pin) cudaFreeHost(h->pin);
  delete h;
}

}  // extern "C"
