// mm_map_plain_fp64_noalloc: the plain FP64 map (direct-sum deflection, then
// inverse polygon mapping) for callers that cannot allocate device memory.
//
// All scratch lives in one file-scope device array, g_scratch, of fixed size:
// star copies, the mapped vertices, the fixed-point accumulator, the row
// difference array, counters and the map descriptor.  Every GPU that loads
// this library holds that array until the process exits.  Host code must not
// use g_scratch's name as a device address (on the host it is only a
// stand-in): its device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, and cached for the life of the
// process (a cudaDeviceReset on that device invalidates it).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "mm.h"
#include "mm_kernels.h"

using namespace mm;

namespace {

constexpr int64_t kMaxStars = 16384;
constexpr int64_t kMaxVertices = 1 << 19;
constexpr int32_t kMaxPix = 256;

// byte offsets inside g_scratch (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffSx = 0;
constexpr size_t kOffSy = align256(kOffSx + kMaxStars * sizeof(double));
constexpr size_t kOffSm = align256(kOffSy + kMaxStars * sizeof(double));
constexpr size_t kOffVerts = align256(kOffSm + kMaxStars * sizeof(double));
constexpr size_t kOffAcc = align256(kOffVerts + kMaxVertices * sizeof(Vtx));
constexpr size_t kOffSpan = align256(kOffAcc + (size_t)kMaxPix * kMaxPix * 8);
constexpr size_t kOffStat = align256(kOffSpan + (size_t)kMaxPix * (kMaxPix + 1) * 8);
constexpr size_t kOffCounter = align256(kOffStat + 8 * 8);
constexpr size_t kOffErr = align256(kOffCounter + 8);
constexpr size_t kOffMapDev = align256(kOffErr + 8);
constexpr size_t kScratchBytes = align256(kOffMapDev + sizeof(MapDev));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// device address of g_scratch per device ordinal (looked up once)
constexpr int kMaxDevices = 64;
unsigned char *g_addr[kMaxDevices] = {nullptr};
std::mutex g_mutex;

mm_status fail(mm_status s, const char *msg, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess)
    snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(buf, sizeof buf, "%s", msg);
  mm::set_last_error(buf);
  return s;
}

__global__ void k_split_stars(const double *__restrict__ pos, const double *__restrict__ m,
                              int64_t n, double *sx, double *sy, double *sm) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  sx[t] = pos[2 * t];
  sy[t] = pos[2 * t + 1];
  sm[t] = m[t];
}

__global__ void k_write_mapdev(MapDev md, MapDev *out) { *out = md; }

// Whether p is device (or managed) memory that device `dev` can address as
// its own; a host pointer or another device's buffer would fault in a kernel.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the (non-sticky) error an unknown pointer leaves
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" mm_status mm_map_plain_fp64_noalloc(
    double kappa_tot, double shear, double smooth_fraction, int64_t n_stars,
    const double *masses, const double *pos_xy, double half_length, int32_t npix,
    const double *center_y, const int64_t *ray_grid, const double *grid_origin,
    const double *grid_spacing, float *map_out, void *stream) {
  if (n_stars < 0 || n_stars > kMaxStars)
    return fail(MM_EINVAL, "n_stars outside [0, 16384], the no-allocation limit");
  if (n_stars > 0 && (!masses || !pos_xy)) return fail(MM_EINVAL, "star arrays are NULL");
  if (npix < 1 || npix > kMaxPix)
    return fail(MM_EINVAL, "npix outside [1, 256], the no-allocation limit");
  if (!ray_grid || !grid_origin || !grid_spacing || !map_out)
    return fail(MM_EINVAL, "NULL grid or output argument");
  if (ray_grid[0] < 2 || ray_grid[1] < 2 || ray_grid[0] > kMaxVertices ||
      ray_grid[1] > kMaxVertices || ray_grid[0] * ray_grid[1] > kMaxVertices)
    return fail(MM_EINVAL, "ray grid needs 2..N rays per axis and at most 2^19 rays in all, "
                           "the no-allocation limit");
  if (!(half_length > 0.0) || !(grid_spacing[0] > 0.0) || !(grid_spacing[1] > 0.0))
    return fail(MM_EINVAL, "half_length and ray spacings must be > 0");
  if (!(smooth_fraction >= 0.0 && smooth_fraction <= 1.0))
    return fail(MM_EINVAL, "smooth_fraction outside [0, 1]");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MM_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return fail(MM_ECUDA, "device ordinal out of range");
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return fail(MM_ECUDA, "cudaGetSymbolAddress(g_scratch)", e);
      g_addr[dev] = static_cast<unsigned char *>(p);
    }
    base = g_addr[dev];
  }
  // every pointer the kernels touch must be this device's memory: reject
  // anything else before any work is enqueued
  if (n_stars > 0 && (!on_device(masses, dev) || !on_device(pos_xy, dev)))
    return fail(MM_EINVAL, "masses and pos_xy must be device memory of the current device");
  if (!on_device(map_out, dev))
    return fail(MM_EINVAL, "map_out must be device memory of the current device");
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail(MM_ECUDA, "cudaDeviceGetAttribute(multiprocessor count)", e);
  sms = sms > 0 ? sms : 1;
  double *sx = reinterpret_cast<double *>(base + kOffSx);
  double *sy = reinterpret_cast<double *>(base + kOffSy);
  double *sm = reinterpret_cast<double *>(base + kOffSm);
  Vtx *verts = reinterpret_cast<Vtx *>(base + kOffVerts);
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(base + kOffAcc);
  unsigned long long *span = reinterpret_cast<unsigned long long *>(base + kOffSpan);
  unsigned long long *stat = reinterpret_cast<unsigned long long *>(base + kOffStat);
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(base + kOffCounter);
  unsigned *err = reinterpret_cast<unsigned *>(base + kOffErr);
  MapDev *d_md = reinterpret_cast<MapDev *>(base + kOffMapDev);
  cudaStream_t st = (cudaStream_t)stream;

  const int64_t n0 = ray_grid[0], n1 = ray_grid[1];
  const double cx = center_y ? center_y[0] : 0.0, cy = center_y ? center_y[1] : 0.0;
  const double delta = 2.0 * half_length / (double)npix;
  DirectConst C;
  C.kappa = kappa_tot;
  C.gamma = shear;
  C.kappa_star = (1.0 - smooth_fraction) * kappa_tot;
  C.x0 = grid_origin[0];
  C.y0 = grid_origin[1];
  C.hx = grid_spacing[0];
  C.hy = grid_spacing[1];
  C.lox = cx - half_length;
  C.loy = cy - half_length;
  C.delta = delta;
  C.rect_c1 = C.rect_c2 = 0.0;  // star disk

  MapDev md;
  memset(&md, 0, sizeof md);
  md.n0 = n0;
  md.n1 = n1;
  md.row_begin = 0;
  md.row_end = n1 - 1;
  md.col_begin = 0;
  md.col_end = n0 - 1;
  md.rows_per_item = 64;
  md.npix = npix;
  md.npix_y = npix;  // square map
  md.err = err;
  md.acc = acc;
  md.span = span;
  md.stat = stat;

  // everything the kernels accumulate into starts at zero on every call
  const size_t np = (size_t)npix * npix;
  if ((e = cudaMemsetAsync(acc, 0, np * 8, st)) != cudaSuccess)
    return fail(MM_ECUDA, "clearing the accumulator", e);
  if ((e = cudaMemsetAsync(span, 0, (size_t)npix * (npix + 1) * 8, st)) != cudaSuccess)
    return fail(MM_ECUDA, "clearing the row difference array", e);
  if ((e = cudaMemsetAsync(stat, 0, 8 * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(counter, 0, 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(err, 0, 4, st)) != cudaSuccess)
    return fail(MM_ECUDA, "clearing counters", e);
  if (n_stars > 0) {
    k_split_stars<<<(unsigned)((n_stars + 255) / 256), 256, 0, st>>>(pos_xy, masses, n_stars, sx,
                                                                     sy, sm);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(MM_ECUDA, "star copy", e);
  }
  k_write_mapdev<<<1, 1, 0, st>>>(md, d_md);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(MM_ECUDA, "map descriptor", e);
  if ((e = launch_direct64_vertices(sx, sy, sm, n_stars, C, 0, n0, 0, n1 - 1, verts, st)) !=
      cudaSuccess)
    return fail(MM_ECUDA, "direct-sum deflection", e);
  if ((e = launch_ipm_vertices(d_md, verts, n0, 0, n1 - 1, counter, err, 2 * sms, st)) !=
      cudaSuccess)
    return fail(MM_ECUDA, "inverse polygon mapping", e);
  const double scale = std::ldexp(0.5 * C.hx * C.hy / (delta * delta), -32);
  if ((e = launch_normalize(acc, span, npix, npix, scale, map_out, st)) != cudaSuccess)
    return fail(MM_ECUDA, "normalisation", e);
  // the kernels' error word (an index check of the MM_DEBUG build): the copy
  // to pageable host memory returns once the stream has reached it
  unsigned err_word = 0;
  if ((e = cudaMemcpyAsync(&err_word, err, sizeof err_word, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(MM_ECUDA, "reading the error word", e);
  if (err_word != 0) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "the map kernels reported error bits 0x%x (8: a map index out of range, access "
             "skipped); map_out is not valid",
             err_word);
    return fail(MM_ECUDA, msg);
  }
  return MM_OK;
}
