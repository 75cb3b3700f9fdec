"""GB300-native magnification maps for gravitational microlensing.

Thin ctypes binding over ``libmm.so`` (declared in ``include/mm.h``): the
functions below only marshal arguments; every step of the path runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or no CUDA device is present, the calls raise.

Typical use::

    import paper_2506_02114_gb300 as mm
    h = mm.create(kappa, gamma, s, masses, pos, half_length, npix,
                  rays_per_pixel=9.0, fmm_order=25)
    mm.run(h)                  # on torch's current CUDA stream
    mu = mm.get_map(h)         # numpy (npix_y, npix) float32, row = y
    mm.destroy(h)
"""
import ctypes
import os

import numpy as np

from . import build as _build

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ETIMEOUT, MM_ESTATE = range(6)
MM_FMM_FP32, MM_PLAIN_FP64, MM_FMM_IRS = 0, 1, 2
_STATUS = {0: "MM_OK", 1: "MM_EINVAL", 2: "MM_ENOMEM", 3: "MM_ECUDA", 4: "MM_ETIMEOUT",
           5: "MM_ESTATE"}


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("time_stages", ctypes.c_int32),
                ("img_half", ctypes.c_double * 2), ("ray_grid", ctypes.c_int64 * 2),
                ("flux_fraction_f", ctypes.c_double), ("center_y", ctypes.c_double * 2),
                ("row_begin", ctypes.c_int64), ("row_end", ctypes.c_int64),
                ("rows_per_item", ctypes.c_int32), ("sub_levels", ctypes.c_int32),
                ("col_begin", ctypes.c_int64), ("col_end", ctypes.c_int64),
                ("no_cull", ctypes.c_int32), ("big_queue_slots", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p), ("critical_mu", ctypes.c_double),
                ("star_rect", ctypes.c_double * 2), ("npix_y", ctypes.c_int32),
                ("reserved1", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("gamma", ctypes.c_double),
                ("smooth_fraction", ctypes.c_double), ("kappa_star", ctypes.c_double),
                ("a1", ctypes.c_double), ("a2", ctypes.c_double),
                ("mu_macro", ctypes.c_double), ("mean_m", ctypes.c_double),
                ("m2_over_m", ctypes.c_double), ("flux_fraction_f", ctypes.c_double),
                ("r_border", ctypes.c_double), ("half_length", ctypes.c_double),
                ("npix", ctypes.c_int32), ("npix_y", ctypes.c_int32),
                ("delta", ctypes.c_double), ("center_y", ctypes.c_double * 2),
                ("img_center", ctypes.c_double * 2), ("img_half", ctypes.c_double * 2),
                ("n", ctypes.c_int64 * 2), ("h", ctypes.c_double * 2),
                ("x0", ctypes.c_double * 2), ("half_length_y", ctypes.c_double)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if hasattr(getattr(self, k), "__len__")
                    else getattr(self, k)) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("params", Params), ("mode", ctypes.c_int32), ("fmm_order", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("eval_order", ctypes.c_int32), ("sub_levels", ctypes.c_int32),
                ("n_stars", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("leaves", ctypes.c_int64), ("active_leaves", ctypes.c_int64),
                ("root_half_length", ctypes.c_double),
                ("min_leaf_half_length", ctypes.c_double),
                ("mean_near_stars", ctypes.c_double), ("rays", ctypes.c_int64),
                ("cells", ctypes.c_int64), ("triangles_dropped", ctypes.c_int64),
                ("triangles_clipped", ctypes.c_int64), ("triangles_line", ctypes.c_int64),
                ("triangles_quad", ctypes.c_int64),
                ("triangles_box", ctypes.c_int64), ("triangles_rows", ctypes.c_int64),
                ("rows_culled", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms_tree", ctypes.c_double),
                ("ms_expansions", ctypes.c_double), ("ms_shoot", ctypes.c_double),
                ("ms_normalize", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_first_pass", ctypes.c_double), ("ms_second_pass", ctypes.c_double),
                ("rows_per_item", ctypes.c_int32), ("autotuned", ctypes.c_int32),
                ("ms_autotune", ctypes.c_double), ("triangles_near_critical", ctypes.c_int64),
                ("error_bits", ctypes.c_uint32), ("queue_slots", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "params"}
        d["params"] = self.params.as_dict()
        return d


EXPORTS = ["mm_derive_params", "mm_create", "mm_run", "mm_run_cells", "mm_run_batch",
           "mm_get_map", "mm_get_map_fixed", "mm_normalize_fixed", "mm_shoot_points",
           "mm_get_stats", "mm_map_plain_fp64_noalloc", "mm_measure_peak", "mm_last_error",
           "mm_destroy"]

MM_PEAK_FP32_FMA, MM_PEAK_FP64_FMA, MM_PEAK_L2_RED_U64, MM_PEAK_L2_RED_U64_ROWS = 0, 1, 2, 3

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libmm.so (building it when absent or stale); raises if it cannot.
    With MM_DEBUG_BUILD=1 in the environment, the MM_DEBUG variant is used
    (bounds-checked map atomics; violations reported in
    mm_get_stats().error_bits)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("MM_DEBUG_BUILD") == "1"
    if build_if_missing:
        path = _build.build(debug=debug)
    else:
        path = _build.LIB_DEBUG if debug else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libmm.so is missing: run paper_2506_02114_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.mm_derive_params.restype = ctypes.c_int
    L.mm_derive_params.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int64, _dp, ctypes.c_double, ctypes.c_int32,
                                   ctypes.c_double, ctypes.POINTER(Options),
                                   ctypes.POINTER(Params)]
    L.mm_create.restype = ctypes.c_int
    L.mm_create.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                            _dp, _dp, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Options),
                            ctypes.POINTER(_vp)]
    L.mm_run.restype = ctypes.c_int
    L.mm_run.argtypes = [_vp, _vp]
    L.mm_run_cells.restype = ctypes.c_int
    L.mm_run_cells.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, _vp]
    L.mm_normalize_fixed.restype = ctypes.c_int
    L.mm_normalize_fixed.argtypes = [_vp, _vp, _vp, _vp]
    L.mm_measure_peak.restype = ctypes.c_int
    L.mm_measure_peak.argtypes = [ctypes.c_int32, _dp, _dp, _vp]
    L.mm_run_batch.restype = ctypes.c_int
    L.mm_run_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, _vp]
    L.mm_get_map.restype = ctypes.c_int
    L.mm_get_map.argtypes = [_vp, _vp, ctypes.c_int32]
    L.mm_get_map_fixed.restype = ctypes.c_int
    L.mm_get_map_fixed.argtypes = [_vp, _vp, ctypes.c_int32]
    L.mm_shoot_points.restype = ctypes.c_int
    L.mm_shoot_points.argtypes = [_vp, ctypes.c_int64, _dp, _dp]
    L.mm_get_stats.restype = ctypes.c_int
    L.mm_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
    L.mm_map_plain_fp64_noalloc.restype = ctypes.c_int
    L.mm_map_plain_fp64_noalloc.argtypes = [
        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64, _vp, _vp,
        ctypes.c_double, ctypes.c_int32, _dp, ctypes.POINTER(ctypes.c_int64), _dp, _dp, _vp, _vp]
    L.mm_last_error.restype = ctypes.c_char_p
    L.mm_last_error.argtypes = []
    L.mm_destroy.restype = None
    L.mm_destroy.argtypes = [_vp]
    _lib = L
    return L


def last_error():
    return lib().mm_last_error().decode()


def _check(status):
    if status != MM_OK:
        raise MMError(status, last_error())


def _f64(a):
    if a is None:
        return None
    if hasattr(a, "detach"):  # torch tensor
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None and a.size else None


def make_options(mode=MM_FMM_FP32, time_stages=False, img_half=None, ray_grid=None,
                 flux_fraction_f=0.0, center_y=(0.0, 0.0), row_begin=0, row_end=0,
                 rows_per_item=0, col_begin=0, col_end=0, sub_levels=0, cull=True,
                 big_queue_slots=0, autotune=False, tune_cache=None, critical_mu=0.0,
                 star_rect=None, npix_y=0):
    o = Options()
    o.mode = int(mode)
    o.time_stages = 1 if time_stages else 0
    if img_half is not None:
        o.img_half[0], o.img_half[1] = float(img_half[0]), float(img_half[1])
    if ray_grid is not None:
        o.ray_grid[0], o.ray_grid[1] = int(ray_grid[0]), int(ray_grid[1])
    o.flux_fraction_f = float(flux_fraction_f)
    o.center_y[0], o.center_y[1] = float(center_y[0]), float(center_y[1])
    o.row_begin, o.row_end = int(row_begin), int(row_end)
    o.rows_per_item = int(rows_per_item)
    o.sub_levels = int(sub_levels)
    o.no_cull = 0 if cull else 1
    o.big_queue_slots = int(big_queue_slots)
    o.col_begin, o.col_end = int(col_begin), int(col_end)
    o.autotune = 1 if autotune else 0
    o.critical_mu = float(critical_mu)
    if star_rect is not None:
        o.star_rect[0], o.star_rect[1] = float(star_rect[0]), float(star_rect[1])
    o.npix_y = int(npix_y)
    # (the structure keeps the encoded path alive while it lives)
    o.tune_cache = os.fsencode(tune_cache) if tune_cache is not None else None
    return o


def derive_params(kappa, gamma, s, masses, half_length, npix, rays_per_pixel=0.0,
                  **opts) -> Params:
    """Derived scalars of a run (host only; no GPU needed)."""
    m = _f64(masses)
    p = Params()
    o = make_options(**opts)
    _check(lib().mm_derive_params(float(kappa), float(gamma), float(s), m.size, _ptr(m),
                                  float(half_length), int(npix), float(rays_per_pixel),
                                  ctypes.byref(o), ctypes.byref(p)))
    return p


class Handle:
    """Owns an mm_map*; destroyed explicitly or when garbage collected."""

    def __init__(self, ptr, npix, npix_y=None):
        self.ptr = ptr
        self.npix = npix
        self.npix_y = npix_y or npix

    def __del__(self):
        try:
            destroy(self)
        except Exception:
            pass


def create(kappa, gamma, s, masses, pos_xy, half_length, npix, rays_per_pixel=0.0,
           fmm_order=0, leaf_size=0, **opts) -> Handle:
    m = _f64(masses)
    pos = _f64(pos_xy)
    if pos is not None:
        pos = pos.reshape(-1)
    o = make_options(**opts)
    out = _vp()
    _check(lib().mm_create(float(kappa), float(gamma), float(s), m.size, _ptr(m), _ptr(pos),
                           float(half_length), int(npix), float(rays_per_pixel),
                           int(fmm_order), int(leaf_size), ctypes.byref(o), ctypes.byref(out)))
    return Handle(out, int(npix), int(o.npix_y) or int(npix))


def current_stream():
    """torch's current CUDA stream handle (0 = legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def run(h: Handle, stream=None):
    _check(lib().mm_run(h.ptr, _vp(current_stream() if stream is None else stream)))


def run_cells(h: Handle, row_begin, row_end, col_begin, col_end, stream=None):
    """Run the map over cell rows [row_begin, row_end) and columns
    [col_begin, col_end) only, with the handle's whole plan (mm_run_cells)."""
    _check(lib().mm_run_cells(h.ptr, int(row_begin), int(row_end), int(col_begin),
                              int(col_end), _vp(current_stream() if stream is None else stream)))


def run_batch(hs, stream=None):
    arr = (_vp * len(hs))(*[x.ptr for x in hs])
    _check(lib().mm_run_batch(arr, len(hs),
                              _vp(current_stream() if stream is None else stream)))


def get_map(h: Handle, out=None):
    """Magnification map.  out=None: new numpy (npix_y, npix) float32 array.
    out may be a torch CUDA float32 tensor with npix_y*npix elements."""
    n = h.npix_y * h.npix
    if out is not None and hasattr(out, "is_cuda"):
        if not out.is_cuda:
            out_np = out.numpy()          # a CPU tensor shares its storage
            _check_out(out_np, n)
            _check(lib().mm_get_map(h.ptr, out_np.ctypes.data_as(_vp), 0))
            return out
        if str(out.dtype) != "torch.float32" or out.numel() != n or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 tensor of %d elements" % n)
        _check(lib().mm_get_map(h.ptr, _vp(out.data_ptr()), 1))
        return out
    a = np.empty((h.npix_y, h.npix), dtype=np.float32) if out is None else out
    _check_out(a, n)
    _check(lib().mm_get_map(h.ptr, a.ctypes.data_as(_vp), 0))
    return a


def _check_out(a, n):
    if (not isinstance(a, np.ndarray) or a.dtype != np.float32 or a.size != n
            or not a.flags.c_contiguous or not a.flags.writeable):
        raise ValueError("out must be a writeable C-contiguous float32 array of %d elements" % n)


def get_map_fixed(h: Handle, out=None):
    """Raw fixed-point accumulator (npix_y, npix) uint64: sum of round(frac*2^32).
    out may be a contiguous CUDA int64 tensor of npix_y*npix elements (the
    same 64 bits; enqueued on the handle's last stream)."""
    n = h.npix_y * h.npix
    if out is not None:
        _check_dev(out, "torch.int64", n, "out")
        _check(lib().mm_get_map_fixed(h.ptr, _vp(out.data_ptr()), 1))
        return out
    a = np.empty((h.npix_y, h.npix), dtype=np.uint64)
    _check(lib().mm_get_map_fixed(h.ptr, a.ctypes.data_as(_vp), 0))
    return a


def normalize_fixed(h: Handle, acc, out, stream=None):
    """Magnification from a fixed-point accumulator (mm_normalize_fixed):
    acc a contiguous CUDA int64 tensor of npix_y*npix elements (the u64 bits,
    e.g. the sum of several bands' maps), out a CUDA float32 tensor of as many.
    Enqueued on `stream` (torch's current stream by default)."""
    n = h.npix_y * h.npix
    _check_dev(acc, "torch.int64", n, "acc")
    _check_dev(out, "torch.float32", n, "out")
    _check(lib().mm_normalize_fixed(h.ptr, _vp(acc.data_ptr()), _vp(out.data_ptr()),
                                    _vp(current_stream() if stream is None else stream)))
    return out


def measure_peak(kind, stream=None):
    """(value, ms) of one of the MM_PEAK_* microbenchmarks on the current
    device: TFLOP/s for the FMA kinds, 1e9 u64 reductions/s for the L2 kind."""
    v, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().mm_measure_peak(int(kind), ctypes.byref(v), ctypes.byref(ms),
                                 _vp(current_stream() if stream is None else stream)))
    return v.value, ms.value


def shoot_points(h: Handle, z_xy):
    """Source positions w (n, 2) of image-plane points z (n, 2), FP64 out."""
    z = _f64(z_xy).reshape(-1, 2)
    w = np.empty_like(z)
    _check(lib().mm_shoot_points(h.ptr, z.shape[0], _ptr(z), w.ctypes.data_as(_dp)))
    return w


def map_plain_fp64_noalloc(kappa, gamma, s, masses_dev, pos_dev, half_length, npix, ray_grid,
                           grid_origin, grid_spacing, map_out_dev, center_y=(0.0, 0.0),
                           stream=None):
    """Plain FP64 map with no device allocation (see mm.h): masses_dev,
    pos_dev ((n, 2) or (2n,)) and map_out_dev (npix*npix float32) are CUDA
    tensors; the grid arguments are host sequences.  Asynchronous."""
    n = int(masses_dev.numel())
    _check_dev(masses_dev, "torch.float64", n, "masses_dev")
    _check_dev(pos_dev, "torch.float64", 2 * n, "pos_dev")
    _check_dev(map_out_dev, "torch.float32", int(npix) * int(npix), "map_out_dev", at_least=True)
    rg = (ctypes.c_int64 * 2)(int(ray_grid[0]), int(ray_grid[1]))
    org = (ctypes.c_double * 2)(float(grid_origin[0]), float(grid_origin[1]))
    hh = (ctypes.c_double * 2)(float(grid_spacing[0]), float(grid_spacing[1]))
    cy = (ctypes.c_double * 2)(float(center_y[0]), float(center_y[1]))
    _check(lib().mm_map_plain_fp64_noalloc(
        float(kappa), float(gamma), float(s), n, _vp(masses_dev.data_ptr() if n else 0),
        _vp(pos_dev.data_ptr() if n else 0), float(half_length), int(npix),
        ctypes.cast(cy, _dp), rg, ctypes.cast(org, _dp), ctypes.cast(hh, _dp),
        _vp(map_out_dev.data_ptr()), _vp(current_stream() if stream is None else stream)))
    return map_out_dev


def _check_dev(t, dtype, numel, name, at_least=False):
    size_ok = int(t.numel()) >= numel if at_least else int(t.numel()) == numel
    if not getattr(t, "is_cuda", False) or str(t.dtype) != dtype or not size_ok \
            or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor of %s%d elements"
                         % (name, dtype[len("torch."):], "at least " if at_least else "", numel))
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on cuda:%s, not the current device cuda:%d"
                         % (name, t.device.index, torch.cuda.current_device()))


def shard_rows(n_rows, rank, world):
    """Cell rows [begin, end) of `rank` when one map's n_rows cell rows are
    split over `world` ranks in contiguous bands (the first n_rows % world
    bands one row longer).  Each rank maps its band (``row_begin/row_end``);
    the fixed-point maps of the bands add up exactly to the whole map."""
    if world < 1 or not 0 <= rank < world or n_rows < 0:
        raise ValueError("bad shard request")
    q, r = divmod(int(n_rows), int(world))
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def get_stats(h: Handle) -> dict:
    s = Stats()
    _check(lib().mm_get_stats(h.ptr, ctypes.byref(s)))
    return s.as_dict()


def destroy(h: Handle):
    if h is not None and h.ptr is not None and h.ptr.value:
        lib().mm_destroy(h.ptr)
        h.ptr = _vp()
