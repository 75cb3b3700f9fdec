"""Oracle: plain FP64 CPU reference for the magnification-map path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may
import this package.  It shares no code with ``paper_2506_02114_gb300`` and
never imports it.

The C library (``oracle.c``) computes, in FP64 and in the paper's notation:

* ``derive_params``  -- kappa_star (Sec. 2.1), mu_macro (Sec. 3.1), the border
  radius r of App. A and the shooting region of Sec. 2.3, and the ray grid
  (Sec. 3.2, Table 1 caption);
* ``deflect``        -- the complex lens equation of Sec. 2.2 with the circular
  smooth sheet of Sec. 3.1, by direct summation over every star;
* ``magnification_map`` -- inverse polygon mapping (Sec. 3.2): two triangles
  per cell, each pixel receiving area(T n pixel)/|area(T)| from per-pixel
  Sutherland-Hodgman clipping and the shoelace formula;
* ``irs_map`` -- inverse ray shooting (Sec. 3.2, Table 1's IRS column): each
  grid vertex is a ray counted in the pixel it lands in.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class Params(ctypes.Structure):
    _fields_ = [
        ("kappa", ctypes.c_double), ("gamma", ctypes.c_double),
        ("smooth_fraction", ctypes.c_double), ("kappa_star", ctypes.c_double),
        ("a1", ctypes.c_double), ("a2", ctypes.c_double),
        ("mu_macro", ctypes.c_double), ("mean_m", ctypes.c_double),
        ("m2_over_m", ctypes.c_double), ("flux_fraction_f", ctypes.c_double),
        ("r_border", ctypes.c_double), ("half_length", ctypes.c_double),
        ("npix", ctypes.c_int32), ("npix_y", ctypes.c_int32), ("delta", ctypes.c_double),
        ("center_y", ctypes.c_double * 2), ("img_center", ctypes.c_double * 2),
        ("img_half", ctypes.c_double * 2), ("n", ctypes.c_int64 * 2),
        ("h", ctypes.c_double * 2), ("x0", ctypes.c_double * 2),
        ("star_rect", ctypes.c_double * 2), ("half_length_y", ctypes.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class MapStats(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_int64), ("dropped", ctypes.c_int64),
                ("pieces", ctypes.c_int64)]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_derive_params.restype = ctypes.c_int
        L.or_derive_params.argtypes = [
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64, _dp,
            ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _dp,
            _dp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(Params)]
        L.or_alpha_rect.restype = None
        L.or_alpha_rect.argtypes = [ctypes.POINTER(Params), ctypes.c_double, ctypes.c_double,
                                    _dp, _dp]
        L.or_deflect.restype = None
        L.or_deflect.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _dp, _dp,
                                 ctypes.c_int64, _dp, _dp, ctypes.c_int]
        L.or_map.restype = ctypes.c_int
        L.or_map.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _dp, _dp,
                             ctypes.c_int64, ctypes.c_int64, _dp, _dp,
                             ctypes.POINTER(MapStats), ctypes.c_int]
        L.or_map_tile.restype = ctypes.c_int
        L.or_map_tile.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _dp, _dp,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  _dp, _dp, ctypes.POINTER(MapStats), ctypes.c_int]
        L.or_map_from_vertices.restype = ctypes.c_int
        L.or_map_from_vertices.argtypes = [ctypes.POINTER(Params), _dp, ctypes.c_int64,
                                           ctypes.c_int64, _dp, _dp,
                                           ctypes.POINTER(MapStats), ctypes.c_int]
        L.or_map_tile_from_vertices.restype = ctypes.c_int
        L.or_map_tile_from_vertices.argtypes = [ctypes.POINTER(Params), _dp, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                _dp, _dp, ctypes.POINTER(MapStats),
                                                ctypes.c_int]
        L.or_irs_tile.restype = ctypes.c_int
        L.or_irs_tile.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _dp, _dp,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64), _dp,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        L.or_tri_rect_area.restype = ctypes.c_double
        L.or_tri_rect_area.argtypes = [_dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None and a.size else None


def default_threads():
    return max(1, os.cpu_count() or 1)


def derive_params(kappa, gamma, smooth_fraction, masses, half_length, npix,
                  rays_per_pixel=0.0, flux_fraction_f=0.0, center_y=None,
                  img_half=None, ray_grid=None, star_rect=None, npix_y=0) -> Params:
    m = _f64(masses)
    p = Params()
    cy = _f64(center_y) if center_y is not None else None
    ih = _f64(img_half) if img_half is not None else None
    rg = (np.ascontiguousarray(np.asarray(ray_grid, dtype=np.int64))
          if ray_grid is not None else None)
    rc = lib().or_derive_params(
        float(kappa), float(gamma), float(smooth_fraction), m.size, _ptr(m),
        float(half_length), int(npix), int(npix_y), float(rays_per_pixel),
        float(flux_fraction_f),
        _ptr(cy), _ptr(ih),
        rg.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if rg is not None else None,
        ctypes.byref(p))
    if rc != 0:
        raise ValueError("oracle: invalid parameters")
    if star_rect is not None:
        p.star_rect[0], p.star_rect[1] = float(star_rect[0]), float(star_rect[1])
    return p


def alpha_rect(params: Params, x, y):
    """App. B's deflection of the rectangular sheet of params.star_rect at (x, y)."""
    ax, ay = ctypes.c_double(), ctypes.c_double()
    lib().or_alpha_rect(ctypes.byref(params), float(x), float(y), ctypes.byref(ax),
                        ctypes.byref(ay))
    return complex(ax.value, ay.value)


def deflect(params: Params, masses, pos_xy, z_xy, nthreads=None):
    """w (n, 2) at points z_xy (n, 2) by direct summation over all stars."""
    m = _f64(masses)
    xy = _f64(pos_xy).reshape(-1, 2)
    z = _f64(z_xy).reshape(-1, 2)
    w = np.empty_like(z)
    lib().or_deflect(ctypes.byref(params), m.size, _ptr(m), _ptr(xy), z.shape[0],
                     _ptr(z), w.ctypes.data_as(_dp), nthreads or default_threads())
    return w


def grid_vertices(params: Params, i, j):
    """FP64 image-plane positions of ray-grid vertices (i, j)."""
    i = np.asarray(i, dtype=np.float64)
    j = np.asarray(j, dtype=np.float64)
    return np.stack([params.x0[0] + i * params.h[0], params.x0[1] + j * params.h[1]], -1)


def magnification_map(params: Params, masses, pos_xy, row_begin=0, row_end=0,
                      nthreads=None, return_acc=False):
    """Magnification map (npix, npix) from the cell rows [row_begin, row_end)."""
    m = _f64(masses)
    xy = _f64(pos_xy).reshape(-1, 2)
    n, ny = params.npix, params.npix_y
    mu = np.zeros((ny, n), dtype=np.float64)
    acc = np.zeros((ny, n), dtype=np.float64)
    st = MapStats()
    rc = lib().or_map(ctypes.byref(params), m.size, _ptr(m), _ptr(xy), int(row_begin),
                      int(row_end), mu.ctypes.data_as(_dp), acc.ctypes.data_as(_dp),
                      ctypes.byref(st), nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle: bad row range or out of memory")
    stats = {"triangles": st.triangles, "dropped": st.dropped, "pieces": st.pieces}
    return (mu, acc, stats) if return_acc else (mu, stats)


def magnification_map_tile(params: Params, masses, pos_xy, row_begin, row_end, col_begin,
                           col_end, nthreads=None):
    """Map from the cells of rows [row_begin, row_end) and columns
    [col_begin, col_end) of the ray grid."""
    m = _f64(masses)
    xy = _f64(pos_xy).reshape(-1, 2)
    n, ny = params.npix, params.npix_y
    mu = np.zeros((ny, n), dtype=np.float64)
    acc = np.zeros((ny, n), dtype=np.float64)
    st = MapStats()
    rc = lib().or_map_tile(ctypes.byref(params), m.size, _ptr(m), _ptr(xy), int(row_begin),
                           int(row_end), int(col_begin), int(col_end), mu.ctypes.data_as(_dp),
                           acc.ctypes.data_as(_dp), ctypes.byref(st),
                           nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle: bad tile or out of memory")
    return mu, {"triangles": st.triangles, "dropped": st.dropped, "pieces": st.pieces}


def map_from_vertices(params: Params, w_xy, row_begin, row_end, nthreads=None):
    """IPM only: map from source positions of the vertices of rows
    [row_begin, row_end] (inclusive)."""
    w = _f64(w_xy).reshape(-1, 2)
    n, ny = params.npix, params.npix_y
    mu = np.zeros((ny, n), dtype=np.float64)
    acc = np.zeros((ny, n), dtype=np.float64)
    st = MapStats()
    rc = lib().or_map_from_vertices(ctypes.byref(params), _ptr(w), int(row_begin),
                                    int(row_end), mu.ctypes.data_as(_dp),
                                    acc.ctypes.data_as(_dp), ctypes.byref(st),
                                    nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle: bad row range")
    return mu, acc, {"triangles": st.triangles, "dropped": st.dropped, "pieces": st.pieces}


def map_tile_from_vertices(params: Params, w_xy, row_begin, row_end, col_begin, col_end,
                           nthreads=None):
    """IPM only: map of the cells of rows [row_begin, row_end) and columns
    [col_begin, col_end) from the source positions of their vertices (rows
    row_begin..row_end, columns col_begin..col_end inclusive, row-major)."""
    w = _f64(w_xy).reshape(-1, 2)
    if w.shape[0] != (row_end - row_begin + 1) * (col_end - col_begin + 1):
        raise ValueError("oracle: vertex array does not match the tile")
    n, ny = params.npix, params.npix_y
    mu = np.zeros((ny, n), dtype=np.float64)
    acc = np.zeros((ny, n), dtype=np.float64)
    st = MapStats()
    rc = lib().or_map_tile_from_vertices(ctypes.byref(params), _ptr(w), int(row_begin),
                                         int(row_end), int(col_begin), int(col_end),
                                         mu.ctypes.data_as(_dp), acc.ctypes.data_as(_dp),
                                         ctypes.byref(st), nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle: bad tile")
    return mu, {"triangles": st.triangles, "dropped": st.dropped, "pieces": st.pieces}


def irs_map(params: Params, masses, pos_xy, row_begin=0, row_end=-1, col_begin=0,
            col_end=-1, nthreads=None):
    """Inverse ray shooting over the vertices of rows [row_begin, row_end] and
    columns [col_begin, col_end] (inclusive; -1: the last).  Returns
    (mu, counts (npix, npix) int64, dropped)."""
    m = _f64(masses)
    xy = _f64(pos_xy).reshape(-1, 2)
    n, ny = params.npix, params.npix_y
    mu = np.zeros((ny, n), dtype=np.float64)
    cnt = np.zeros((ny, n), dtype=np.int64)
    dropped = ctypes.c_int64(0)
    rc = lib().or_irs_tile(ctypes.byref(params), m.size, _ptr(m), _ptr(xy), int(row_begin),
                           int(row_end), int(col_begin), int(col_end),
                           cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           mu.ctypes.data_as(_dp), ctypes.byref(dropped),
                           nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle: bad vertex range or out of memory")
    return mu, cnt, dropped.value


def tri_rect_area(tri, xlo, ylo, xhi, yhi):
    t = _f64(tri).reshape(6)
    return lib().or_tri_rect_area(_ptr(t), float(xlo), float(ylo), float(xhi), float(yhi))
