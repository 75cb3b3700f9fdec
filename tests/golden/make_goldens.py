"""Writes the stored oracle maps the full-size parity tests compare against.

Every value written here comes from the FP64 oracle (``oracle/``) on the
seeded star fields of ``synthetic`` -- nothing from the CUDA path.  Run from
the repository root; each part is written to its own file:

    python tests/golden/make_goldens.py twin     # fmm_fp32_salpeter_2000's twin
    python tests/golden/make_goldens.py tiles near_critical_5000
    python tests/golden/make_goldens.py tiles large_kroupa_10000
    python tests/golden/make_goldens.py sweep    # 16 sweep-shaped maps

twin: the 2000^2-pixel FP32 workload's downscaled twin -- the same stars,
  kappa, gamma, s and map extent, 400^2 pixels and ~20 rays landing per
  pixel -- as a full oracle map, plus the oracle's mean magnification of the
  same twin at ~5 rays landing per pixel.  Two ray densities of one map give
  the size of the discretisation error of the mean (see the parity test).

tiles: 8 tiles of 256 x 256 cells of a full-size ray grid, chosen from the
  oracle's own deflections at a sample of candidate tiles (never from map
  values): the two whose sampled triangles have the most near-critical
  orientation changes and largest local |mu|, the two with the most sampled
  multi-pixel triangles, and one straddling each of the four map edges --
  each among the tiles whose oracle map fits 1024 x 1024 pixels.
  For each tile: the oracle's map over the tile's pixel window, and from
  the oracle's FP64 vertices the near-critical triangle count (local |mu|
  above 1e3, not wholly beyond one map edge), the pixels those triangles'
  boxes touch, and the count of triangles spanning more than one pixel.

sweep: the full oracle maps of 16 of the 128 sweep-shaped maps of the batch
  test (tests/_sweep.py, seed 21), picked from the draws alone.
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synthetic  # noqa: E402
import _sweep  # noqa: E402

TILE = 256
CRITICAL_MU = 1e3
MAX_WINDOW = 1024   # pixels per axis of a stored tile map


def log(*a):
    print(time.strftime("%H:%M:%S"), *a, flush=True)


# ---------------------------------------------------------------------------
# twin of the 2000^2 FP32 workload
# ---------------------------------------------------------------------------

TWIN_NAME = "fmm_fp32_salpeter_2000"
TWIN_NPIX = 400
TWIN_LANDING = 20.0     # rays landing per pixel
TWIN_LANDING_COARSE = 5.0


def twin_params(wl, m, landing):
    mu = 1.0 / abs((1 - wl.kappa) ** 2 - wl.gamma ** 2)
    return oracle.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, TWIN_NPIX,
                                rays_per_pixel=landing / mu)


def make_twin():
    wl = synthetic.workload(TWIN_NAME)
    m, pos = wl.stars()
    out = {}
    for tag, landing in (("coarse", TWIN_LANDING_COARSE), ("", TWIN_LANDING)):
        p = twin_params(wl, m, landing)
        log("twin", tag or "main", "grid", p.n[0], p.n[1], "stars", len(m))
        t0 = time.time()
        mu, st = oracle.magnification_map(p, m, pos)
        log("  done in %.0f s, mean %.9f" % (time.time() - t0, mu.mean()))
        if tag:
            out["mean_coarse"] = mu.mean()
            out["rpp_coarse"] = landing * abs((1 - wl.kappa) ** 2 - wl.gamma ** 2)
        else:
            out["mu"] = mu.astype(np.float32)
            out["mean"] = mu.mean()
            out["dropped"] = st["dropped"]
            out["rpp"] = landing * abs((1 - wl.kappa) ** 2 - wl.gamma ** 2)
            out["n"] = np.array(p.n)
    out["npix"] = TWIN_NPIX
    out["n_stars"] = len(m)
    out["star_checksum"] = np.array([m.sum(), pos.sum(), (pos * pos).sum()])
    path = os.path.join(HERE, "twin_%s.npz" % TWIN_NAME)
    np.savez_compressed(path, **out)
    log("wrote", path)


# ---------------------------------------------------------------------------
# tiles of the 5000^2 and 10000^2 workloads
# ---------------------------------------------------------------------------

def tri_geometry(p, w00, w10, w11):
    """Signed source area (pixel^2), local |mu| and pixel box of triangles."""
    d = p.delta
    lox = p.center_y[0] - p.half_length
    loy = p.center_y[1] - p.half_length_y
    u = [((w[..., 0] - lox) / d, (w[..., 1] - loy) / d) for w in (w00, w10, w11)]
    area2 = ((u[1][0] - u[0][0]) * (u[2][1] - u[0][1])
             - (u[1][1] - u[0][1]) * (u[2][0] - u[0][0]))
    img2 = p.h[0] * p.h[1] / (d * d)         # twice the image triangle's area in px^2
    with np.errstate(divide="ignore"):
        mu_loc = img2 / np.abs(area2)
    xs = np.stack([u[k][0] for k in range(3)])
    ys = np.stack([u[k][1] for k in range(3)])
    return area2, mu_loc, xs, ys


def beyond_one_edge(p, xs, ys):
    return ((xs < 0).all(0) | (xs >= p.npix).all(0) | (ys < 0).all(0)
            | (ys >= p.npix_y).all(0))


def sample_candidates(p, m, pos, n_cand, n_cells, seed):
    """Random candidate tiles whose macro image meets the map, each sampled
    at n_cells random cells (triangle v00, v10, v11) plus its corners."""
    n_rows, n_cols = p.n[1] - 1, p.n[0] - 1
    a1, a2 = p.a1, p.a2
    reach = p.r_border + 2.0 * TILE * max(p.h) * max(abs(a1), abs(a2))
    rows, cols = [], []
    k = 0
    while len(rows) < n_cand:
        u = synthetic.uniform(seed, 500 + k, 2)
        k += 1
        r0 = int(u[0] * (n_rows - TILE))
        c0 = int(u[1] * (n_cols - TILE))
        zc = oracle.grid_vertices(p, c0 + TILE / 2, r0 + TILE / 2)
        yc = (a1 * zc[0] - p.center_y[0], a2 * zc[1] - p.center_y[1])
        if abs(yc[0]) <= p.half_length + reach and abs(yc[1]) <= p.half_length_y + reach:
            rows.append(r0)
            cols.append(c0)
    rows = np.array(rows)
    cols = np.array(cols)
    ui = synthetic.uniform(seed, 9000, n_cand * n_cells).reshape(n_cand, n_cells)
    uj = synthetic.uniform(seed, 9001, n_cand * n_cells).reshape(n_cand, n_cells)
    ci = cols[:, None] + (ui * TILE).astype(np.int64)
    cj = rows[:, None] + (uj * TILE).astype(np.int64)
    pts = np.concatenate([oracle.grid_vertices(p, ci, cj).reshape(-1, 2),
                          oracle.grid_vertices(p, ci + 1, cj).reshape(-1, 2),
                          oracle.grid_vertices(p, ci + 1, cj + 1).reshape(-1, 2)])
    log("  deflecting %d sample points" % len(pts))
    w = oracle.deflect(p, m, pos, pts).reshape(3, n_cand, n_cells, 2)
    return rows, cols, w


def score_candidates(p, w):
    area2, mu_loc, xs, ys = tri_geometry(p, w[0], w[1], w[2])
    live = ~beyond_one_edge(p, xs, ys)
    # near-critical: both orientations among the live samples, then large |mu|
    pos_o = ((area2 > 0) & live).any(1)
    neg_o = ((area2 < 0) & live).any(1)
    crit = (pos_o & neg_o) * 1e6 + np.where(live, np.minimum(mu_loc, 1e6), 0).max(1)
    multi = ((np.floor(xs).min(0) != np.floor(xs).max(0))
             | (np.floor(ys).min(0) != np.floor(ys).max(0))) & live
    multi_score = multi.sum(1)
    # edges: sampled points on both sides of each map edge, within the other
    # axis's extent
    xall = w[..., 0].transpose(1, 0, 2).reshape(w.shape[1], -1)
    yall = w[..., 1].transpose(1, 0, 2).reshape(w.shape[1], -1)
    lox = p.center_y[0] - p.half_length
    hix = p.center_y[0] + p.half_length
    loy = p.center_y[1] - p.half_length_y
    hiy = p.center_y[1] + p.half_length_y
    iny = (yall >= loy) & (yall < hiy)
    inx = (xall >= lox) & (xall < hix)
    edges = []
    for line, coord, inside in ((lox, xall, iny), (hix, xall, iny), (loy, yall, inx),
                                (hiy, yall, inx)):
        a = ((coord < line) & inside).sum(1)
        b = ((coord >= line) & inside).sum(1)
        edges.append(np.minimum(a, b))
    return crit, multi_score, edges


def tile_reference(p, m, pos, r0, c0):
    """The oracle's map of one tile (over its pixel window) and the FP64
    vertex statistics of its triangles."""
    t0 = time.time()
    ii, jj = np.meshgrid(np.arange(c0, c0 + TILE + 1), np.arange(r0, r0 + TILE + 1))
    z = oracle.grid_vertices(p, ii.ravel(), jj.ravel())
    w = oracle.deflect(p, m, pos, z).reshape(TILE + 1, TILE + 1, 2)
    mu, st = oracle.map_tile_from_vertices(p, w, r0, r0 + TILE, c0, c0 + TILE)
    w00, w10, w11, w01 = w[:-1, :-1], w[:-1, 1:], w[1:, 1:], w[1:, :-1]
    crit_mask = np.zeros((p.npix_y, p.npix), dtype=bool)
    n_crit = n_multi = 0
    for a, b, c in ((w00, w10, w11), (w00, w11, w01)):
        area2, mu_loc, xs, ys = tri_geometry(p, a, b, c)
        live = ~beyond_one_edge(p, xs, ys) & np.isfinite(area2) & (area2 != 0)
        crit = live & (mu_loc > CRITICAL_MU)
        n_crit += int(crit.sum())
        fx0, fx1 = np.floor(xs.min(0)), np.floor(xs.max(0))
        fy0, fy1 = np.floor(ys.min(0)), np.floor(ys.max(0))
        n_multi += int((live & ((fx0 != fx1) | (fy0 != fy1))).sum())
        for x0, x1, y0, y1 in zip(fx0[crit], fx1[crit], fy0[crit], fy1[crit]):
            x0, x1 = int(max(x0, 0)), int(min(x1, p.npix - 1))
            y0, y1 = int(max(y0, 0)), int(min(y1, p.npix_y - 1))
            if x0 <= x1 and y0 <= y1:
                crit_mask[y0:y1 + 1, x0:x1 + 1] = True
    nz = np.argwhere((mu > 0) | crit_mask)
    if len(nz):
        (py0, px0), (py1, px1) = nz.min(0), nz.max(0) + 1
    else:
        py0 = px0 = 0
        py1 = px1 = 1
    log("  tile r%d c%d: %.0f s, %d near-critical, %d multi-pixel, window %dx%d, sum %.6g"
        % (r0, c0, time.time() - t0, n_crit, n_multi, px1 - px0, py1 - py0, mu.sum()))
    return dict(window=np.array([py0, py1, px0, px1]), mu=mu[py0:py1, px0:px1],
                crit_mask=crit_mask[py0:py1, px0:px1], n_crit=n_crit, n_multi=n_multi,
                dropped=st["dropped"], total=mu.sum())


def make_tiles(name, n_cand=2000, n_cells=16):
    wl = synthetic.workload(name)
    m, pos = wl.stars()
    p = oracle.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, wl.npix,
                             rays_per_pixel=wl.rays_per_pixel)
    log(name, "grid", p.n[0], p.n[1], "stars", len(m))
    rows, cols, w = sample_candidates(p, m, pos, n_cand, n_cells, seed=7000 + len(m) % 997)
    crit, multi, edges = score_candidates(p, w)
    picks, kinds = [], []

    def overlaps(k):
        return any(abs(rows[k] - rows[q]) < TILE and abs(cols[k] - cols[q]) < TILE
                   for q in picks)

    def take(order, kind, n, need=None):
        got = 0
        for k in order:
            if got == n:
                break
            if overlaps(k) or (need is not None and not need(k)):
                continue
            picks.append(k)
            kinds.append(kind)
            got += 1

    refs = {}

    def compact(k):
        # the tile's oracle map must fit a window of MAX_WINDOW^2 pixels (a
        # tile holding a star spreads its cells over the whole map)
        if k not in refs:
            refs[k] = tile_reference(p, m, pos, int(rows[k]), int(cols[k]))
        py0, py1, px0, px1 = refs[k]["window"]
        return py1 - py0 <= MAX_WINDOW and px1 - px0 <= MAX_WINDOW

    take(np.argsort(-crit, kind="stable"), "near_critical", 2, need=compact)
    take(np.argsort(-multi, kind="stable"), "multi_pixel", 2, need=compact)
    for e, tag in enumerate(("edge_left", "edge_right", "edge_bottom", "edge_top")):
        take(np.argsort(-edges[e], kind="stable"), tag, 1,
             need=lambda k, e=e: edges[e][k] > 0 and compact(k))
    out = {"name": name, "tile": TILE, "n": np.array(p.n), "n_stars": len(m),
           "star_checksum": np.array([m.sum(), pos.sum(), (pos * pos).sum()])}
    for t, (k, kind) in enumerate(zip(picks, kinds)):
        ref = refs[k]
        out["t%d_origin" % t] = np.array([rows[k], cols[k]])
        out["t%d_kind" % t] = kind
        for key, v in ref.items():
            out["t%d_%s" % (t, key)] = v.astype(np.float32) if key == "mu" else v
    out["n_tiles"] = len(picks)
    path = os.path.join(HERE, "tiles_%s.npz" % name)
    np.savez_compressed(path, **out)
    log("wrote", path, "with", len(picks), "tiles")


# ---------------------------------------------------------------------------
# 16 of the 128 sweep-shaped maps
# ---------------------------------------------------------------------------

SWEEP_SEED = 21
SWEEP_MAPS = 128
SWEEP_PICK = 16


def make_sweep():
    maps = _sweep.batch_maps(oracle, SWEEP_MAPS, seed=SWEEP_SEED)
    assert len(maps) == SWEEP_MAPS
    picks = _sweep.pick_spread(maps, SWEEP_PICK)
    out = {"picks": np.array(picks)}
    for k in picks:
        w = maps[k]
        p = _sweep.oracle_params(oracle, w)
        t0 = time.time()
        mu, st = oracle.magnification_map(p, w["m"], w["pos"])
        log("sweep map %d: %d stars, %dx%d rays, npix %d, s %.1f, mu_macro %.2f: %.0f s"
            % (k, len(w["m"]), p.n[0], p.n[1], w["npix"], w["s"], p.mu_macro,
               time.time() - t0))
        out["m%d_mu" % k] = mu.astype(np.float32)
        out["m%d_mean" % k] = mu.mean()
        out["m%d_dropped" % k] = st["dropped"]
        out["m%d_draw" % k] = w["draw"]
    path = os.path.join(HERE, "sweep%d.npz" % SWEEP_PICK)
    np.savez_compressed(path, **out)
    log("wrote", path)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else ""
    if what == "twin":
        make_twin()
    elif what == "tiles":
        make_tiles(sys.argv[2])
    elif what == "sweep":
        make_sweep()
    else:
        sys.exit(__doc__)
