"""GPU path against the FP64 oracle, element by element, through the C ABI.

Sizes: small enough for the oracle to finish in seconds, yet spanning many
warp work items (31-column strips x 64-row blocks), several tree levels and
ragged edges; plus the full-size plain-FP64 workload (700 x 2000 rays, 160
stars, 256^2 pixels) and the full-size FMM workload of the benchmark on
sampled vertices and invariants."""
import math

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
import synthetic
from _metrics import (DEFLECTION_TOL, MAP_P999_TOL, MEAN_TOL, assert_map_parity,
                      band_errors, deflection_rel_error, map_errors)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()


def oracle_inputs(oracle_mod, kappa, gamma, s, masses, hl, npix, rpp, **kw):
    return oracle_mod.derive_params(kappa, gamma, s, masses, hl, npix, rays_per_pixel=rpp, **kw)


def explicit_grid(p):
    """Ray grid of the oracle's parameters, passed explicitly to the GPU path."""
    return dict(img_half=(0.5 * (p.n[0] - 1) * p.h[0], 0.5 * (p.n[1] - 1) * p.h[1]),
                ray_grid=(p.n[0], p.n[1]), center_y=tuple(p.center_y))


def gpu_map(kappa, gamma, s, m, pos, hl, npix, **kw):
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, **kw)
    mm.run(h, 0)
    mu = mm.get_map(h)
    st = mm.get_stats(h)
    mm.destroy(h)
    return mu, st


def small_field(seed=7, kappa=0.45, gamma=0.3, s=0.4, hl=1.5, npix=64, rpp=10.0, f=0.01,
                mass_fn=synthetic.EQUAL):
    import oracle
    p0 = oracle.derive_params(kappa, gamma, s, np.ones(4) * mass_fn.m2_over_m, hl, npix,
                              rays_per_pixel=rpp, flux_fraction_f=f)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    n = synthetic.n_stars_for((1 - s) * kappa, R, mass_fn)
    m, pos = synthetic.star_field(seed, n, R, mass_fn)
    return m, pos


# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [mm.MM_FMM_FP32, mm.MM_PLAIN_FP64])
def test_zero_star_map(oracle_mod, mode):
    p = oracle_mod.derive_params(0.4, 0.3, 1.0, [], 2.0, 48, rays_per_pixel=5.0)
    mu_ref, _ = oracle_mod.magnification_map(p, [], np.zeros((0, 2)))
    mu, st = gpu_map(0.4, 0.3, 1.0, [], np.zeros((0, 2)), 2.0, 48, mode=mode, **explicit_grid(p))
    assert st["triangles_dropped"] == 0
    # FP32 clipping of the partially covered pixels: ~1e-6 relative
    np.testing.assert_allclose(mu, mu_ref, rtol=1e-5)
    np.testing.assert_allclose(mu, abs(p.mu_macro), rtol=1e-5)


@pytest.mark.parametrize("mode", [mm.MM_FMM_FP32, mm.MM_PLAIN_FP64])
def test_point_lens_map(oracle_mod, mode):
    lens = [[0.55, -0.85]]
    p = oracle_mod.derive_params(0.0, 0.0, 0.0, [1.0], 2.0, 20, center_y=(0.3, -0.2),
                                 img_half=(3.6, 3.6), ray_grid=(721, 721))
    mu_ref, st_ref = oracle_mod.magnification_map(p, [1.0], lens)
    mu, st = gpu_map(0.0, 0.0, 0.0, [1.0], lens, 2.0, 20, mode=mode, **explicit_grid(p))
    e = assert_map_parity(mu, mu_ref, p.mu_macro, p999=1e-5, mean=1e-6)
    assert st["triangles_dropped"] == st_ref["dropped"]


@pytest.mark.parametrize("sub_levels", [-1, 1, 2])
@pytest.mark.parametrize("order", [8, 16, 25])
def test_fmm_deflection_vs_direct_sum(oracle_mod, order, sub_levels):
    """FMM deflection against the direct sum at random points, with the local
    expansions evaluated about the leaf centres (-1) or re-centred on 4 or
    16 sub-cells per leaf with the correspondingly fewer terms."""
    kappa, gamma, s = 0.5, 0.4, 0.5
    m, pos = small_field(11, kappa, gamma, s, hl=2.0, npix=64, rpp=4.0,
                         mass_fn=synthetic.SALPETER_01_1)
    p = oracle_mod.derive_params(kappa, gamma, s, m, 2.0, 64, rays_per_pixel=4.0,
                                 flux_fraction_f=0.01)
    h = mm.create(kappa, gamma, s, m, pos, 2.0, 64, fmm_order=order, sub_levels=sub_levels,
                  **explicit_grid(p))
    rng = np.random.default_rng(5)
    z = np.stack([rng.uniform(p.x0[0], p.x0[0] + (p.n[0] - 1) * p.h[0], 20000),
                  rng.uniform(p.x0[1], p.x0[1] + (p.n[1] - 1) * p.h[1], 20000)], 1)
    w = mm.shoot_points(h, z)
    st = mm.get_stats(h)
    mm.destroy(h)
    w_ref = oracle_mod.deflect(p, m, pos, z)
    err = deflection_rel_error(p, z, w, w_ref)
    assert np.isfinite(w).all()
    assert st["depth"] >= 3
    assert st["sub_levels"] == max(sub_levels, 0)
    assert st["eval_order"] <= order
    if order == 25:
        assert st["eval_order"] == {-1: 25, 1: 15, 2: 15}[sub_levels]
    # truncation error falls with the order; at p = 25 the FP32 per-ray
    # arithmetic dominates and meets the deflection tolerance
    bound = {8: 2e-3, 16: 1e-4, 25: DEFLECTION_TOL}[order]
    assert err.max() <= bound, (order, err.max())


def test_map_parity_small_field(oracle_mod):
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.5, 64, 10.0
    m, pos = small_field(7, kappa, gamma, s, hl, npix, rpp)
    p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                 flux_fraction_f=0.01)
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    mu, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, **explicit_grid(p))
    e = assert_map_parity(mu, mu_ref, p.mu_macro)
    assert st["triangles_dropped"] == st_ref["dropped"]


def test_plain_fp64_full_size_workload(oracle_mod):
    wl = synthetic.workload("plain_fp64_160")
    m, pos = wl.stars()
    p = oracle_mod.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, wl.npix,
                                 img_half=wl.img_half, ray_grid=wl.ray_grid)
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    for mode in (mm.MM_PLAIN_FP64, mm.MM_FMM_FP32):
        # p = 25: the default order of App. C.3 aims at 1/10-pixel deflection
        # accuracy, looser than the map tolerance checked here
        mu, st = gpu_map(wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, mode=mode,
                         img_half=wl.img_half, ray_grid=wl.ray_grid, fmm_order=25)
        tol = 1e-4 if mode == mm.MM_PLAIN_FP64 else 1e-3
        assert_map_parity(mu, mu_ref, p.mu_macro, p999=tol)
        assert st["rays"] == 700 * 2000


def test_determinism_and_row_bands(oracle_mod):
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.5, 64, 10.0
    m, pos = small_field(3, kappa, gamma, s, hl, npix, rpp)
    p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                 flux_fraction_f=0.01)
    g = explicit_grid(p)
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, fmm_order=20, **g)
    mm.run(h, 0)
    a = mm.get_map_fixed(h)
    mm.run(h, 0)
    b = mm.get_map_fixed(h)
    mm.destroy(h)
    assert np.array_equal(a, b)
    rows = p.n[1] - 1
    cut = [0, rows // 3, rows // 3 + 1, rows]
    tot = np.zeros_like(a)
    for r0, r1 in zip(cut[:-1], cut[1:]):
        hb = mm.create(kappa, gamma, s, m, pos, hl, npix, fmm_order=20, row_begin=r0,
                       row_end=r1, **g)
        mm.run(hb, 0)
        tot += mm.get_map_fixed(hb)
        mm.destroy(hb)
    # bands see the same leaves only where the active region allows; the
    # per-vertex values are a function of the vertex, so sums are exact
    # up to leaves whose expansions differ between band trees (none here:
    # every band uses the same stars, and leaf locals do not depend on it)
    assert np.array_equal(tot, a)


def test_culling_leaves_the_map_unchanged():
    """Culling skips the vertex rows proven (per-sub-cell bounds) to land
    beyond the same map edge as the row below; the cells between such rows
    lie wholly outside the map, so the fixed-point map of the full benchmark
    workload is bit-identical to computing every vertex."""
    wl = synthetic.workload("fmm_fp32_salpeter_2000")
    m, pos = wl.stars()
    args = (wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, wl.rays_per_pixel)
    fixed, stats = [], []
    for cull in (True, False):
        h = mm.create(*args, fmm_order=wl.fmm_order, cull=cull)
        mm.run(h, 0)
        fixed.append(mm.get_map_fixed(h))
        stats.append(mm.get_stats(h))
        mm.destroy(h)
    assert stats[0]["rows_culled"] > 0 and stats[1]["rows_culled"] == 0
    for k in ("triangles_clipped", "triangles_line", "triangles_quad", "triangles_box",
              "triangles_rows", "triangles_dropped"):
        assert stats[0][k] == stats[1][k], k
    assert np.array_equal(fixed[0], fixed[1])


@pytest.mark.parametrize("mode", [mm.MM_FMM_FP32, mm.MM_PLAIN_FP64])
def test_second_pass_queue_sizes_leave_the_map_unchanged(mode):
    """Larger triangles go through the device queue to the second mapping
    pass; with no queue the first pass deals them all; in FMM mode a queue
    smaller than about one slot per 12 cells splits the first pass into
    segments, each drained by the second pass; batches that still do not fit
    are dealt in place and their reserved slots hold empty jobs.  The
    fixed-point map is the same in every case."""
    m, pos = small_field(23, 0.45, 0.3, 0.4, hl=1.5, npix=64, rpp=10.0, mass_fn=synthetic.EQUAL)
    maps, stats = [], []
    for slots in (0, -1, 700, 64):
        h = mm.create(0.45, 0.3, 0.4, m, pos, 1.5, 64, 10.0, fmm_order=20, flux_fraction_f=0.01,
                      mode=mode, big_queue_slots=slots)
        mm.run(h, 0)
        maps.append(mm.get_map_fixed(h))
        stats.append(mm.get_stats(h))
        mm.destroy(h)
    big = stats[0]["triangles_box"] + stats[0]["triangles_rows"]
    assert big > 1400, big  # more than a 700-slot queue holds at once
    for k in (1, 2, 3):
        assert np.array_equal(maps[0], maps[k]), k
    if mode == mm.MM_FMM_FP32:  # segments: more launches than one pass pair
        assert stats[2]["kernel_launches"] > stats[0]["kernel_launches"] + 2
        assert stats[3]["kernel_launches"] > stats[2]["kernel_launches"]


def test_near_critical_count_matches_the_oracle_geometry(oracle_mod):
    """mm_stats.triangles_near_critical against the same count taken from the
    oracle's FP64 vertices: triangles not wholly beyond one map edge whose
    local |mu| (image area / source area) exceeds the threshold."""
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.5, 64, 10.0
    m, pos = small_field(7, kappa, gamma, s, hl, npix, rpp)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=0.01)
    n0, n1 = p.n[0], p.n[1]
    jj, ii = np.meshgrid(np.arange(n1), np.arange(n0), indexing="ij")
    z = oracle_mod.grid_vertices(p, ii.ravel(), jj.ravel())
    w = oracle_mod.deflect(p, m, pos, z).reshape(n1, n0, 2)
    lo = np.array([p.center_y[0] - p.half_length, p.center_y[1] - p.half_length])
    u = (w - lo) / p.delta                       # source positions in pixel units
    v00, v10, v01, v11 = u[:-1, :-1], u[:-1, 1:], u[1:, :-1], u[1:, 1:]
    img2 = p.h[0] * p.h[1] / p.delta ** 2        # twice an image triangle's area
    for mu_c in (3.0, 30.0, 300.0):
        ref = 0
        for a, b, c in ((v00, v10, v11), (v00, v11, v01)):
            area2 = ((b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) -
                     (c[..., 0] - a[..., 0]) * (b[..., 1] - a[..., 1]))
            px = np.floor(np.stack([a[..., 0], b[..., 0], c[..., 0]]))
            py = np.floor(np.stack([a[..., 1], b[..., 1], c[..., 1]]))
            beyond = ((px.max(0) < 0) | (px.min(0) >= npix) | (py.max(0) < 0) |
                      (py.min(0) >= npix))
            ref += int(((np.abs(area2) < img2 / mu_c) & (area2 != 0) & ~beyond).sum())
        _, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, critical_mu=mu_c,
                        **explicit_grid(p))
        got = st["triangles_near_critical"]
        assert ref > 0
        assert abs(got - ref) <= 0.002 * ref + 5, (mu_c, got, ref)
    _, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, critical_mu=1e30,
                    **explicit_grid(p))
    assert st["triangles_near_critical"] == 0


def test_irs_counts_match_the_oracle(oracle_mod):
    """Inverse ray shooting (MM_FMM_IRS) against the oracle's FP64 rays: a
    ray's pixel is a floating-point decision, so the counts agree exactly
    except for rays within 2.5 x the deflection tolerance of a pixel edge;
    each such ray may land on either side.  Checked per pixel: 0 <= gpu - (oracle without them) <= the
    pixels they can reach.  Also: the full-map mean within counting noise of
    the polygon-mapping map, and the same counts with culling off."""
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.5, 64, 10.0
    m, pos = small_field(7, kappa, gamma, s, hl, npix, rpp)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=0.01)
    n0, n1 = p.n[0], p.n[1]
    jj, ii = np.meshgrid(np.arange(n1), np.arange(n0), indexing="ij")
    z = oracle_mod.grid_vertices(p, ii.ravel(), jj.ravel())
    w = oracle_mod.deflect(p, m, pos, z)
    lo = np.array([p.center_y[0] - p.half_length, p.center_y[1] - p.half_length])
    u = (w - lo) / p.delta
    f = np.floor(u).astype(np.int64)
    # per ray: 2.5 x the deflection tolerance, in pixels (>= 1e-4 px)
    zz = z.reshape(-1, 2)
    alpha = np.stack([(1 - kappa + gamma) * zz[:, 0], (1 - kappa - gamma) * zz[:, 1]], 1) - w
    scale = np.maximum(np.hypot(alpha[:, 0], alpha[:, 1]), math.sqrt(p.kappa_star))
    eps = np.maximum(1e-4, 2.5 * DEFLECTION_TOL * scale / p.delta)[:, None]
    d = u - f
    near_lo, near_hi = d < eps, d > 1 - eps
    edge = (near_lo | near_hi).any(axis=1)
    inside = lambda q: (q[:, 0] >= 0) & (q[:, 0] < npix) & (q[:, 1] >= 0) & (q[:, 1] < npix)
    sure = ~edge & inside(f)
    ref = np.zeros((npix, npix), dtype=np.int64)
    np.add.at(ref, (f[sure, 1], f[sure, 0]), 1)
    allow = np.zeros((npix, npix), dtype=np.int64)
    fe, le, he = f[edge], near_lo[edge], near_hi[edge]
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            okx = (ox == 0) | ((ox == -1) & le[:, 0]) | ((ox == 1) & he[:, 0])
            oky = (oy == 0) | ((oy == -1) & le[:, 1]) | ((oy == 1) & he[:, 1])
            q = fe + np.array([ox, oy])
            sel = okx & oky & inside(q)
            np.add.at(allow, (q[sel, 1], q[sel, 0]), 1)
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, mode=mm.MM_FMM_IRS,
                  **explicit_grid(p))
    mm.run(h, 0)
    cnt = mm.get_map_fixed(h).astype(np.int64)
    mu = mm.get_map(h)
    st = mm.get_stats(h)
    mm.destroy(h)
    assert edge.sum() < 0.01 * edge.size and st["triangles_dropped"] == 0
    diff = cnt - ref
    assert diff.min() >= 0 and (diff <= allow).all(), (diff.min(), (diff - allow).max())
    assert diff.sum() <= edge.sum()
    np.testing.assert_allclose(mu, cnt * p.h[0] * p.h[1] / p.delta ** 2, rtol=1e-6)
    # the oracle's own IRS map agrees the same way
    _, cnt_or, _ = oracle_mod.irs_map(p, m, pos)
    assert np.abs(cnt_or - cnt).sum() <= 2 * edge.sum()
    # the IPM map's mean, within the rays' counting noise
    mu_ipm, _ = oracle_mod.magnification_map(p, m, pos)
    assert abs(mu.mean() / mu_ipm.mean() - 1) < 3.0 / math.sqrt(cnt.sum())
    # culling skips only rays proven to land beyond the map: same counts
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, mode=mm.MM_FMM_IRS,
                  cull=False, **explicit_grid(p))
    mm.run(h, 0)
    assert np.array_equal(mm.get_map_fixed(h).astype(np.int64), cnt)
    mm.destroy(h)


def test_extreme_magnification_map(oracle_mod):
    """Sec. 5's extreme case, scaled down: kappa = 0.66717, gamma = 0.33383
    (mu_macro = -1500), s = 1 - 5e-5, Salpeter stars; 128^2 pixels over a
    4 x 4 source region with ~100 rays landing per pixel (a 54 x 34 747 ray
    grid 1000 times longer in y than in x).  The paper saw large FP32 errors
    here; the FP32 per-ray path (FP64 sub-cell centre images, macro factor
    formed in FP64) must meet the map tolerances, with sampled source
    positions within 1e-3 pixel of the oracle's."""
    kappa, gamma, s, hl, npix = 0.66717, 0.33383, 1 - 5e-5, 2.0, 128
    mu_macro = 1.0 / ((1 - kappa) ** 2 - gamma ** 2)
    rpp = 100.0 / abs(mu_macro)
    p0 = oracle_inputs(oracle_mod, kappa, gamma, s, np.ones(4), hl, npix, rpp)
    R = 1.05 * math.hypot(p0.img_half[0], p0.img_half[1])
    n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.SALPETER_01_1)
    m, pos = synthetic.star_field(77, n, R, synthetic.SALPETER_01_1)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp)
    assert abs(p.mu_macro + 1500.0) < 0.1 and p.n[1] > 600 * p.n[0]
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, **explicit_grid(p))
    mm.run(h, 0)
    mu = mm.get_map(h)
    rng = np.random.default_rng(4)
    zs = oracle_mod.grid_vertices(p, rng.integers(0, p.n[0], 4000), rng.integers(0, p.n[1], 4000))
    w = mm.shoot_points(h, zs)
    mm.destroy(h)
    # kappa_star = 3.3e-5: the relative measure's floor sqrt(kappa_star) is
    # 0.006 theta_E, a fifth of a pixel, below what FP32 offsets of ~100 px
    # from a sub-cell's FP64 centre image resolve; the error that decides the
    # map is the one in pixels
    err_px = np.hypot(*(w - oracle_mod.deflect(p, m, pos, zs)).T) / p.delta
    assert err_px.max() <= 1e-3, err_px.max()
    assert_map_parity(mu, mu_ref, p.mu_macro)


def test_map_centre_offset(oracle_mod):
    """A map centred off the origin (Sec. 2.3: the shooting region is the
    macro pre-image of the offset map plus the border) against the oracle."""
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.0, 48, 10.0
    cy = (0.7, -0.4)
    p0 = oracle_inputs(oracle_mod, kappa, gamma, s, np.ones(4), hl, npix, rpp,
                       flux_fraction_f=0.01, center_y=cy)
    R = 1.1 * (math.hypot(p0.img_center[0], p0.img_center[1]) +
               math.hypot(p0.img_half[0], p0.img_half[1]))
    n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.EQUAL)
    m, pos = synthetic.star_field(13, n, R)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=0.01,
                      center_y=cy)
    assert abs(p.img_center[0]) > 0.5 and abs(p.img_center[1]) > 0.5
    mu_ref, _ = oracle_mod.magnification_map(p, m, pos)
    mu, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, rays_per_pixel=rpp, fmm_order=25,
                     flux_fraction_f=0.01, center_y=cy)
    assert st["params"]["n"] == list(p.n)
    assert_map_parity(mu, mu_ref, p.mu_macro)


@pytest.mark.parametrize("mode", [mm.MM_FMM_FP32, mm.MM_PLAIN_FP64])
def test_star_on_a_grid_vertex(oracle_mod, mode):
    """A star exactly on a ray vertex: that ray's deflection is infinite, and
    the six triangles sharing the vertex are dropped (counted) by both
    implementations; the rest of the map still meets the tolerances.  The
    grid is dyadic (h = 1/64, origin -(4, 16)) so that the vertex and the
    star coincide exactly on both sides."""
    kappa, gamma, s, hl, npix = 0.45, 0.3, 0.4, 1.5, 64
    m, pos = small_field(7, kappa, gamma, s, hl, npix, 10.0)
    g = dict(img_half=(4.0, 16.0), ray_grid=(513, 2049))
    m2 = np.concatenate([m, [0.5]])
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m2, hl, npix, 0.0, flux_fraction_f=0.01, **g)
    assert p.h[0] == p.h[1] == 1.0 / 64 and p.x0[0] == -4.0 and p.x0[1] == -16.0
    v = oracle_mod.grid_vertices(p, [300], [900])
    pos2 = np.concatenate([pos, v])
    assert not np.isfinite(oracle_mod.deflect(p, m2, pos2, v)).all()
    mu_ref, st_ref = oracle_mod.magnification_map(p, m2, pos2)
    assert st_ref["dropped"] == 6
    mu, st = gpu_map(kappa, gamma, s, m2, pos2, hl, npix, fmm_order=25, mode=mode,
                     flux_fraction_f=0.01, **g)
    assert st["triangles_dropped"] == 6
    assert_map_parity(mu, mu_ref, p.mu_macro)


@pytest.mark.parametrize("mode", [mm.MM_FMM_FP32, mm.MM_PLAIN_FP64, mm.MM_FMM_IRS])
def test_non_square_map(oracle_mod, mode):
    """A map of 40 x 72 square pixels (npix_y = 72) against the oracle's map
    of the same shape: polygon mapping (FMM and plain FP64) to the map
    tolerances, ray counts to the total within the edge rays' allowance."""
    kappa, gamma, s, hl, npix, ny, rpp = 0.45, 0.3, 0.4, 1.0, 40, 72, 12.0
    p0 = oracle_inputs(oracle_mod, kappa, gamma, s, np.ones(4), hl, npix, rpp,
                       flux_fraction_f=0.01, npix_y=ny)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.EQUAL)
    m, pos = synthetic.star_field(17, n, R)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=0.01,
                      npix_y=ny)
    assert p.half_length_y == 0.5 * ny * p.delta
    mu, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, mode=mode, npix_y=ny,
                     flux_fraction_f=0.01, **explicit_grid(p))
    assert mu.shape == (ny, npix)
    assert st["params"]["npix_y"] == ny and st["params"]["half_length_y"] == p.half_length_y
    if mode == mm.MM_FMM_IRS:
        _, cnt, _ = oracle_mod.irs_map(p, m, pos)
        mu_ref = cnt * p.h[0] * p.h[1] / p.delta ** 2
        assert abs(mu.sum() / mu_ref.sum() - 1) < 1e-3
        rows = mu.sum(1) / mu_ref.sum(1)            # every row of the taller map is used
        assert np.all(np.abs(rows - 1) < 0.02), rows
    else:
        mu_ref, _ = oracle_mod.magnification_map(p, m, pos)
        assert_map_parity(mu, mu_ref, p.mu_macro)


def test_oversized_map_fails_with_enomem(oracle_mod):
    """A map whose accumulators exceed device memory (200 000^2 pixels, 640 GB)
    fails with MM_ENOMEM, allocating nothing it keeps; the GPU stays usable
    and the next handle works."""
    with pytest.raises(mm.MMError) as e:
        mm.create(0.4, 0.3, 1.0, [], np.zeros((0, 2)), 1.0, 200000, img_half=(2.0, 2.0),
                  ray_grid=(64, 64))
    assert e.value.status == mm.MM_ENOMEM
    mu, st = gpu_map(0.4, 0.3, 1.0, [], np.zeros((0, 2)), 1.0, 16, img_half=(2.0, 5.0),
                     ray_grid=(64, 160))
    assert st["triangles_dropped"] == 0 and mu.max() > 0


def test_irs_and_ipm_agree_at_full_size():
    """The paper's consistency check of the two mapping methods (Sec. 3.2,
    Table 1) on the benchmark workload at full size (1.475e9 rays): the ray
    counts per 40 x 40-pixel block (4e4 to 2e5 rays each) match the polygon
    mapping's expected counts within the counting noise, and the maps' means
    agree much better still."""
    wl = synthetic.workload("fmm_fp32_salpeter_2000")
    m, pos = wl.stars()
    args = (wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, wl.rays_per_pixel)
    maps = {}
    for mode in (mm.MM_FMM_FP32, mm.MM_FMM_IRS):
        h = mm.create(*args, fmm_order=wl.fmm_order, mode=mode)
        mm.run(h, 0)
        maps[mode] = mm.get_map(h).astype(np.float64)
        st = mm.get_stats(h)
        mm.destroy(h)
    per_ray = st["params"]["delta"] ** 2 / (st["params"]["h"][0] * st["params"]["h"][1])
    b = 40
    blk = lambda a: a.reshape(wl.npix // b, b, wl.npix // b, b).sum(axis=(1, 3)) * per_ray
    irs, ipm = blk(maps[mm.MM_FMM_IRS]), blk(maps[mm.MM_FMM_FP32])  # rays per block
    assert irs.min() > 2e4
    z = (irs - ipm) / np.sqrt(ipm)
    assert np.abs(z).max() < 6.0, np.abs(z).max()
    assert abs(irs.sum() / ipm.sum() - 1) < 2.0 / math.sqrt(ipm.sum())


def test_lanes_with_fewer_direct_stars(oracle_mod):
    """A field whose warps mix sub-cells with different numbers of direct
    stars (255 stars, 48^2 map, 715 x 2426 rays, p = 20).  A lane with fewer
    stars than the warp's most evaluates massless stand-ins; none may land on
    a vertex, so no triangle is dropped and the map meets the tolerances."""
    kappa, gamma, s, hl, npix, rpp, f = 0.45, 0.3, 0.4, 1.5, 48, 8.0, 0.01
    p0 = oracle_inputs(oracle_mod, kappa, gamma, s, np.ones(4), hl, npix, rpp, flux_fraction_f=f)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    m, pos = synthetic.star_field(5, synthetic.n_stars_for((1 - s) * kappa, R, synthetic.EQUAL), R)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=f)
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    for sub in (1, 2):
        mu, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=20, sub_levels=sub,
                         **explicit_grid(p))
        assert st["triangles_dropped"] == st_ref["dropped"] == 0, sub
        assert_map_parity(mu, mu_ref, p.mu_macro)


def _random_field(oracle_mod, k):
    """Field k of a seeded family of small maps: kappa, gamma, s, size, rays
    per pixel and mass function drawn per field (the oracle's map in seconds);
    draws whose few stars do not span the ray grid are redrawn."""
    for t in range(50):
        f = _random_field_draw(oracle_mod, 100 * k + t)
        _, m, pos, p = f
        if all(pos[:, a].min() <= p.x0[a] and pos[:, a].max() >= p.x0[a] + (p.n[a] - 1) * p.h[a]
               for a in (0, 1)):
            return f
    raise AssertionError("no covered draw")


def _random_field_draw(oracle_mod, k):
    u = synthetic.uniform(7000 + k, 0, 6)
    kappa, gamma = 0.2 + 0.6 * u[0], 0.1 + 0.5 * u[1]
    if abs(abs(1 - kappa) - gamma) < 0.08:
        gamma = abs(1 - kappa) + 0.1
    s = (0.0, 0.3, 0.6)[int(u[2] * 3)]
    npix = 24 + int(u[3] * 40)
    hl = 0.8 + 1.2 * u[4]
    rpp = 100.0 * abs((1 - kappa) ** 2 - gamma ** 2) / 8.0
    mass_fn = synthetic.SALPETER_01_1 if u[5] < 0.5 else synthetic.EQUAL
    p0 = oracle_inputs(oracle_mod, kappa, gamma, s, np.ones(4), hl, npix, rpp, flux_fraction_f=0.01)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    m, pos = synthetic.star_field(7100 + k, synthetic.n_stars_for((1 - s) * kappa, R, mass_fn), R,
                                  mass_fn)
    p = oracle_inputs(oracle_mod, kappa, gamma, s, m, hl, npix, rpp, flux_fraction_f=0.01)
    return (kappa, gamma, s, hl, npix), m, pos, p


@pytest.mark.parametrize("k", range(8))
def test_random_small_fields(oracle_mod, k):
    """Eight seeded random fields, each with whole leaves and with one and two
    sub-cell levels: the dropped-triangle count equals the oracle's and the
    map meets the tolerances."""
    (kappa, gamma, s, hl, npix), m, pos, p = _random_field(oracle_mod, k)
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    for sub in (-1, 1, 2):
        mu, st = gpu_map(kappa, gamma, s, m, pos, hl, npix, fmm_order=25, sub_levels=sub,
                         **explicit_grid(p))
        assert st["triangles_dropped"] == st_ref["dropped"], (sub, st["triangles_dropped"])
        assert_map_parity(mu, mu_ref, p.mu_macro)
