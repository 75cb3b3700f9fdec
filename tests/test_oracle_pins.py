"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: values printed in
the paper (tests/golden/paper_numbers.txt), closed forms (the point lens, the
linear macro map), invariants (area conservation, symmetry, linearity) and
brute force (Monte-Carlo areas).  A dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def cross2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


# ---------------------------------------------------------------------------
# parameters (Sec. 2.1, 2.3, 3.1, App. A)
# ---------------------------------------------------------------------------

def test_extreme_example_macro_magnification(oracle_mod):
    """Sec. 5 prints (1-k+g)^-1 = 1.5 and (1-k-g)^-1 = -1000; the macro
    magnification must be their product, -1500."""
    g = golden()
    a1, a2 = 1.0 / g["inv_a1_extreme"], 1.0 / g["inv_a2_extreme"]
    kappa = 1.0 - 0.5 * (a1 + a2)
    gamma = 0.5 * (a1 - a2)
    p = oracle_mod.derive_params(kappa, gamma, g["smooth_extreme"], [1.0], 5.0, 64,
                                 rays_per_pixel=1.0)
    assert p.mu_macro == pytest.approx(g["inv_a1_extreme"] * g["inv_a2_extreme"], rel=1e-9)
    assert p.a1 == pytest.approx(a1, rel=1e-12)
    assert p.a2 == pytest.approx(a2, rel=1e-9)
    assert p.kappa_star == pytest.approx((1 - g["smooth_extreme"]) * kappa, rel=1e-12)


def test_refined_border_reduces_to_basic_rule(oracle_mod):
    """App. A's r = sqrt(kappa_* <m^2>/(f <m>)) with equal masses and f = 1/100
    is the basic 99%-flux border r = 10 sqrt(kappa_*) of Sec. 2.3."""
    g = golden()
    for kappa, s in [(0.4, 0.0), (0.7, 0.5), (0.2, 0.9)]:
        p = oracle_mod.derive_params(kappa, 0.1, s, np.ones(7), 3.0, 32, rays_per_pixel=1.0,
                                     flux_fraction_f=g["basic_border_flux_fraction"])
        ks = (1 - s) * kappa
        assert p.r_border == pytest.approx(g["basic_border_coeff"] * math.sqrt(ks), rel=1e-12)
    # default f is 1/1000: the border grows by sqrt(10)
    p = oracle_mod.derive_params(0.4, 0.1, 0.0, np.ones(7), 3.0, 32, rays_per_pixel=1.0)
    assert p.flux_fraction_f == g["default_flux_fraction"]
    assert p.r_border == pytest.approx(10 * math.sqrt(0.4) * math.sqrt(10), rel=1e-12)


def test_border_uses_mass_spectrum_moments(oracle_mod):
    """App. A: the tail of the deflection PDF scales with <m^2>/<m>; doubling
    every mass at fixed kappa_* scales r by sqrt(2)."""
    m, _ = synthetic.star_field(3, 500, 10.0, synthetic.SALPETER_01_1)
    p1 = oracle_mod.derive_params(0.5, 0.2, 0.3, m, 4.0, 32, rays_per_pixel=1.0)
    p2 = oracle_mod.derive_params(0.5, 0.2, 0.3, 2 * m, 4.0, 32, rays_per_pixel=1.0)
    assert p2.r_border / p1.r_border == pytest.approx(math.sqrt(2), rel=1e-12)


def test_shooting_region_is_macro_preimage_plus_border(oracle_mod):
    """Sec. 2.3: with no microlens deflection the map's corners must be the
    images of the shooting-region corners shrunk by the border: mapping the
    region's corner through the diagonal macro model gives the map corner
    plus r on each axis (absolute values)."""
    cy = (1.5, -0.75)
    p = oracle_mod.derive_params(0.3, 0.45, 0.2, np.ones(10), 2.5, 50, rays_per_pixel=4.0,
                                 center_y=cy)
    # region centre maps to the map centre under the macro model (Sec. 2.3)
    assert p.img_center[0] * p.a1 == pytest.approx(cy[0], rel=1e-14)
    assert p.img_center[1] * p.a2 == pytest.approx(cy[1], rel=1e-14)
    # half-widths map to half_length + r
    assert abs(p.img_half[0] * p.a1) == pytest.approx(2.5 + p.r_border, rel=1e-14)
    assert abs(p.img_half[1] * p.a2) == pytest.approx(2.5 + p.r_border, rel=1e-14)


def test_ray_grid_reading(oracle_mod):
    """Table 1 caption: rays per pixel counted in the absence of lensing, so
    spacing delta/sqrt(rpp); the grid covers the region and is centred on it."""
    p = oracle_mod.derive_params(0.5, 0.4, 0.5, np.ones(3), 10.0, 2000, rays_per_pixel=9.0)
    d = 20.0 / 2000
    assert p.h[0] == p.h[1] == pytest.approx(d / 3.0, rel=1e-15)
    for k in range(2):
        span = (p.n[k] - 1) * p.h[k]
        assert span >= 2 * p.img_half[k]
        assert span < 2 * p.img_half[k] + p.h[k] * 1.000001
        assert p.x0[k] + 0.5 * span == pytest.approx(p.img_center[k], abs=1e-12)
    # an explicit grid spans the explicit region exactly
    q = oracle_mod.derive_params(0.4, 0.3, 0.0, np.ones(3), 4.0, 256,
                                 img_half=(16 / 3, 16.0), ray_grid=(700, 2000))
    assert q.n[0] == 700 and q.n[1] == 2000
    assert q.x0[0] == pytest.approx(-16 / 3) and q.x0[1] == pytest.approx(-16.0)
    assert q.x0[0] + 699 * q.h[0] == pytest.approx(16 / 3, rel=1e-14)


def test_invalid_parameters_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.derive_params(0.5, 0.5, 0.0, [1.0], 1.0, 8, rays_per_pixel=1.0)  # |1-k|=g
    with pytest.raises(ValueError):
        oracle_mod.derive_params(0.5, 0.2, 1.5, [1.0], 1.0, 8, rays_per_pixel=1.0)
    with pytest.raises(ValueError):
        oracle_mod.derive_params(0.5, 0.2, 0.0, [1.0], 0.0, 8, rays_per_pixel=1.0)


# ---------------------------------------------------------------------------
# lens equation (Sec. 2.1-2.2, Sec. 3.1 footnote)
# ---------------------------------------------------------------------------

def _point_lens_params(oracle_mod, hl=2.0, npix=20, img_half=3.5, n=701):
    return oracle_mod.derive_params(0.0, 0.0, 0.0, [1.0], hl, npix,
                                    img_half=(img_half, img_half), ray_grid=(n, n))


def test_point_lens_image_positions(oracle_mod):
    """A unit point mass (kappa = gamma = 0): a source at distance u has images
    at x+- = (u +- sqrt(u^2+4))/2 along its direction (textbook point lens);
    the Einstein ring maps to the lens position."""
    p = _point_lens_params(oracle_mod)
    rng = np.random.default_rng(1)
    u = rng.uniform(0.05, 3.0, 50)
    phi = rng.uniform(0, 2 * np.pi, 50)
    e = np.stack([np.cos(phi), np.sin(phi)], 1)
    for sgn in (+1, -1):
        x = ((u + sgn * np.sqrt(u * u + 4)) / 2)[:, None] * e
        w = oracle_mod.deflect(p, [1.0], [[0.0, 0.0]], x)
        np.testing.assert_allclose(w, u[:, None] * e, rtol=0, atol=1e-12)
    ring = np.stack([np.cos(phi), np.sin(phi)], 1)
    w = oracle_mod.deflect(p, [1.0], [[0.0, 0.0]], ring)
    np.testing.assert_allclose(w, 0.0, atol=1e-14)


def test_macro_model_is_diagonal_matrix(oracle_mod):
    """No stars, kappa_* = 0: w = diag(1-k+g, 1-k-g) x (Sec. 2.1, vector form)."""
    p = oracle_mod.derive_params(0.3, 0.2, 1.0, [], 2.0, 8, rays_per_pixel=1.0)
    z = np.random.default_rng(2).normal(size=(20, 2)) * 5
    w = oracle_mod.deflect(p, [], np.zeros((0, 2)), z)
    np.testing.assert_allclose(w[:, 0], (1 - 0.3 + 0.2) * z[:, 0], rtol=1e-15)
    np.testing.assert_allclose(w[:, 1], (1 - 0.3 - 0.2) * z[:, 1], rtol=1e-15)


def test_sheet_term_compensates_star_mass(oracle_mod):
    """Sec. 3.1: the sheet has the stars' mean density with opposite sign, so
    inside a uniform star disk the mean of alpha_* + alpha_s over realisations
    vanishes; without the sheet it would be kappa_* z."""
    kappa, gamma, s = 0.6, 0.0, 0.0
    R, z0 = 30.0, np.array([[7.0, -4.0]])
    ks = (1 - s) * kappa
    n = synthetic.n_stars_for(ks, R, synthetic.EQUAL)
    p = oracle_mod.derive_params(kappa, gamma, s, np.ones(n), 2.0, 8, rays_per_pixel=1.0)
    nets = []
    for seed in range(60):
        m, pos = synthetic.star_field(500 + seed, n, R)
        w = oracle_mod.deflect(p, m, pos, z0)
        nets.append(((1 - kappa) * z0 - w)[0])        # alpha_* + alpha_s (gamma = 0)
    nets = np.array(nets)
    mean = nets.mean(0)
    sem = nets.std(0) / math.sqrt(len(nets))
    assert np.all(np.abs(mean) < 4 * sem + 0.05), (mean, sem)
    # the star term alone is far from zero: it is ~kappa_* z
    assert np.hypot(*(ks * z0[0])) > 10 * np.hypot(*sem)


def test_deflection_symmetries_and_linearity(oracle_mod):
    """Point reflection (z, z_i) -> (-z, -z_i) flips w; reflection about the
    x axis conjugates it (gamma real); the star term is additive over subsets."""
    m, pos = synthetic.star_field(11, 40, 6.0, synthetic.SALPETER_01_1)
    p = oracle_mod.derive_params(0.45, 0.25, 0.3, m, 2.0, 8, rays_per_pixel=1.0)
    z = np.random.default_rng(3).uniform(-3, 3, size=(30, 2))
    w = oracle_mod.deflect(p, m, pos, z)
    np.testing.assert_allclose(oracle_mod.deflect(p, m, -pos, -z), -w, rtol=1e-13, atol=1e-12)
    flip = np.array([1.0, -1.0])
    np.testing.assert_allclose(oracle_mod.deflect(p, m, pos * flip, z * flip), w * flip,
                               rtol=1e-13, atol=1e-12)
    p0 = oracle_mod.derive_params(0.45, 0.25, 0.3, m, 2.0, 8, rays_per_pixel=1.0)
    macro = oracle_mod.deflect(p0, [], np.zeros((0, 2)), z)
    a = oracle_mod.deflect(p, m[:17], pos[:17], z) - macro
    b = oracle_mod.deflect(p, m[17:], pos[17:], z) - macro
    np.testing.assert_allclose(a + b, w - macro, rtol=1e-12, atol=1e-11)
    # a star's pull is toward it: w is displaced away from the star direction
    one = oracle_mod.deflect(p0, [1.0], [[0.0, 0.0]], [[0.5, 0.0]]) - \
        oracle_mod.deflect(p0, [], np.zeros((0, 2)), [[0.5, 0.0]])
    assert one[0, 0] == pytest.approx(-2.0, rel=1e-14) and one[0, 1] == 0.0


# ---------------------------------------------------------------------------
# inverse polygon mapping (Sec. 3.2)
# ---------------------------------------------------------------------------

def test_triangle_rectangle_area_monte_carlo(oracle_mod):
    """Exact clipped area against Monte-Carlo point counting (brute force)."""
    rng = np.random.default_rng(4)
    pts = rng.uniform(size=(400000, 2)) * 3 - 0.5      # box [-0.5, 2.5]^2, area 9
    for _ in range(12):
        tri = rng.uniform(-0.3, 2.3, size=(3, 2))
        a, b, c = tri
        d = cross2(b - a, c - a)
        s1 = cross2(b - a, pts - a) * d >= 0
        s2 = cross2(c - b, pts - b) * d >= 0
        s3 = cross2(a - c, pts - c) * d >= 0
        inside = s1 & s2 & s3
        for (x0, y0) in [(0, 0), (1, 0), (0, 1), (1, 1)]:
            inr = (pts[:, 0] >= x0) & (pts[:, 0] < x0 + 1) & (pts[:, 1] >= y0) & (pts[:, 1] < y0 + 1)
            mc = 9.0 * np.mean(inside & inr)
            ex = oracle_mod.tri_rect_area(tri.ravel(), x0, y0, x0 + 1, y0 + 1)
            assert ex == pytest.approx(mc, abs=4 * math.sqrt(9 * mc / len(pts)) + 1e-3)


def test_triangle_fractions_conserve_area(oracle_mod):
    """A triangle well inside the map splits its unit of flux exactly among
    the pixels it covers, whatever its orientation (Sec. 3.2)."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        c = rng.uniform(3, 5, size=2)
        tri = c + rng.normal(size=(3, 2)) * rng.uniform(0.05, 1.5)
        tot = sum(oracle_mod.tri_rect_area(tri.ravel(), x, y, x + 1, y + 1)
                  for x in range(0, 9) for y in range(0, 9))
        area = 0.5 * abs(cross2(tri[1] - tri[0], tri[2] - tri[0]))
        assert tot == pytest.approx(area, rel=1e-11)


def test_zero_star_map_is_macro_magnification(oracle_mod):
    """No stars (s = 1): the mapping is linear, so every pixel covered by the
    mapped grid has exactly |mu_macro| (Sec. 3.1)."""
    for kappa, gamma in [(0.4, 0.3), (0.8, 0.25), (1.3, 0.2)]:
        p = oracle_mod.derive_params(kappa, gamma, 1.0, [], 2.0, 24, rays_per_pixel=5.0)
        mu, st = oracle_mod.magnification_map(p, [], np.zeros((0, 2)))
        assert st["dropped"] == 0
        np.testing.assert_allclose(mu, abs(p.mu_macro), rtol=1e-11)


def test_map_vs_brute_force_sampling(oracle_mod):
    """Tiny map: per-pixel area fractions against Monte-Carlo sampling of each
    mapped triangle (uniform barycentric points), an independent estimator."""
    m, pos = synthetic.star_field(21, 6, 2.0)
    p = oracle_mod.derive_params(0.3, 0.2, 0.0, m, 1.0, 6, img_half=(1.6, 1.6),
                                 ray_grid=(9, 9))
    mu, acc, st = oracle_mod.magnification_map(p, m, pos, return_acc=True)
    n = p.n[0]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n))
    w = oracle_mod.deflect(p, m, pos, oracle_mod.grid_vertices(p, ii.ravel(), jj.ravel()))
    w = ((w - (np.array(p.center_y) - p.half_length)) / p.delta).reshape(n, n, 2)
    rng = np.random.default_rng(6)
    K = 20000
    est = np.zeros((p.npix, p.npix))
    for j in range(n - 1):
        for i in range(n - 1):
            v00, v10, v01, v11 = w[j, i], w[j, i + 1], w[j + 1, i], w[j + 1, i + 1]
            for tri in ((v00, v10, v11), (v00, v11, v01)):
                r1, r2 = rng.uniform(size=K), rng.uniform(size=K)
                s = np.sqrt(r1)
                pts = (1 - s)[:, None] * tri[0] + (s * (1 - r2))[:, None] * tri[1] + \
                    (s * r2)[:, None] * tri[2]
                px = np.floor(pts).astype(int)
                ok = (px[:, 0] >= 0) & (px[:, 0] < p.npix) & (px[:, 1] >= 0) & (px[:, 1] < p.npix)
                np.add.at(est, (px[ok, 1], px[ok, 0]), 1.0 / K)
    assert st["triangles"] == 2 * (n - 1) ** 2
    err = np.abs(acc - est)
    assert np.all(err <= 0.02 + 0.02 * est), err.max()


def _pixel_average_point_lens(hl, npix, center=(0.0, 0.0), lens=(0.0, 0.0), order=12):
    """Pixel average of the point-lens magnification (u^2+2)/(u sqrt(u^2+4)),
    u the source distance from the lens, by Gauss-Legendre quadrature."""
    x, wgt = np.polynomial.legendre.leggauss(order)
    d = 2 * hl / npix
    out = np.zeros((npix, npix))
    for py in range(npix):
        for px in range(npix):
            xs = center[0] - hl + (px + 0.5 * (x + 1)) * d - lens[0]
            ys = center[1] - hl + (py + 0.5 * (x + 1)) * d - lens[1]
            X, Y = np.meshgrid(xs, ys)
            u = np.hypot(X, Y)
            mu = (u * u + 2) / (u * np.sqrt(u * u + 4))
            out[py, px] = 0.25 * np.sum(wgt[:, None] * wgt[None, :] * mu)
    return out


@pytest.mark.parametrize("center,lens,n,tol", [
    ((0.0, 0.0), (0.0, 0.0), 1441, 1e-4),
    ((0.3, -0.2), (0.55, -0.85), 721, 3e-4),
])
def test_point_lens_map_matches_closed_form(oracle_mod, center, lens, n, tol):
    """A single unit mass with no macro model: the IPM map converges (as h^2)
    to the pixel-averaged point-lens magnification (textbook closed form).
    The offset case pins the map orientation (row = y) and its centre."""
    hl, npix = 2.0, 20
    p = oracle_mod.derive_params(0.0, 0.0, 0.0, [1.0], hl, npix, center_y=center,
                                 img_half=(3.6, 3.6), ray_grid=(n, n))
    mu, st = oracle_mod.magnification_map(p, [1.0], [list(lens)])
    ref = _pixel_average_point_lens(hl, npix, center, lens)
    d = 2 * hl / npix
    cx = center[0] - hl + (np.arange(npix) + 0.5) * d - lens[0]
    cy = center[1] - hl + (np.arange(npix) + 0.5) * d - lens[1]
    X, Y = np.meshgrid(cx, cy)
    far = np.hypot(X, Y) > 2.5 * d            # quadrature is poor next to u = 0
    rel = np.abs(mu - ref) / ref
    assert rel[far].max() < tol, rel[far].max()
    # the total flux over the well-resolved pixels agrees far better
    assert abs(mu[far].sum() / ref[far].sum() - 1) < 1e-6


def test_mean_magnification_approaches_macro(oracle_mod):
    """App. A: averaged over realisations the map's mean is the macro
    magnification, up to the flux fraction f lost beyond the border."""
    kappa, gamma, s = 0.4, 0.2, 0.5
    ks = (1 - s) * kappa
    means = []
    for seed in range(4):
        p0 = oracle_mod.derive_params(kappa, gamma, s, np.ones(4), 2.0, 16,
                                      rays_per_pixel=4.0)
        R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
        n = synthetic.n_stars_for(ks, R, synthetic.EQUAL)
        m, pos = synthetic.star_field(700 + seed, n, R)
        p = oracle_mod.derive_params(kappa, gamma, s, m, 2.0, 16, rays_per_pixel=4.0)
        mu, st = oracle_mod.magnification_map(p, m, pos)
        means.append(mu.mean())
    mu_macro = 1.0 / ((1 - kappa) ** 2 - gamma ** 2)
    assert abs(np.mean(means) / mu_macro - 1) < 0.05, (means, mu_macro)


def test_map_rows_partition(oracle_mod):
    """Maps of disjoint cell-row bands add up to the full map (deterministic
    per-row work, used by the sampled CPU baseline)."""
    m, pos = synthetic.star_field(31, 30, 8.0)
    p = oracle_mod.derive_params(0.3, 0.1, 0.0, m, 2.0, 16, rays_per_pixel=2.0)
    full, _ = oracle_mod.magnification_map(p, m, pos)
    mid = (p.n[1] - 1) // 3
    a, _ = oracle_mod.magnification_map(p, m, pos, 0, mid)
    b, _ = oracle_mod.magnification_map(p, m, pos, mid, p.n[1] - 1)
    np.testing.assert_allclose(a + b, full, rtol=1e-12, atol=1e-12)


def test_irs_zero_star_counts_closed_form(oracle_mod):
    """Inverse ray shooting with no stars (s = 1): w = (a1 x, a2 y) with
    a1,2 = 1 - kappa -+ gamma (Sec. 2.1-2.2), so the rays per pixel are the
    product of per-axis lattice counts.  Every number here is dyadic, so the
    oracle's FP64 is exact and the counts are compared with exact rational
    arithmetic (ties on a pixel edge included)."""
    from fractions import Fraction as Fr
    kappa, gamma, hl, npix = 0.25, 0.125, 2.0, 16
    nx, ny, ihx, ihy = 41, 57, 2.5, 3.5
    p = oracle_mod.derive_params(kappa, gamma, 1.0, [], hl, npix, img_half=(ihx, ihy),
                                 ray_grid=(nx, ny))
    mu, cnt, dropped = oracle_mod.irs_map(p, [], np.zeros((0, 2)))
    assert dropped == 0
    delta = Fr(2 * hl) / npix

    def axis_counts(a, half, n):
        c = np.zeros(npix, dtype=np.int64)
        h = Fr(2 * half) / (n - 1)
        for i in range(n):
            k = math.floor((Fr(a) * (-Fr(half) + i * h) + Fr(hl)) / delta)
            if 0 <= k < npix:
                c[k] += 1
        return c

    cx = axis_counts(1 - kappa + gamma, ihx, nx)
    cy = axis_counts(1 - kappa - gamma, ihy, ny)
    np.testing.assert_array_equal(cnt, np.outer(cy, cx))   # row = y pixel
    np.testing.assert_allclose(mu, cnt * p.h[0] * p.h[1] / p.delta ** 2, rtol=1e-15)


def test_irs_statistics_agree_with_ipm(oracle_mod):
    """The paper's consistency check of the two mapping methods (Sec. 3.2,
    Table 1): on the same field, inverse ray shooting (rays counted per pixel)
    and inverse polygon mapping (exact areas) give the same magnification
    averaged over blocks of pixels, within the counting noise of the rays."""
    kappa, gamma, s, hl, npix, rpp = 0.45, 0.3, 0.4, 1.5, 32, 12.0
    p0 = oracle_mod.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rays_per_pixel=rpp,
                                  flux_fraction_f=0.01)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.EQUAL)
    m, pos = synthetic.star_field(41, n, R)
    p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                 flux_fraction_f=0.01)
    mu_ipm, _ = oracle_mod.magnification_map(p, m, pos)
    mu_irs, cnt, dropped = oracle_mod.irs_map(p, m, pos)
    assert dropped == 0
    b = 8
    blk = lambda a: a.reshape(npix // b, b, npix // b, b).sum(axis=(1, 3))
    rays = blk(cnt.astype(np.float64))
    ipm_rays = blk(mu_ipm) * p.delta ** 2 / (p.h[0] * p.h[1])   # expected rays per block
    assert rays.min() > 1000
    z = (rays - ipm_rays) / np.sqrt(ipm_rays)
    assert np.abs(z).max() < 5.0, z
    # the totals agree to the lattice's edge effects: much better than Poisson
    assert abs(rays.sum() / ipm_rays.sum() - 1) < 3.0 / math.sqrt(ipm_rays.sum())


# ---------------------------------------------------------------------------
# rectangular star region (App. B)
# ---------------------------------------------------------------------------

def _rect_params(oracle_mod, c1, c2, kappa=0.4, s=0.5):
    return oracle_mod.derive_params(kappa, 0.3, s, np.ones(4), 2.0, 16, rays_per_pixel=4.0,
                                    star_rect=(c1, c2))


def test_rect_sheet_matches_its_defining_integral(oracle_mod):
    """App. B's closed form against the defining area integral of the sheet,
    summed as a lattice of point masses (midpoint rule, O(h^2)): outside the
    rectangle and, with the lattice cell holding the point left out (its
    integral vanishes by symmetry), inside it."""
    c1, c2 = 5.0, 3.0
    p = _rect_params(oracle_mod, c1, c2)
    ks = p.kappa_star
    nx, ny = 1000, 600
    hx, hy = 2 * c1 / nx, 2 * c2 / ny
    X, Y = np.meshgrid(-c1 + (np.arange(nx) + 0.5) * hx, -c2 + (np.arange(ny) + 0.5) * hy)
    Z = X + 1j * Y
    mcell = -ks * hx * hy / math.pi           # point mass of one lattice cell
    for z in (8 + 2j, 1 + 5j, -7 - 4j, 5.5 + 0.2j):
        ref = np.sum(mcell / np.conj(z - Z))
        got = oracle_mod.alpha_rect(p, z.real, z.imag)
        assert abs(got - ref) < 1e-6 * abs(ref), (z, got, ref)
    for kx, ky in ((500, 300), (123, 77), (990, 20)):
        z = Z[ky, kx]
        d = np.conj(z - Z)
        d[ky, kx] = np.inf
        ref = np.sum(mcell / d)
        got = oracle_mod.alpha_rect(p, z.real, z.imag)
        assert abs(got - ref) < 2e-4 * ks * c1, (z, got, ref)


def test_rect_sheet_symmetry_continuity_and_limit(oracle_mod):
    """Odd in z and mirror-symmetric about the real axis (the sheet is);
    continuous across the rectangle's edges (the boxcar and step terms undo
    the branch cuts); and near the centre of a large square it is the
    disk's -kappa_star z."""
    c1, c2 = 4.0, 2.5
    p = _rect_params(oracle_mod, c1, c2)
    a = lambda z: oracle_mod.alpha_rect(p, z.real, z.imag)
    assert abs(a(0j)) < 1e-14
    for z in (1.3 + 0.4j, -3.1 + 2.0j, 6.0 - 3.0j, 0.2 - 2.4j):
        assert abs(a(-z) + a(z)) < 1e-12
        assert abs(a(z.conjugate()) - a(z).conjugate()) < 1e-12
    e = 1e-9
    for z in (c1 + 0.7j, -c1 - 1.9j, 1.1 + c2 * 1j, -2.2 - c2 * 1j, c1 + 2.4999j):
        d = z / abs(z)                         # outward-ish step across the edge
        assert abs(a(z + e * d) - a(z - e * d)) < 1e-7, z
    big = _rect_params(oracle_mod, 1000.0, 1000.0)
    for z in (3 + 2j, -5 + 7j):
        got = oracle_mod.alpha_rect(big, z.real, z.imag)
        assert abs(got + big.kappa_star * z) < 1e-4 * abs(big.kappa_star * z)


def test_rect_sheet_compensates_star_mass(oracle_mod):
    """As for the disk (Sec. 3.1): stars uniform in the rectangle plus its
    sheet have zero mean deflection inside it, over realisations."""
    kappa, gamma, s = 0.6, 0.0, 0.0
    c1, c2 = 24.0, 12.0
    z0 = np.array([[9.0, -5.0]])
    ks = (1 - s) * kappa
    n = synthetic.n_stars_for_rect(ks, (c1, c2), synthetic.EQUAL)
    p = oracle_mod.derive_params(kappa, gamma, s, np.ones(n), 2.0, 8, rays_per_pixel=1.0,
                                 star_rect=(c1, c2))
    nets = []
    for seed in range(60):
        m, pos = synthetic.star_field_rect(900 + seed, n, (c1, c2))
        w = oracle_mod.deflect(p, m, pos, z0)
        nets.append(((1 - kappa) * z0 - w)[0])
    nets = np.array(nets)
    mean = nets.mean(0)
    sem = nets.std(0) / math.sqrt(len(nets))
    assert np.all(np.abs(mean) < 4 * sem + 0.05), (mean, sem)


def test_non_square_map(oracle_mod):
    """A map of npix x npix_y square pixels (side 2 half_length / npix): its
    half-height is npix_y delta / 2, the shooting region's y half-width is
    (that + r) / |a2| (Sec. 2.3); with no stars every covered pixel has
    |mu_macro| (IPM), and the rays per pixel are exact lattice counts (IRS)."""
    from fractions import Fraction as Fr
    kappa, gamma, hl, nx, ny = 0.25, 0.125, 2.0, 16, 6
    p = oracle_mod.derive_params(kappa, gamma, 1.0, [], hl, nx, rays_per_pixel=5.0, npix_y=ny)
    assert (p.npix, p.npix_y) == (nx, ny) and p.half_length_y == 0.5 * ny * p.delta
    assert abs(p.img_half[1] - (p.half_length_y + p.r_border) / abs(p.a2)) < 1e-14
    mu, st = oracle_mod.magnification_map(p, [], np.zeros((0, 2)))
    assert mu.shape == (ny, nx) and st["dropped"] == 0
    np.testing.assert_allclose(mu, abs(p.mu_macro), rtol=1e-11)
    # IRS on a dyadic grid: per-axis lattice counts, exactly
    q = oracle_mod.derive_params(kappa, gamma, 1.0, [], hl, nx, img_half=(2.5, 3.5),
                                 ray_grid=(41, 57), npix_y=ny)
    _, cnt, _ = oracle_mod.irs_map(q, [], np.zeros((0, 2)))
    delta, hy = Fr(2 * hl) / nx, Fr(ny) * Fr(2 * hl) / nx / 2

    def axis(a, half, n, lo, npx):
        c = np.zeros(npx, dtype=np.int64)
        for i in range(n):
            k = math.floor((Fr(a) * (-Fr(half) + i * Fr(2 * half) / (n - 1)) - lo) / delta)
            if 0 <= k < npx:
                c[k] += 1
        return c

    cx = axis(1 - kappa + gamma, 2.5, 41, -Fr(hl), nx)
    cy = axis(1 - kappa - gamma, 3.5, 57, -hy, ny)
    np.testing.assert_array_equal(cnt, np.outer(cy, cx))


def test_tile_map_from_vertices_equals_the_tile_map(oracle_mod):
    """map_tile_from_vertices (the polygon mapping of given source positions,
    used to write the stored tile maps) apportions exactly what the direct
    tile map does: same vertices in, same map out."""
    m, pos = synthetic.star_field(61, 80, 9.0)
    p = oracle_mod.derive_params(0.45, 0.3, 0.4, m, 1.5, 40, rays_per_pixel=6.0,
                                 flux_fraction_f=0.01)
    r0, r1, c0, c1 = 40, 77, 13, 58
    ii, jj = np.meshgrid(np.arange(c0, c1 + 1), np.arange(r0, r1 + 1))
    w = oracle_mod.deflect(p, m, pos, oracle_mod.grid_vertices(p, ii.ravel(), jj.ravel()))
    a, sa = oracle_mod.map_tile_from_vertices(p, w, r0, r1, c0, c1)
    b, sb = oracle_mod.magnification_map_tile(p, m, pos, r0, r1, c0, c1)
    assert sa == sb and sa["triangles"] == 2 * (r1 - r0) * (c1 - c0)
    np.testing.assert_array_equal(a, b)
    with pytest.raises(ValueError):
        oracle_mod.map_tile_from_vertices(p, w[:-1], r0, r1, c0, c1)
