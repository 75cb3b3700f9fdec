"""Rectangular star region (App. B) through the C ABI against the oracle:
deflections (FMM with and without sub-cells, and the plain FP64 path) and a
small field's full map; plus the rectangle's validation."""
import math

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
import synthetic
from _metrics import DEFLECTION_TOL, assert_map_parity, deflection_rel_error

pytestmark = pytest.mark.gpu

KAPPA, GAMMA, S, HL, NPIX, RPP = 0.45, 0.3, 0.4, 1.5, 64, 10.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()


def rect_field(oracle_mod, seed=5, widen=(1.1, 1.0), kappa=KAPPA, gamma=GAMMA, s=S, hl=HL,
               npix=NPIX, rpp=RPP):
    """Stars uniform in a rectangle a little wider than the shooting region
    (half-widths widen[0] x the region's + widen[1] theta_E), as the paper
    suggests."""
    p0 = oracle_mod.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rays_per_pixel=rpp,
                                  flux_fraction_f=0.01)
    rect = (widen[0] * p0.img_half[0] + widen[1], widen[0] * p0.img_half[1] + widen[1])
    n = synthetic.n_stars_for_rect((1 - s) * kappa, rect, synthetic.EQUAL)
    m, pos = synthetic.star_field_rect(seed, n, rect)
    p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                 flux_fraction_f=0.01, star_rect=rect)
    return m, pos, p, rect


def grid(p):
    return dict(img_half=(0.5 * (p.n[0] - 1) * p.h[0], 0.5 * (p.n[1] - 1) * p.h[1]),
                ray_grid=(p.n[0], p.n[1]), center_y=tuple(p.center_y))


@pytest.mark.parametrize("sub_levels", [-1, 0])
def test_rect_deflection_vs_oracle(oracle_mod, sub_levels):
    # whole leaves (sub_levels -1) need corners farther away than sub-cells
    m, pos, p, rect = rect_field(oracle_mod, widen=(1.1, 1.0) if sub_levels == 0 else (2.0, 5.0))
    h = mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, RPP, fmm_order=25, flux_fraction_f=0.01,
                  sub_levels=sub_levels, star_rect=rect, **grid(p))
    rng = np.random.default_rng(2)
    z = oracle_mod.grid_vertices(p, rng.integers(0, p.n[0], 5000), rng.integers(0, p.n[1], 5000))
    w = mm.shoot_points(h, z)
    mm.destroy(h)
    err = deflection_rel_error(p, z, w, oracle_mod.deflect(p, m, pos, z))
    assert err.max() <= DEFLECTION_TOL, err.max()
    # the disk's sheet instead would be far off: the App. B terms are in use
    p_disk = oracle_mod.derive_params(KAPPA, GAMMA, S, m, HL, NPIX, rays_per_pixel=RPP,
                                      flux_fraction_f=0.01)
    err_disk = deflection_rel_error(p, z, w, oracle_mod.deflect(p_disk, m, pos, z))
    assert err_disk.max() > 1e3 * DEFLECTION_TOL


def test_rect_plain_fp64_deflection(oracle_mod):
    m, pos, p, rect = rect_field(oracle_mod, seed=6)
    h = mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, RPP, flux_fraction_f=0.01,
                  mode=mm.MM_PLAIN_FP64, star_rect=rect, **grid(p))
    rng = np.random.default_rng(3)
    z = oracle_mod.grid_vertices(p, rng.integers(0, p.n[0], 2000), rng.integers(0, p.n[1], 2000))
    w = mm.shoot_points(h, z)
    mm.destroy(h)
    err = deflection_rel_error(p, z, w, oracle_mod.deflect(p, m, pos, z))
    assert err.max() <= 1e-11, err.max()


def test_rect_map_parity(oracle_mod):
    m, pos, p, rect = rect_field(oracle_mod, seed=7)
    mu_ref, st_ref = oracle_mod.magnification_map(p, m, pos)
    h = mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, RPP, fmm_order=25, flux_fraction_f=0.01,
                  star_rect=rect, **grid(p))
    mm.run(h, 0)
    mu = mm.get_map(h)
    st = mm.get_stats(h)
    mm.destroy(h)
    assert_map_parity(mu, mu_ref, p.mu_macro)
    assert st["triangles_dropped"] == st_ref["dropped"]


def test_rect_must_contain_the_shooting_region(oracle_mod):
    m, pos, p, rect = rect_field(oracle_mod, seed=8)
    for bad in ((rect[0], 0.5 * p.img_half[1]), (0.9 * p.img_half[0], rect[1]), (-1.0, 2.0)):
        with pytest.raises(mm.MMError) as e:
            mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, RPP, fmm_order=25, flux_fraction_f=0.01,
                      star_rect=bad, **grid(p))
        assert e.value.status == mm.MM_EINVAL


def test_rect_corner_too_close_is_refused(oracle_mod):
    """A rectangle hugging the shooting region puts a corner next to a
    sub-cell, where the sheet's series would converge too slowly."""
    m, pos, p, rect = rect_field(oracle_mod, seed=9, widen=(1.01, 0.02))
    # four stars near the corners so that the stars still cover the region
    corners = 0.999 * np.array([[1, 1], [1, -1], [-1, 1], [-1, -1]]) * np.array(rect)
    m, pos = np.concatenate([m, np.ones(4)]), np.concatenate([pos, corners])
    with pytest.raises(mm.MMError) as e:
        mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, RPP, fmm_order=25, flux_fraction_f=0.01,
                  star_rect=rect, **grid(p))
    assert e.value.status == mm.MM_EINVAL and "star_rect" in str(e.value)
