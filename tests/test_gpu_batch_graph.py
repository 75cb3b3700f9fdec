"""Batched maps in one persistent launch, CUDA-graph capture of mm_run, and
the full-size 5e5- and 1e6-star workloads on tiles of their ray grids, all
through the C ABI and against the FP64 oracle where it can afford it."""
import math

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
import synthetic
from _metrics import (DEFLECTION_TOL, MAP_P999_TOL, MEAN_TOL, assert_map_parity,
                      band_errors, deflection_rel_error)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()
    return torch


def batch_maps(oracle_mod, n_maps, seed=7):
    """Draws like the batched sweep (kappa, gamma, s, sizes), scaled down so the
    test is quick: npix 64-160, half-length 1.5-4, ~20 rays landing per pixel."""
    out = []
    for d in synthetic.batch_draws(seed, n_maps):
        kappa, gamma, s = d["kappa"], d["gamma"], d["s"]
        npix = 64 + (d["npix"] - 500) // 16
        hl = 1.5 + (d["half_length"] - 5.0) / 6.0
        rpp = 20.0 * abs((1 - kappa) ** 2 - gamma ** 2)
        ks = (1 - s) * kappa
        p0 = oracle_mod.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rays_per_pixel=rpp,
                                      flux_fraction_f=0.01)
        R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
        n = synthetic.n_stars_for(ks, R, synthetic.SALPETER_01_1)
        if n < 20 or n > 20000:
            continue
        m, pos = synthetic.star_field(d["seed"], n, R, synthetic.SALPETER_01_1)
        # few stars may not reach the shooting region's corners: skip those
        p = oracle_mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp,
                                     flux_fraction_f=0.01)
        if any(pos[:, k].min() > p.x0[k] or pos[:, k].max() < p.x0[k] + (p.n[k] - 1) * p.h[k]
               for k in (0, 1)):
            continue
        out.append(dict(kappa=kappa, gamma=gamma, s=s, npix=npix, hl=hl, rpp=rpp, m=m, pos=pos))
        if len(out) == n_maps:
            return out
    return out


def make(w, **kw):
    return mm.create(w["kappa"], w["gamma"], w["s"], w["m"], w["pos"], w["hl"], w["npix"],
                     w["rpp"], fmm_order=20, flux_fraction_f=0.01, **kw)


def test_batch_equals_single_runs_and_oracle(oracle_mod, torch_cuda):
    maps = batch_maps(oracle_mod, 6)
    assert len(maps) == 6
    hs = [make(w) for w in maps]
    mm.run_batch(hs, 0)
    batched = [mm.get_map_fixed(h) for h in hs]
    for h, b in zip(hs, batched):
        mm.run(h, 0)
        assert np.array_equal(mm.get_map_fixed(h), b)
    # the cheapest map of the batch against the oracle
    k = min(range(len(maps)), key=lambda i: mm.get_stats(hs[i])["rays"] * len(maps[i]["m"]))
    w = maps[k]
    mu = mm.get_map(hs[k])
    for h in hs:
        mm.destroy(h)
    p = oracle_mod.derive_params(w["kappa"], w["gamma"], w["s"], w["m"], w["hl"], w["npix"],
                                 rays_per_pixel=w["rpp"], flux_fraction_f=0.01)
    mu_ref, _ = oracle_mod.magnification_map(p, w["m"], w["pos"])
    assert_map_parity(mu, mu_ref, p.mu_macro)


def test_graph_capture_replays_the_same_map(torch_cuda):
    torch = torch_cuda
    maps = batch_maps(__import__("oracle"), 1, seed=11)
    h = make(maps[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        mm.run(h, s.cuda_stream)
    s.synchronize()
    eager = mm.get_map_fixed(h)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mm.run(h, s.cuda_stream)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(mm.get_map_fixed(h), eager)
    mm.destroy(h)


@pytest.mark.parametrize("name", ["near_critical_5000", "large_kroupa_10000"])
def test_full_size_workload_tiles(oracle_mod, torch_cuda, name):
    """Full-size grids (3.7e10 / 1.7e10 rays): sampled vertex deflections and
    the map of a 96 x 96-cell tile at the grid centre against the oracle."""
    wl = synthetic.workload(name)
    m, pos = wl.stars()
    p = oracle_mod.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, wl.npix,
                                 rays_per_pixel=wl.rays_per_pixel)
    args = (wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, wl.rays_per_pixel)
    c0, r0 = (p.n[0] - 1) // 2 - 48, (p.n[1] - 1) // 2 - 48
    h = mm.create(*args, fmm_order=wl.fmm_order, col_begin=c0, col_end=c0 + 96, row_begin=r0,
                  row_end=r0 + 96)
    st = mm.get_stats(h)
    assert st["params"]["n"] == list(p.n) and st["cells"] == 96 * 96
    mm.run(h, 0)
    mu = mm.get_map(h)
    rng = np.random.default_rng(3)
    i = rng.integers(c0, c0 + 97, 400)
    j = rng.integers(r0, r0 + 97, 400)
    z = oracle_mod.grid_vertices(p, i, j)
    w = mm.shoot_points(h, z)
    mm.destroy(h)
    err = deflection_rel_error(p, z, w, oracle_mod.deflect(p, m, pos, z))
    assert err.max() <= DEFLECTION_TOL, err.max()
    mu_ref, _ = oracle_mod.magnification_map_tile(p, m, pos, r0, r0 + 96, c0, c0 + 96)
    assert (mu_ref > 0).sum() > 10
    e = band_errors(mu, mu_ref, p.mu_macro)
    assert e["p999"] <= MAP_P999_TOL and e["mean_rel"] <= MEAN_TOL, e


def test_sweep_of_128_maps_autotuned_in_one_graph(oracle_mod, torch_cuda, tmp_path):
    """The batched sweep's shape: 128 maps of uneven sizes and (kappa, gamma,
    s), each autotuned (one shared cache), run as one batch captured in a
    CUDA graph.  The replay reproduces the eager batch bit for bit, single
    runs equal it, and the cheapest map meets the oracle."""
    torch = torch_cuda
    maps = batch_maps(oracle_mod, 128, seed=21)
    assert len(maps) == 128
    cache = str(tmp_path / "tune.jsonl")
    hs = [make(w, autotune=True, tune_cache=cache) for w in maps]
    assert {mm.get_stats(h)["autotuned"] for h in hs} <= {1, 2}
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        mm.run_batch(hs, s.cuda_stream)
    s.synchronize()
    eager = [mm.get_map_fixed(h) for h in hs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mm.run_batch(hs, s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    for h, e in zip(hs, eager):
        assert np.array_equal(mm.get_map_fixed(h), e)
    for k in (0, 63, 127):
        mm.run(hs[k], 0)
        assert np.array_equal(mm.get_map_fixed(hs[k]), eager[k])
    k = min(range(len(maps)), key=lambda i: mm.get_stats(hs[i])["rays"] * len(maps[i]["m"]))
    mu = mm.get_map(hs[k])
    for h in hs:
        mm.destroy(h)
    w = maps[k]
    p = oracle_mod.derive_params(w["kappa"], w["gamma"], w["s"], w["m"], w["hl"], w["npix"],
                                 rays_per_pixel=w["rpp"], flux_fraction_f=0.01)
    mu_ref, _ = oracle_mod.magnification_map(p, w["m"], w["pos"])
    assert_map_parity(mu, mu_ref, p.mu_macro)
