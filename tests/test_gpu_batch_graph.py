"""Batched maps in one persistent launch and CUDA-graph capture of mm_run
and mm_run_batch, through the C ABI, against the FP64 oracle (live, or the
stored oracle maps of tests/golden/sweep16.npz for 16 of the 128 maps of the
batched sweep's shape)."""
import os

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
from _metrics import assert_map_parity
from _sweep import batch_maps, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()
    return torch


def make(w, **kw):
    return mm.create(w["kappa"], w["gamma"], w["s"], w["m"], w["pos"], w["hl"], w["npix"],
                     w["rpp"], fmm_order=20, flux_fraction_f=0.01, **kw)


GOLDEN_SWEEP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep16.npz")


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


def test_sweep_of_128_maps_autotuned_in_one_graph(oracle_mod, torch_cuda, tmp_path):
    """The batched sweep's shape: 128 maps of uneven sizes and (kappa, gamma,
    s), each autotuned (one shared cache), run as one batch captured in a
    CUDA graph.  The replay reproduces the eager batch bit for bit, single
    runs equal it, and 16 maps spread over the sweep meet the oracle."""
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
    # 16 maps spread over the sweep (extremes of N_star and |mu_macro|, every
    # s, the oracle's costliest) against the oracle's stored maps
    g = np.load(GOLDEN_SWEEP)
    picks = [int(k) for k in g["picks"]]
    assert len(picks) == 16
    mus = {k: mm.get_map(hs[k]) for k in picks}
    for h in hs:
        mm.destroy(h)
    for k in picks:
        w = maps[k]
        assert int(g["m%d_draw" % k]) == w["draw"]
        p = oracle_params(oracle_mod, w)
        e = assert_map_parity(mus[k], g["m%d_mu" % k].astype(np.float64), p.mu_macro)
        print("sweep map %d (%d stars, s %.1f, mu_macro %.2f): p99.9 %.2e, mean rel %.2e"
              % (k, len(w["m"]), w["s"], p.mu_macro, e["p999"], e["mean_rel"]))
