"""The autotuner of mm_create (mm_options.autotune and tune_cache): it picks
among its candidate settings, the map it then computes meets the oracle's
tolerances, its choice is written to a JSON-lines cache and reused from
there, and the tuned handle equals one created with the chosen settings
given explicitly (bit for bit, also inside a batch)."""
import json

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
from _metrics import assert_map_parity
from test_gpu_parity import explicit_grid, small_field

pytestmark = pytest.mark.gpu

KAPPA, GAMMA, S, HL, NPIX, RPP = 0.45, 0.3, 0.4, 1.5, 64, 10.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()


def field(oracle_mod, seed=7):
    m, pos = small_field(seed, KAPPA, GAMMA, S, HL, NPIX, RPP)
    p = oracle_mod.derive_params(KAPPA, GAMMA, S, m, HL, NPIX, rays_per_pixel=RPP,
                                 flux_fraction_f=0.01)
    return m, pos, p


def make(m, pos, p, **kw):
    return mm.create(KAPPA, GAMMA, S, m, pos, HL, NPIX, fmm_order=25, **explicit_grid(p), **kw)


def fixed_map(h):
    mm.run(h, 0)
    return mm.get_map_fixed(h)


def choice(st):
    return st["leaf_size"], st["sub_levels"], st["rows_per_item"]


def default_queue(cells, jobs_per_mcell):
    """The default second-pass queue of a map that fits half the L2: the
    larger triangles the tuner counted, scaled to the grid, plus a quarter
    (else one per 12 cells), within 2^16 .. 2^27 slots."""
    if jobs_per_mcell >= 0:
        est = -(-cells * jobs_per_mcell // 2**20)
        return min(2**27, max(2**16, est + est // 4 + 4096))
    return min(2**27, max(2**16, cells // 12))


def test_autotune_chooses_caches_and_meets_the_oracle(oracle_mod, tmp_path):
    m, pos, p = field(oracle_mod)
    cache = tmp_path / "tune.jsonl"
    h = make(m, pos, p, autotune=True, tune_cache=str(cache))
    st = mm.get_stats(h)
    assert st["autotuned"] == 1 and st["ms_autotune"] > 0.0
    assert st["leaf_size"] in (16, 32, 64) and st["sub_levels"] in (1, 2)
    fixed = fixed_map(h)
    after = mm.get_stats(h)
    jobs = after["triangles_box"] + after["triangles_rows"]
    mu = mm.get_map(h)
    mm.destroy(h)
    mu_ref, _ = oracle_mod.magnification_map(p, m, pos)
    assert_map_parity(mu, mu_ref, p.mu_macro)

    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["key"].startswith("sm_") and rec["ms_estimate"] > 0.0
    assert (rec["leaf_size"], rec["sub_levels"]) == (st["leaf_size"], st["sub_levels"])
    assert rec["rows_per_item"] in (0, 64, 512)
    # the larger triangles the tuner counted size the handle's queue: at
    # least the ones this run queued (statistics box + rows), one per slot
    assert jobs > 0 and rec["jobs_per_mcell"] >= 0
    assert st["queue_slots"] == default_queue(st["cells"], rec["jobs_per_mcell"])
    assert st["queue_slots"] >= jobs

    # the cached choice is taken without timing, and the map is the same
    h2 = make(m, pos, p, autotune=True, tune_cache=str(cache))
    st2 = mm.get_stats(h2)
    assert st2["autotuned"] == 2 and choice(st2) == choice(st)
    assert np.array_equal(fixed_map(h2), fixed)
    mm.destroy(h2)
    assert len(cache.read_text().splitlines()) == 1

    # the same settings given explicitly: the same map
    h3 = make(m, pos, p, leaf_size=rec["leaf_size"], sub_levels=rec["sub_levels"],
              rows_per_item=rec["rows_per_item"])
    st3 = mm.get_stats(h3)
    assert st3["autotuned"] == 0 and st3["ms_autotune"] == 0.0 and choice(st3) == choice(st)
    assert np.array_equal(fixed_map(h3), fixed)
    mm.destroy(h3)

    # nothing left 0: nothing to tune, the cache is not touched
    h4 = make(m, pos, p, leaf_size=32, sub_levels=2, rows_per_item=64, autotune=True,
              tune_cache=str(tmp_path / "unused.jsonl"))
    assert mm.get_stats(h4)["autotuned"] == 0
    mm.destroy(h4)
    assert not (tmp_path / "unused.jsonl").exists()


def test_unusable_cache_lines_are_ignored(oracle_mod, tmp_path):
    m, pos, p = field(oracle_mod, seed=8)
    first = tmp_path / "a.jsonl"
    h = make(m, pos, p, autotune=True, tune_cache=str(first))
    mm.destroy(h)
    key = json.loads(first.read_text().splitlines()[0])["key"]
    bad = tmp_path / "b.jsonl"
    bad.write_text("not json at all\n"
                   '{"key": "%s", "leaf_size": 0, "sub_levels": 2, "rows_per_item": 0}\n'
                   '{"key": "%s", "leaf_size": 32}\n'
                   '{"key": "sm_00/other", "leaf_size": 32, "sub_levels": 2, '
                   '"rows_per_item": 0}\n' % (key, key))
    h = make(m, pos, p, autotune=True, tune_cache=str(bad))
    st = mm.get_stats(h)
    mm.destroy(h)
    assert st["autotuned"] == 1
    assert len(bad.read_text().splitlines()) == 5
    # a valid line for the key, after them, is taken
    bad.write_text(bad.read_text() +
                   '{"key": "%s", "leaf_size": 16, "sub_levels": 1, "rows_per_item": 64, '
                   '"ms_estimate": 1.0}\n' % key)
    h = make(m, pos, p, autotune=True, tune_cache=str(bad))
    st = mm.get_stats(h)
    mm.destroy(h)
    assert st["autotuned"] == 2 and choice(st) == (16, 1, 64)
    # (a line without jobs_per_mcell: one slot per 12 cells)
    assert st["queue_slots"] == default_queue(st["cells"], -1)


def test_autotuned_handles_batch_like_single_runs(oracle_mod, tmp_path):
    hs = []
    for seed in (9, 10, 11):
        m, pos, p = field(oracle_mod, seed)
        hs.append(make(m, pos, p, autotune=True, tune_cache=str(tmp_path / "t.jsonl")))
    mm.run_batch(hs, 0)
    batched = [mm.get_map_fixed(h) for h in hs]
    for h, b in zip(hs, batched):
        assert np.array_equal(fixed_map(h), b)
        mm.destroy(h)
