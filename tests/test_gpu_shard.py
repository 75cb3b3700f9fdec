"""One map over cell rectangles and bands (mm_run_cells, mm_normalize_fixed,
paper_2506_02114_gb300.shard) on one GPU, through the C ABI: rectangles
that partition a map's cells add up to its map bit for bit in every mode
and queue setting, and the sharded-map path -- each band's fixed-point map,
an integer sum, one normalisation -- gives mm_run's map bit for bit.  With
several devices the sum is an all-reduce (tests/test_multi_rank.py covers
that reduction on CPU ranks)."""
import math

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
from paper_2506_02114_gb300 import shard
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    mm.lib()
    return torch


def field(kappa=0.45, gamma=0.3, s=0.4, hl=1.5, npix=64, rpp=10.0):
    p0 = mm.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rpp, flux_fraction_f=0.01)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    m, pos = synthetic.star_field(31, synthetic.n_stars_for((1 - s) * kappa, R, synthetic.EQUAL),
                                  R)
    return (kappa, gamma, s, m, pos, hl, npix, rpp)


@pytest.mark.parametrize("opts", [
    dict(),                                               # FMM, default queue
    dict(big_queue_slots=64),                             # FMM, a queue run in segments
    dict(big_queue_slots=-1, sub_levels=-1),              # FMM, no queue, whole leaves
    dict(mode=mm.MM_PLAIN_FP64),                          # plain FP64
])
def test_cell_rectangles_partition_the_map(torch_cuda, opts):
    args = field()
    h = mm.create(*args, fmm_order=20, flux_fraction_f=0.01, **opts)
    mm.run(h, 0)
    full = mm.get_map_fixed(h)
    st = mm.get_stats(h)
    rows, cols = st["params"]["n"][1] - 1, st["params"]["n"][0] - 1
    rcut = [0, rows // 3 + 7, rows // 3 + 8, rows]          # a one-row band in the middle
    ccut = [0, 45, cols]                                    # not a multiple of 31
    tot = np.zeros_like(full)
    for a, b in zip(rcut[:-1], rcut[1:]):
        for c, d in zip(ccut[:-1], ccut[1:]):
            mm.run_cells(h, a, b, c, d, 0)
            part = mm.get_map_fixed(h)
            assert mm.get_stats(h)["error_bits"] == 0
            tot += part
    mm.destroy(h)
    assert full.sum() > 0 and np.array_equal(tot, full)


@pytest.mark.parametrize("world", [1, 3, 5])
def test_sharded_map_equals_single_run(torch_cuda, world):
    """The sharded path with `world` bands summed on one device (the sum an
    all-reduce performs across devices) and normalised once equals mm_run's
    map, fixed point and floats, bit for bit."""
    torch = torch_cuda
    args = field(npix=48, rpp=12.0)
    h = mm.create(*args, fmm_order=20, flux_fraction_f=0.01)
    mm.run(h, 0)
    ref_fixed = mm.get_map_fixed(h)
    ref = mm.get_map(h)
    dev = torch.device("cuda", torch.cuda.current_device())
    acc = torch.zeros(h.npix_y * h.npix, dtype=torch.int64, device=dev)
    for r in range(world):
        acc += shard.band_fixed(h, r, world)
    out = torch.empty(h.npix_y * h.npix, dtype=torch.float32, device=dev)
    mm.normalize_fixed(h, acc, out)
    torch.cuda.synchronize()
    assert np.array_equal(acc.cpu().numpy().view(np.uint64).reshape(ref_fixed.shape), ref_fixed)
    assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref)
    if world == 1:
        # the whole path as one call (no process group: the sum is the band)
        mu = shard.sharded_map(h, 0, 1)
        torch.cuda.synchronize()
        assert np.array_equal(mu.cpu().numpy().reshape(ref.shape), ref)
    mm.destroy(h)


def test_more_ranks_than_rows_gives_empty_bands(torch_cuda):
    torch = torch_cuda
    args = field(npix=16, rpp=1.0, hl=0.6)
    h = mm.create(*args, fmm_order=12, flux_fraction_f=0.01)
    rows = mm.get_stats(h)["params"]["n"][1] - 1
    mm.run(h, 0)
    ref_fixed = mm.get_map_fixed(h)
    world = rows + 3
    dev = torch.device("cuda", torch.cuda.current_device())
    acc = torch.zeros(h.npix_y * h.npix, dtype=torch.int64, device=dev)
    for r in range(world):
        acc += shard.band_fixed(h, r, world)
    torch.cuda.synchronize()
    assert np.array_equal(acc.cpu().numpy().view(np.uint64).reshape(ref_fixed.shape), ref_fixed)
    mm.destroy(h)


def test_run_cells_rejects_bad_rectangles(torch_cuda):
    args = field(npix=32)
    h = mm.create(*args, fmm_order=12, flux_fraction_f=0.01, row_begin=10, row_end=40)
    cols = mm.get_stats(h)["params"]["n"][0] - 1
    for r in [(5, 20, 0, cols), (10, 41, 0, cols), (20, 20, 0, cols), (10, 20, 0, cols + 1),
              (10, 20, 7, 7)]:
        with pytest.raises(mm.MMError) as e:
            mm.run_cells(h, *r)
        assert e.value.status == mm.MM_EINVAL
    mm.run_cells(h, 10, 40, 0, cols, 0)
    mm.destroy(h)
