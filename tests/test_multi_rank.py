"""Multi-rank host logic on CPU (gloo, world size 2): sharding one map's cell
rows over ranks and summing the band maps, the integer all-reduce of the
fixed-point maps that paper_2506_02114_gb300.shard performs, and the
max-over-ranks step time that bench.py reports.  The band maps here come
from the FP64 oracle, so no GPU is needed; on GPUs the same bands come from
mm_run_cells (tests/test_gpu_shard.py runs that path on one device)."""
import os
import socket

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm


def test_shard_rows_partition():
    for n in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            bands = [mm.shard_rows(n, r, world) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == n
            for (a, b), (c, d) in zip(bands, bands[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in bands]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        mm.shard_rows(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    import synthetic
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    kappa, gamma, s = 0.45, 0.3, 0.4
    m, pos = synthetic.star_field(21, 60, 9.0, synthetic.EQUAL)
    p = oracle.derive_params(kappa, gamma, s, m, 1.5, 48, rays_per_pixel=6.0, flux_fraction_f=0.01)
    n_rows = p.n[1] - 1
    r0, r1 = mm.shard_rows(n_rows, rank, world)
    _, acc, st = oracle.magnification_map(p, m, pos, r0, r1, nthreads=2, return_acc=True)
    t = torch.from_numpy(acc.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    tri = torch.tensor([float(st["triangles"])], dtype=torch.float64)
    dist.all_reduce(tri, op=dist.ReduceOp.SUM)
    # the step time bench.py reports is the slowest rank's
    ms = torch.tensor([10.0 + 5.0 * rank], dtype=torch.float64)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(os.path.join(out_dir, "sum.npy"), t.numpy())
        np.save(os.path.join(out_dir, "meta.npy"), np.array([tri.item(), ms.item(), n_rows]))
    dist.barrier()
    dist.destroy_process_group()


def test_band_maps_sum_to_the_whole_map(tmp_path, oracle_mod):
    import torch.multiprocessing as tmp
    import synthetic
    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    summed = np.load(tmp_path / "sum.npy")
    tri, ms, n_rows = np.load(tmp_path / "meta.npy")
    m, pos = synthetic.star_field(21, 60, 9.0, synthetic.EQUAL)
    p = oracle_mod.derive_params(0.45, 0.3, 0.4, m, 1.5, 48, rays_per_pixel=6.0,
                                 flux_fraction_f=0.01)
    _, full, st = oracle_mod.magnification_map(p, m, pos, return_acc=True)
    assert tri == st["triangles"] == 2 * n_rows * (p.n[0] - 1)
    np.testing.assert_allclose(summed, full, rtol=1e-12, atol=1e-12)
    assert ms == 15.0


def _reduce_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2506_02114_gb300 import shard
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    acc = torch.from_numpy(_rank_u64(rank).view(np.int64).copy())
    shard.reduce_fixed(acc)
    if rank == 0:
        np.save(os.path.join(out_dir, "u64.npy"), acc.numpy().view(np.uint64))
    # a float tensor is refused: the maps travel as int64
    with pytest.raises(mm.MMError):
        shard.reduce_fixed(acc.double())
    dist.barrier()
    dist.destroy_process_group()


def _rank_u64(rank):
    """Rank's fixed-point map: u64 values across the whole range, including
    ones at and above 2^63 (negative as int64)."""
    rng = np.random.default_rng(100 + rank)
    a = rng.integers(0, 2 ** 63, 4096, dtype=np.uint64) * np.uint64(2)
    a[:8] = np.array([0, 1, 2 ** 32, 2 ** 63 - 1, 2 ** 63, 2 ** 64 - 1, 2 ** 62, 12345],
                     dtype=np.uint64)
    return a


def test_fixed_point_maps_sum_exactly_over_ranks(tmp_path):
    """shard.reduce_fixed on two gloo ranks: the int64 all-reduce of u64 bits
    equals the u64 sum modulo 2^64 exactly (what makes a sharded map
    bit-identical to one device's)."""
    import torch.multiprocessing as tmp
    world = 2
    tmp.spawn(_reduce_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "u64.npy")
    with np.errstate(over="ignore"):
        want = _rank_u64(0) + _rank_u64(1)
    assert got.dtype == np.uint64 and np.array_equal(got, want)
