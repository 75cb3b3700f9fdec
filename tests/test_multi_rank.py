"""Multi-rank host logic on CPU (gloo, world size 2): sharding one map's cell
rows over ranks and summing the band maps, and the max-over-ranks step time
that bench.py reports.  The band maps come from the FP64 oracle, so no GPU
is needed; on GPUs the same bands come from mm_run with row_begin/row_end."""
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
