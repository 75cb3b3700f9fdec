"""One magnification map sharded over ranks by ray-grid row bands.

Every rank holds a handle of the same map (the same stars and parameters, so
the same plan) and maps only its contiguous band of cell rows
(``mm_run_cells``).  The bands' fixed-point accumulators (u64, 2^32 = one
triangle) are summed with one integer all-reduce -- integer addition is exact
and independent of the reduction's order, so the sum is bit-identical to a
single device's map -- and ``mm_normalize_fixed`` turns the sum into
magnification.  The paper names several GPUs as the remaining speed-up of its
method (Sec. 6); this is that split for one map.

The u64 accumulators travel as int64 tensors (the same 64 bits; a sum in
two's complement wraps exactly like an unsigned one).  torch.distributed is
the transport only; every step of the map runs in libmm's kernels.
"""
from . import (MM_EINVAL, MMError, get_map_fixed, get_stats, normalize_fixed, run_cells,
               shard_rows)


def band_fixed(h, rank, world, out=None):
    """Map this rank's band of cell rows on torch's current stream and return
    its fixed-point map as a CUDA int64 tensor of npix_y*npix elements (`out`
    if given), ready in stream order for the collective."""
    import torch
    st = get_stats(h)["params"]
    cols = int(st["n"][0]) - 1
    rows = int(st["n"][1]) - 1
    b, e = shard_rows(rows, rank, world)
    n = h.npix_y * h.npix
    if out is None:
        out = torch.empty(n, dtype=torch.int64,
                          device=torch.device("cuda", torch.cuda.current_device()))
    if e > b:
        run_cells(h, b, e, 0, cols)   # torch's current stream
        get_map_fixed(h, out)         # enqueued after it, on the same stream
    else:  # more ranks than rows: this rank's band is empty
        out.zero_()
    return out


def reduce_fixed(acc, group=None):
    """Sum the ranks' fixed-point maps in place (int64 all-reduce; exact)."""
    import torch
    import torch.distributed as dist
    if acc.dtype != torch.int64:
        raise MMError(MM_EINVAL, "fixed-point maps travel as int64 tensors")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc


def sharded_map(h, rank, world, group=None):
    """The whole map on every rank: this rank's band, the integer sum over
    ranks, then normalisation, all in order on torch's current stream.
    Returns a CUDA float32 tensor of npix_y*npix magnifications."""
    import torch
    acc = band_fixed(h, rank, world)
    reduce_fixed(acc, group)
    out = torch.empty(h.npix_y * h.npix, dtype=torch.float32, device=acc.device)
    normalize_fixed(h, acc, out)
    return out
