"""mm_map_plain_fp64_noalloc: the plain FP64 map for callers that cannot
allocate device memory (their device memory belongs to their own pool
allocator, or they cannot accept the synchronisation a cudaMalloc may imply).

The entry point must give the same map as the allocating path
(mm_create(mode=MM_PLAIN_FP64) + mm_run + mm_get_map) on two calls in a row,
its scratch living in a fixed device array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
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


@pytest.mark.parametrize("s, center_y", [(0.0, (0.0, 0.0)), (0.4, (0.7, -0.3))])
def test_noalloc_matches_allocating_path_twice(torch_cuda, s, center_y):
    """Two calls in a row equal the allocating plain FP64 path: all mass in
    stars on a centred map, and a smooth fraction (the kappa_star sheet term)
    on an off-centre map."""
    torch = torch_cuda
    kappa, gamma, hl, npix = 0.4, 0.3, 4.0, 128
    m, pos = synthetic.star_field(77, 300, 14.0)
    opts = dict(img_half=(6.0, 9.0), ray_grid=(420, 600), center_y=center_y)
    h = mm.create(kappa, gamma, s, m, pos, hl, npix, mode=mm.MM_PLAIN_FP64, **opts)
    mm.run(h, 0)
    ref = mm.get_map(h).astype(np.float64)
    prm = mm.get_stats(h)["params"]
    mm.destroy(h)
    assert ref.sum() > 0

    dev = torch.device("cuda", torch.cuda.current_device())
    m_d = torch.tensor(m, dtype=torch.float64, device=dev)
    pos_d = torch.tensor(pos, dtype=torch.float64, device=dev)
    for call in range(2):
        out = torch.full((npix * npix,), -1.0, dtype=torch.float32, device=dev)
        mm.map_plain_fp64_noalloc(kappa, gamma, s, m_d, pos_d, hl, npix, prm["n"], prm["x0"],
                                  prm["h"], out, center_y=center_y,
                                  stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.view(npix, npix).cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9 * ref.max(),
                                   err_msg="call %d" % call)


def test_noalloc_rejects_host_pointers_before_any_work(torch_cuda):
    """Host memory passed where device buffers belong is refused with
    MM_EINVAL by the C entry point itself (no kernel sees it)."""
    import ctypes
    torch = torch_cuda
    L = mm.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    m_h = np.ones(4)
    pos_h = np.zeros(8)
    m_d = torch.ones(4, dtype=torch.float64, device=dev)
    pos_d = torch.zeros(8, dtype=torch.float64, device=dev)
    out_d = torch.zeros(64 * 64, dtype=torch.float32, device=dev)
    out_h = np.zeros(64 * 64, dtype=np.float32)
    rg = (ctypes.c_int64 * 2)(100, 100)
    org = (ctypes.c_double * 2)(-1.005, -1.005)   # no vertex on the stars at the origin
    hh = (ctypes.c_double * 2)(0.02, 0.02)
    vp = ctypes.c_void_p

    def call(masses, pos, out):
        return L.mm_map_plain_fp64_noalloc(0.4, 0.3, 0.0, 4, vp(masses), vp(pos), 4.0, 64,
                                           None, rg, ctypes.cast(org, ctypes.POINTER(ctypes.c_double)),
                                           ctypes.cast(hh, ctypes.POINTER(ctypes.c_double)),
                                           vp(out), vp(0))
    for args in [(m_h.ctypes.data, pos_d.data_ptr(), out_d.data_ptr()),
                 (m_d.data_ptr(), pos_h.ctypes.data, out_d.data_ptr()),
                 (m_d.data_ptr(), pos_d.data_ptr(), out_h.ctypes.data)]:
        assert call(*args) == mm.MM_EINVAL
        assert "device memory" in mm.last_error()
    assert call(m_d.data_ptr(), pos_d.data_ptr(), out_d.data_ptr()) == mm.MM_OK
    # and the binding refuses a CPU tensor before reaching the library
    with pytest.raises(ValueError):
        mm.map_plain_fp64_noalloc(0.4, 0.3, 0.0, torch.ones(4, dtype=torch.float64), pos_d, 4.0,
                                  64, (100, 100), (-1.0, -1.0), (0.02, 0.02), out_d)


def test_noalloc_rejects_sizes_beyond_its_limit(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", torch.cuda.current_device())
    m_d = torch.ones(4, dtype=torch.float64, device=dev)
    pos_d = torch.zeros(8, dtype=torch.float64, device=dev)
    out = torch.zeros(512 * 512, dtype=torch.float32, device=dev)
    with pytest.raises(mm.MMError) as e:
        mm.map_plain_fp64_noalloc(0.4, 0.3, 0.0, m_d, pos_d, 4.0, 512, (100, 100), (0.0, 0.0),
                                  (0.1, 0.1), out)
    assert e.value.status == mm.MM_EINVAL and "limit" in str(e.value)
    with pytest.raises(mm.MMError) as e:
        mm.map_plain_fp64_noalloc(0.4, 0.3, 0.0, m_d, pos_d, 4.0, 64, (1000, 1000), (0.0, 0.0),
                                  (0.1, 0.1), out)
    assert e.value.status == mm.MM_EINVAL and "limit" in str(e.value)
