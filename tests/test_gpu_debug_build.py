"""The MM_DEBUG build (every map and row-difference index checked on the
device before its atomic; an out-of-range access is skipped and sets bit 8
of the error word) on a spread of real cases: random fields with sub-cells,
ray counting, the plain FP64 path, a rectangular star region, a non-square
map and a batch.  No access may be out of range, and every map must equal
the normal build's bit for bit.  The debug library runs in a subprocess
(MM_DEBUG_BUILD=1), so each process loads one build."""
import hashlib
import inspect
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))
ERR_BOUNDS = 8


def _cases(oracle_mod):
    """(name, positional create args, keyword args) of every case."""
    from test_gpu_parity import _random_field, explicit_grid
    out = []
    for k in range(4):
        (kappa, gamma, s, hl, npix), m, pos, p = _random_field(oracle_mod, k)
        args = (kappa, gamma, s, m, pos, hl, npix)
        out.append(("field%d" % k, args, dict(fmm_order=25, **explicit_grid(p))))
        if k == 0:
            out.append(("irs", args, dict(fmm_order=25, mode=mm.MM_FMM_IRS, **explicit_grid(p))))
            out.append(("queue64", args, dict(fmm_order=25, big_queue_slots=64,
                                              **explicit_grid(p))))
    (kappa, gamma, s, hl, npix), m, pos, p = _random_field(oracle_mod, 6)
    out.append(("plain", (kappa, gamma, s, m, pos, hl, npix),
                dict(mode=mm.MM_PLAIN_FP64, **explicit_grid(p))))
    p0 = oracle_mod.derive_params(0.45, 0.3, 0.4, np.ones(4), 1.5, 64, rays_per_pixel=10.0,
                                  flux_fraction_f=0.01)
    rect = (1.1 * p0.img_half[0] + 1.0, 1.1 * p0.img_half[1] + 1.0)
    n = synthetic.n_stars_for_rect(0.6 * 0.45, rect, synthetic.EQUAL)
    m, pos = synthetic.star_field_rect(5, n, rect)
    out.append(("rect", (0.45, 0.3, 0.4, m, pos, 1.5, 64, 10.0),
                dict(fmm_order=25, flux_fraction_f=0.01, star_rect=rect)))
    p0 = oracle_mod.derive_params(0.45, 0.3, 0.4, np.ones(4), 1.0, 40, rays_per_pixel=12.0,
                                  flux_fraction_f=0.01, npix_y=72)
    R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
    m, pos = synthetic.star_field(17, synthetic.n_stars_for(0.6 * 0.45, R, synthetic.EQUAL), R)
    out.append(("nonsquare", (0.45, 0.3, 0.4, m, pos, 1.0, 40, 12.0),
                dict(fmm_order=25, flux_fraction_f=0.01, npix_y=72)))
    return out


def _covered(args, kw):
    """The stars' bounding box covers the ray grid: the explicit one, else
    the one the C library derives for these arguments (host only)."""
    kappa, gamma, s, m, pos, hl, npix = args[:7]
    if "img_half" in kw:
        lo = [kw["center_y"][a] - kw["img_half"][a] for a in (0, 1)]
        hi = [kw["center_y"][a] + kw["img_half"][a] for a in (0, 1)]
    else:
        opts = inspect.signature(mm.make_options).parameters
        p = mm.derive_params(kappa, gamma, s, m, hl, npix, args[7],
                             **{k: v for k, v in kw.items() if k in opts})
        lo = [p.x0[a] for a in (0, 1)]
        hi = [p.x0[a] + (p.n[a] - 1) * p.h[a] for a in (0, 1)]
    return all(pos[:, a].min() <= lo[a] and pos[:, a].max() >= hi[a] for a in (0, 1))


def _run_all(oracle_mod):
    """{case: (sha256 of the fixed-point map, error bits)} with the loaded build."""
    res = {}
    for name, args, kw in _cases(oracle_mod):
        h = mm.create(*args, **kw)
        mm.run(h, 0)
        fixed = mm.get_map_fixed(h)
        res[name] = (hashlib.sha256(fixed.tobytes()).hexdigest(), mm.get_stats(h)["error_bits"])
        mm.destroy(h)
    # a batch (FMM FP32 handles only) of three fields
    hs = [mm.create(*args, **kw) for name, args, kw in _cases(oracle_mod)
          if name in ("field0", "queue64", "field3")]
    mm.run_batch(hs, 0)
    for i, h in enumerate(hs):
        res["batch%d" % i] = (hashlib.sha256(mm.get_map_fixed(h).tobytes()).hexdigest(),
                              mm.get_stats(h)["error_bits"])
        mm.destroy(h)
    return res


def test_debug_cases_are_valid_inputs(oracle_mod):
    """Host only: every case's stars cover its ray grid, so mm_create accepts
    it and the GPU test exercises the kernels rather than the validation."""
    for name, args, kw in _cases(oracle_mod):
        assert _covered(args, kw), name


@pytest.mark.gpu
def test_debug_build_checks_every_map_index(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, MM_DEBUG_BUILD="1")
    code = ("import sys, json; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
            "import oracle, test_gpu_debug_build as t\n"
            "print(json.dumps(t._run_all(oracle)))\n" % (os.path.dirname(HERE), HERE))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-2000:]
    debug = json.loads(r.stdout.strip().splitlines()[-1])
    normal = _run_all(oracle_mod)
    assert set(debug) == set(normal)
    for name in normal:
        assert debug[name][1] & ERR_BOUNDS == 0, (name, debug[name][1])
        assert debug[name][0] == normal[name][0], name
