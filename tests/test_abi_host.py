"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/mm.h declares; host-side parameter derivation agrees with the
oracle's independent derivation; invalid arguments are rejected; and with no
GPU the product path fails loudly instead of falling back."""
import os
import re

import numpy as np
import pytest

import paper_2506_02114_gb300 as mm
import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = mm.lib()
    names = declared_functions()
    assert set(names) == set(mm.EXPORTS)
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("case", [
    dict(kappa=0.5, gamma=0.4, s=0.5, npix=2000, hl=10.0, rpp=9.0),
    dict(kappa=0.8, gamma=0.25, s=0.0, npix=500, hl=10.0, rpp=2.25),
    dict(kappa=0.3, gamma=0.45, s=0.2, npix=50, hl=2.5, rpp=4.0, center_y=(1.5, -0.75)),
    dict(kappa=1.3, gamma=0.2, s=0.9, npix=64, hl=3.0, rpp=1.0),
    dict(kappa=0.4, gamma=0.3, s=0.0, npix=256, hl=4.0, img_half=(16 / 3, 16.0),
         ray_grid=(700, 2000)),
    dict(kappa=0.66717, gamma=0.33383, s=0.5, npix=1000, hl=50.0, rpp=1.0, npix_y=100),
    dict(kappa=0.45, gamma=0.3, s=0.4, npix=48, hl=1.5, rpp=4.0, npix_y=80,
         center_y=(0.4, -0.2)),
])
def test_derived_parameters_match_oracle(oracle_mod, case):
    m, _ = synthetic.star_field(9, 300, 10.0, synthetic.SALPETER_01_1)
    kw = {}
    for k in ("center_y", "img_half", "ray_grid", "npix_y"):
        if k in case:
            kw[k] = case[k]
    got = mm.derive_params(case["kappa"], case["gamma"], case["s"], m, case["hl"], case["npix"],
                           case.get("rpp", 0.0), **kw).as_dict()
    ref = oracle_mod.derive_params(case["kappa"], case["gamma"], case["s"], m, case["hl"],
                                   case["npix"], rays_per_pixel=case.get("rpp", 0.0),
                                   **kw).as_dict()
    for k in ("kappa_star", "a1", "a2", "mu_macro", "mean_m", "m2_over_m", "r_border",
              "delta", "img_center", "img_half", "h", "x0", "half_length_y"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-14, atol=1e-14, err_msg=k)
    assert list(got["n"]) == list(ref["n"])
    assert got["npix_y"] == ref["npix_y"] == case.get("npix_y", case["npix"])


def test_invalid_arguments_rejected():
    with pytest.raises(mm.MMError) as e:
        mm.derive_params(0.5, 0.5, 0.0, [1.0], 1.0, 8, 1.0)
    assert e.value.status == mm.MM_EINVAL and "critical" in str(e.value)
    for bad in [dict(s=1.5), dict(hl=0.0), dict(npix=0)]:
        args = dict(kappa=0.5, gamma=0.2, s=0.0, hl=1.0, npix=8)
        args.update(bad)
        with pytest.raises(mm.MMError) as e:
            mm.derive_params(args["kappa"], args["gamma"], args["s"], [1.0], args["hl"],
                             args["npix"], 1.0)
        assert e.value.status == mm.MM_EINVAL
    with pytest.raises(mm.MMError):
        mm.derive_params(0.5, 0.2, 0.0, [1.0, -1.0], 1.0, 8, 1.0)
    with pytest.raises(mm.MMError):   # kappa_star > 0 needs stars
        mm.derive_params(0.5, 0.2, 0.0, [], 1.0, 8, 1.0)


def test_create_rejects_bad_orders_before_touching_a_gpu():
    m, pos = synthetic.star_field(1, 50, 10.0)
    for fo, ls in [(-1, 0), (65, 0), (10, -2), (10, 2000)]:
        with pytest.raises(mm.MMError) as e:
            mm.create(0.3, 0.1, 0.0, m, pos, 1.0, 16, 1.0, fmm_order=fo, leaf_size=ls)
        assert e.value.status == mm.MM_EINVAL


def test_create_rejects_uncovered_region():
    m, pos = synthetic.star_field(1, 50, 2.0)   # far too small a disk
    with pytest.raises(mm.MMError) as e:
        mm.create(0.4, 0.1, 0.0, m, pos, 5.0, 16, 1.0)
    assert e.value.status == mm.MM_EINVAL and "cover" in str(e.value)


def test_create_rejects_grid_outside_the_star_disk():
    """A ray grid inside the stars' bounding box but with corners outside the
    disk they fill (radius max |z_i|): the circular sheet's interior form
    -kappa_star z (Sec. 3.1) would not hold there, so mm_create refuses it
    before touching a GPU.  A disk reaching past the corners is accepted as
    far as the host checks go."""
    kappa, gamma, s, hl, npix, rpp = 0.5, 0.05, 0.0, 3.0, 16, 1.0
    p = mm.derive_params(kappa, gamma, s, np.ones(4), hl, npix, rpp)
    X = abs(p.x0[0])
    Y = abs(p.x0[1])
    corner = np.hypot(X, Y)
    R = 1.02 * max(X, Y)
    assert R < 0.98 * corner        # the box is covered, the corners are not
    m, pos = synthetic.star_field(4, 4000, R)
    # the stars reach past the box on all four sides
    assert pos[:, 0].min() < -X and pos[:, 0].max() > X
    assert pos[:, 1].min() < -Y and pos[:, 1].max() > Y
    p = mm.derive_params(kappa, gamma, s, m, hl, npix, rpp)
    assert np.hypot(pos[:, 0], pos[:, 1]).max() < np.hypot(abs(p.x0[0]), abs(p.x0[1]))
    with pytest.raises(mm.MMError) as e:
        mm.create(kappa, gamma, s, m, pos, hl, npix, rpp)
    assert e.value.status == mm.MM_EINVAL and "star disk" in str(e.value)
    # the same grid under a disk wide enough passes the host checks (with no
    # GPU the call then fails at the device, not at validation)
    m2, pos2 = synthetic.star_field(4, 4000, 1.05 * corner)
    try:
        mm.create(kappa, gamma, s, m2, pos2, hl, npix, rpp)
    except mm.MMError as e2:
        assert e2.status in (mm.MM_ECUDA, mm.MM_ENOMEM), str(e2)


def test_no_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m, pos = synthetic.star_field(1, 60, 12.0)
    with pytest.raises(mm.MMError) as e:
        mm.create(0.3, 0.1, 0.0, m, pos, 1.0, 16, img_half=(2.0, 2.0), ray_grid=(8, 8))
    assert e.value.status in (mm.MM_ECUDA, mm.MM_ENOMEM)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of mm_options, mm_params and mm_stats have the C
    structs' size and every field's offset (gcc compiles a probe of mm.h)."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"mm_options": mm.Options, "mm_params": mm.Params, "mm_stats": mm.Stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mm.h"', "int main(void) {"]
    want = []
    for cname, cls in structs.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            want.append(getattr(cls, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_autotune_options_reach_the_structure():
    o = mm.make_options(autotune=True, tune_cache="tune.jsonl")
    assert o.autotune == 1 and o.tune_cache == b"tune.jsonl"
    o = mm.make_options()
    assert o.autotune == 0 and o.tune_cache is None


def test_create_rejects_a_bad_star_rectangle():
    """star_rect must hold two positive half-widths enclosing the shooting
    region (checked before any GPU call)."""
    m, pos = synthetic.star_field_rect(3, 200, (30.0, 30.0))
    for rect in ((-1.0, 30.0), (30.0, 0.5), (float("nan"), 30.0)):
        with pytest.raises(mm.MMError) as e:
            mm.create(0.3, 0.1, 0.0, m, pos, 1.0, 16, 1.0, star_rect=rect)
        assert e.value.status == mm.MM_EINVAL


def test_debug_variant_builds_and_exports_every_symbol():
    """The MM_DEBUG build (bounds-checked map atomics) compiles for sm_103a
    into its own directory and exports the same C ABI."""
    import ctypes
    from paper_2506_02114_gb300 import build as B
    path = B.build(debug=True)
    assert path == B.LIB_DEBUG and path != B.LIB
    L = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(L, n), n


def test_binding_rejects_output_buffers_of_the_wrong_shape():
    """The binding checks caller buffers before the C library writes into
    them: size, dtype, contiguity, writeability and device."""
    import torch
    h = mm.Handle(None, 4, 3)
    for bad in (np.empty(11, np.float32), np.empty(12, np.float64),
                np.empty((3, 8), np.float32)[:, ::2], torch.empty(13, dtype=torch.float32)):
        with pytest.raises(ValueError):
            mm.get_map(h, bad)
    ro = np.empty((3, 4), np.float32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        mm.get_map(h, ro)
    h.ptr = None
    cpu = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="masses_dev"):
        mm.map_plain_fp64_noalloc(0.4, 0.3, 0.0, cpu, torch.zeros(8, dtype=torch.float64), 4.0,
                                  16, (8, 8), (-1.0, -1.0), (0.25, 0.25),
                                  torch.zeros(256, dtype=torch.float32))


def test_non_finite_inputs_rejected_before_touching_a_gpu():
    """Injected faults on the host: a NaN or infinite star position or mass,
    a zero mass, and non-finite lens parameters each return MM_EINVAL from
    mm_create's validation, before any device work."""
    m, pos = synthetic.star_field(1, 60, 12.0)
    cases = []
    for i, v in ((0, float("nan")), (7, float("inf")), (59, -float("inf"))):
        p = pos.copy()
        p[i, i % 2] = v
        cases.append((m, p, 0.3))
    for v in (float("nan"), float("inf"), 0.0):
        mm_ = m.copy()
        mm_[3] = v
        cases.append((mm_, pos, 0.3))
    cases.append((m, pos, float("nan")))
    for masses, positions, kappa in cases:
        with pytest.raises(mm.MMError) as e:
            mm.create(kappa, 0.1, 0.0, masses, positions, 1.0, 16, img_half=(2.0, 2.0),
                      ray_grid=(8, 8))
        assert e.value.status == mm.MM_EINVAL, str(e.value)
