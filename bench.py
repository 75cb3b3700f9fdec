"""Benchmark: rays/s of the FP32 FMM + IPM path, batched, on GB300.

Default workload (the one the metric is quoted on), ``sweep_128``: 128 maps
drawn like the batched sweep -- kappa in U[0.2, 0.9], gamma in U[0.1, 0.8]
(rejecting ||1 - kappa| - gamma| < 0.05), s in {0, 0.3, 0.6, 0.9}, npix in
U{500..2000}, half-length in U[5, 20], ~100 rays landing per pixel (rays per
pixel without lensing 100 / |mu_macro|), Salpeter 0.1-1 stars in a disk of
1.1 x the shooting region's half-diagonal, 1e2 to 1e5 stars per map -- FMM
order 25, each map's leaf size, sub-cell levels and rows per work item chosen
by the library's autotuner (answered from its tune cache when the cache
holds the map's key), all 128 run as one mm_run_batch per step: trees and
expansions per map, then one persistent deflection + polygon-mapping launch
over every map, second passes and normalisation.

Inputs are on the device before the timed region; L2 is flushed (256 MiB
write) before every timed step; steps are timed with CUDA events on the
stream they run on, max over ranks.  Multi-GPU (torchrun): every rank maps
its own replica of the workload (weak scaling, no collective on the data
path); value = rays of all ranks / the slowest rank's time.  With
``--shard one-map`` and a single-map workload the ranks split one map by
ray-grid row bands and sum the fixed-point maps with one integer all-reduce
(strong scaling).

Also reported: the plain FP64 direct-sum path on the same GPU (pairs/s on
row bands of the workload's maps, as rays/s of the whole workload), the map
error of the timed FP32 path against that FP64 path on the same bands, the
end-to-end rate through the C ABI with host buffers (create + run + map
read-back + destroy per step), the hot kernel's roofline against peaks
measured in the same run, the other workloads' single-map rates
(``workloads``), and the FP64 oracle on the host cores (``cpu_baseline``).
"""
import argparse
import dataclasses
import hashlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

SWEEP = "sweep_128"
SWEEP_MAPS = 128
SWEEP_ORDER = 25
SINGLE = ("fmm_fp32_salpeter_2000", "near_critical_5000", "large_kroupa_10000",
          "extreme_mu_10000x1000")
METRIC = "rays/s (FMM+IPM), FP32-batched vs FP64 plain, same GPU, at ≤1e-3 map error"
UNIT = "rays/s"
MAP_P999_TOL, MEAN_TOL = 1e-3, 1e-5
# autotuner choices made on GB300 by this library (JSON lines, mm_options.tune_cache)
TUNE_CACHE = os.path.join(ROOT, "paper_2506_02114_gb300", "tune", "sm_103.jsonl")

# Counters of one ncu capture of the hot kernels on the reduced profiling case
# (profiles/counters_fmm_fp32_salpeter_2000_rpp1.md): valid only for the kernel
# sources they were taken on (hash below), reported beside the live roofline.
NCU_COUNTERS = {
    "sources_sha1": "5517307e56512defd1c015340608c52b0e4ab670",
    "case": "fmm_fp32_salpeter_2000 at 1 ray per pixel (1.64e8 rays), ncu --clock-control none",
    "k_shoot_ipm": {"issue_active": 0.633, "warps_active": 0.194, "alu_active": 0.505,
                    "fma_active": 0.191, "l2_red_requests_per_s": 4.10e10},
    "k_big_ipm": {"issue_active": 0.803, "warps_active": 0.548, "alu_active": 0.630,
                  "fma_active": 0.299, "l2_red_requests_per_s": 9.63e10},
    "k_direct64_vertices": {"fp64_pipe_active": 0.907},
}


def kernel_sources_sha1():
    h = hashlib.sha1()
    for f in ("shoot.cu", "ipm.cuh", "mm_common.cuh"):
        with open(os.path.join(ROOT, "paper_2506_02114_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=SWEEP, choices=(SWEEP,) + SINGLE,
                    help="the batched sweep (default, the metric's configuration) or one "
                         "single-map workload")
    ap.add_argument("--shard", default="none", choices=["none", "one-map"],
                    help="one-map: ranks split one single-map workload by row bands")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="--impl reference: oracle seconds per step (default: ~100 s "
                         "spread over the steps, 2 to 30 s each)")
    ap.add_argument("--no-one-core", action="store_true",
                    help="skip the one-core oracle run beside the all-core one")
    ap.add_argument("--rays-per-pixel", type=float, default=None,
                    help="override a single-map workload's rays per pixel (profiling cases)")
    ap.add_argument("--rows", type=int, default=0,
                    help="single-map workloads: map only a band of this many cell rows "
                         "through the grid's middle, with the whole grid's plan (profiling "
                         "cases at the workload's own ray density)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the map steps only: no FP64, end-to-end, other-workload or "
                         "CPU legs")
    ap.add_argument("--irs", action="store_true",
                    help="single-map workloads: inverse ray shooting instead of polygon "
                         "mapping; implies --kernel-only")
    ap.add_argument("--autotune", action="store_true",
                    help="single-map workloads: let mm_create tune leaf size, sub-cell levels "
                         "and work-item rows (no cache)")
    ap.add_argument("--retune", action="store_true",
                    help="sweep: ignore the shipped tune cache, tune every key and write the "
                         "new cache to --tune-out")
    ap.add_argument("--tune-out", default="tune_sm_103.jsonl",
                    help="--retune: file the new tune cache is written to")
    a = ap.parse_args()
    if a.irs:
        a.kernel_only = True
    if a.irs and a.workload == SWEEP:
        ap.error("--irs needs a single-map workload")
    if a.shard == "one-map" and a.workload == SWEEP:
        ap.error("--shard one-map needs a single-map workload")
    if a.rows and (a.workload == SWEEP or a.shard != "none"):
        ap.error("--rows needs a single-map workload without --shard")
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class MapSpec:
    kappa: float
    gamma: float
    s: float
    m: np.ndarray
    pos: np.ndarray
    half_length: float
    npix: int
    rays_per_pixel: float
    fmm_order: int
    npix_y: int = 0     # rows of square pixels (0: a square map)

    def args(self):
        return (self.kappa, self.gamma, self.s, self.m, self.pos, self.half_length, self.npix,
                self.rays_per_pixel)


def grid_in_star_disk(p, pos):
    """The stars span the ray grid's box and fill a disk (radius max |z_i|)
    reaching its corners (what mm_create requires of a star disk)."""
    lo = [p.x0[k] for k in (0, 1)]
    hi = [p.x0[k] + (p.n[k] - 1) * p.h[k] for k in (0, 1)]
    if any(pos[:, k].min() > lo[k] or pos[:, k].max() < hi[k] for k in (0, 1)):
        return False
    r = float(np.sqrt((pos * pos).sum(axis=1)).max())
    return max(math.hypot(x, y) for x in (lo[0], hi[0]) for y in (lo[1], hi[1])) <= r


def derive(mod, kappa, gamma, s, m, hl, npix, rpp, npix_y=0):
    """Derived run parameters from the library (mod = the package) or, on
    the CPU-only reference arm, from the oracle (mod = oracle); the two
    derivations agree exactly (tests/test_abi_host.py)."""
    if mod.__name__ == "oracle":
        return mod.derive_params(kappa, gamma, s, m, hl, npix, rays_per_pixel=rpp, npix_y=npix_y)
    return mod.derive_params(kappa, gamma, s, m, hl, npix, rpp, npix_y=npix_y)


def sweep_maps(mod, n_maps):
    """The batched sweep's maps: (kappa, gamma, s, npix, half-length) as
    synthetic.batch_draws draws them, ~100 rays landing per pixel, Salpeter
    stars in a disk around the shooting region, 1e2 to 1e5 of them; draws
    whose stars do not cover the ray grid are skipped."""
    out = []
    for d in synthetic.batch_draws(4000, 1 << 30):
        kappa, gamma, s = d["kappa"], d["gamma"], d["s"]
        rpp = 100.0 * abs((1 - kappa) ** 2 - gamma ** 2)
        p0 = derive(mod, kappa, gamma, s, np.ones(4), d["half_length"], d["npix"], rpp)
        R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
        n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.SALPETER_01_1)
        if n < 100 or n > 100000:
            continue
        m, pos = synthetic.star_field(d["seed"], n, R, synthetic.SALPETER_01_1)
        p = derive(mod, kappa, gamma, s, m, d["half_length"], d["npix"], rpp)
        if not grid_in_star_disk(p, pos):
            continue
        out.append(MapSpec(kappa, gamma, s, m, pos, d["half_length"], d["npix"], rpp,
                           SWEEP_ORDER))
        if len(out) == n_maps:
            return out
    return out


def single_spec(name, rays_per_pixel=None):
    wl = synthetic.workload(name)
    if rays_per_pixel:
        wl = dataclasses.replace(wl, rays_per_pixel=rays_per_pixel)
    m, pos = wl.stars()
    return MapSpec(wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, wl.rays_per_pixel,
                   wl.fmm_order, wl.npix_y), wl


def workload_specs(mod, name, rays_per_pixel=None):
    if name == SWEEP:
        return sweep_maps(mod, SWEEP_MAPS)
    return [single_spec(name, rays_per_pixel)[0]]


def median_spec(specs):
    """The map of median star count (the CPU legs' sample)."""
    order = sorted(range(len(specs)), key=lambda i: len(specs[i].m))
    return specs[order[len(order) // 2]]


def pairs_per_ray(specs, rays):
    """Star-ray pairs per ray of the whole workload (a direct sum evaluates
    every star for every ray)."""
    return sum(r * len(sp.m) for sp, r in zip(specs, rays)) / max(1, sum(rays))


def spec_rays(mod, sp):
    p = derive(mod, sp.kappa, sp.gamma, sp.s, sp.m, sp.half_length, sp.npix, sp.rays_per_pixel,
               sp.npix_y)
    return int(p.n[0]) * int(p.n[1])


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_pairs_per_s(sp, label, seconds, nthreads=None):
    """The FP64 oracle (direct sum + per-pixel clipping) on a band of
    full-width cell rows of map `sp`, sized to take ~`seconds`: its
    star-ray pairs per second, and what the sample was."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    p = oracle.derive_params(sp.kappa, sp.gamma, sp.s, sp.m, sp.half_length, sp.npix,
                             rays_per_pixel=sp.rays_per_pixel, npix_y=sp.npix_y)
    mid = (p.n[1] - 1) // 2
    t0 = time.perf_counter()
    oracle.magnification_map(p, sp.m, sp.pos, mid, mid + 1, nthreads=nthreads)
    t1 = time.perf_counter() - t0
    rows = int(max(1, min(256, round(seconds / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    oracle.magnification_map(p, sp.m, sp.pos, mid, mid + rows, nthreads=nthreads)
    dt = time.perf_counter() - t0
    rays = p.n[0] * (rows + 1)
    return rays * len(sp.m) / dt, {
        "cores": nthreads, "seconds": dt, "rays": rays,
        "sample": "%d cell rows x %d rays of %s (full width, all %d stars)"
                  % (rows, p.n[0], label, len(sp.m))}


def oracle_one_core(sp, label):
    """The oracle on one host core over one full-width cell row of `sp`."""
    import oracle
    p = oracle.derive_params(sp.kappa, sp.gamma, sp.s, sp.m, sp.half_length, sp.npix,
                             rays_per_pixel=sp.rays_per_pixel, npix_y=sp.npix_y)
    mid = (p.n[1] - 1) // 2
    t0 = time.perf_counter()
    oracle.magnification_map(p, sp.m, sp.pos, mid, mid + 1, nthreads=1)
    dt = time.perf_counter() - t0
    rays = 2 * p.n[0]
    return {"pairs_per_s": rays * len(sp.m) / dt, "cores": 1,
            "sample": "1 cell row x %d rays of %s (full width, all %d stars)"
                      % (p.n[0], label, len(sp.m))}


def cpu_leg(specs, name, seconds, one_core=True):
    """The oracle's rate on the workload: pairs/s on a band of its median
    map, as rays/s of the whole workload (its pairs per ray)."""
    sp = median_spec(specs)
    label = name if len(specs) == 1 else "the median-star map of %s" % name
    pps, info = oracle_pairs_per_s(sp, label, seconds)
    import oracle
    ppr = pairs_per_ray(specs, [spec_rays(oracle, x) for x in specs])
    out = {"value": pps / ppr, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
           "sample": info["sample"] + "; rays/s = pairs/s / the workload's %.4g pairs per ray"
                     % ppr,
           "pairs_per_s": pps}
    if one_core:
        # one full-width cell row; skipped where that would take over ~30 s
        import oracle
        p = oracle.derive_params(sp.kappa, sp.gamma, sp.s, sp.m, sp.half_length, sp.npix,
                                 rays_per_pixel=sp.rays_per_pixel, npix_y=sp.npix_y)
        est_s = 2 * p.n[0] * len(sp.m) / (pps / info["cores"])
        if est_s <= 30.0:
            oc = oracle_one_core(sp, label)
            oc["value"] = oc["pairs_per_s"] / ppr
            oc["unit"] = UNIT
            out["one_core"] = oc
    return out, info


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle   # the reference arm runs nothing of the library
    specs = workload_specs(oracle, args.workload, args.rays_per_pixel)
    ppr = pairs_per_ray(specs, [spec_rays(oracle, x) for x in specs])
    per_step = (args.ref_seconds if args.ref_seconds is not None
                else max(2.0, min(30.0, 100.0 / max(1, args.steps + args.warmup))))
    vals = []
    info = None
    sp = median_spec(specs)
    label = args.workload if len(specs) == 1 else "the median-star map of %s" % args.workload
    for k in range(args.warmup + args.steps):
        pps, info = oracle_pairs_per_s(sp, label, per_step)
        if k >= args.warmup:
            vals.append(pps / ppr)
    value = float(np.mean(vals))
    sample = info["sample"] + "; rays/s = pairs/s / the workload's %.4g pairs per ray" % ppr
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * info["seconds"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "maps": len(specs), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                         "sample": sample, "pairs_per_s": value * ppr},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# native path: pieces
# ---------------------------------------------------------------------------

def measure_peaks(mm, local):
    """FP32 / FP64 FMA and L2 u64-reduction peaks of this GPU, measured now
    (mm_measure_peak), with the clocks seen while they ran."""
    out = {}
    with ClockSampler(local) as clk:
        for kind, key in ((mm.MM_PEAK_FP32_FMA, "fp32_tflops"),
                          (mm.MM_PEAK_FP64_FMA, "fp64_tflops"),
                          (mm.MM_PEAK_L2_RED_U64, "l2_red_gops"),
                          (mm.MM_PEAK_L2_RED_U64_ROWS, "l2_red_rows_gops")):
            v, ms = mm.measure_peak(kind)
            out[key] = v
            out[key + "_ms"] = ms
    out["clocks"] = clk.summary()
    return out


def make_tune_cache(args):
    """A private copy of the shipped tune cache (appends stay out of the
    repository); with --retune, an empty one."""
    fd, path = tempfile.mkstemp(prefix="mm_tune_", suffix=".jsonl")
    os.close(fd)
    if not args.retune and os.path.exists(TUNE_CACHE):
        shutil.copyfile(TUNE_CACHE, path)
    return path


def create_handles(mm, specs, name, args, tune_cache, **extra):
    if name == SWEEP:
        # each map's second-pass queue holds the larger triangles its tune
        # record counted, plus a quarter (the library's default); in a
        # batch, batches that do not fit are dealt by the first pass
        return [mm.create(*sp.args(), fmm_order=sp.fmm_order, autotune=True,
                          tune_cache=tune_cache, **extra)
                for sp in specs]
    sp = specs[0]
    return [mm.create(*sp.args(), fmm_order=sp.fmm_order, autotune=args.autotune,
                      mode=mm.MM_FMM_IRS if args.irs else mm.MM_FMM_FP32, npix_y=sp.npix_y,
                      **extra)]


def flops_per_ray(st, irs=False):
    """Algorithmic FP32 flops per computed ray: 11 per direct star, 8 per
    complex term of the re-centred local expansion, 8 for the macro term and
    sheet, and the mapping's classification of the ray's two triangles
    (~20; a ray count ~4 for IRS)."""
    return (11.0 * st["mean_near_stars"] + 8.0 * (st["eval_order"] - 1) + 8.0
            + (4.0 if irs else 20.0))


def rays_computed(st):
    # a culled warp row skips the 31 vertex columns of its work item
    return max(0, st["rays"] - 31 * st["rows_culled"])


def roofline(stats, first_ms, peaks, irs=False):
    """Roofline of the first-pass kernel (the fused deflection + mapping
    launch, k_shoot_ipm; k_shoot_irs with --irs) over the timed run."""
    computed = sum(rays_computed(st) for st in stats)
    flops = sum(rays_computed(st) * flops_per_ray(st, irs) for st in stats)
    s = first_ms * 1e-3
    achieved = flops / s / 1e12
    peak = peaks["fp32_tflops"]
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": None,
           "kernel": "k_shoot_irs" if irs else "k_shoot_ipm",
           "kernel_ms": first_ms, "rays_computed": computed,
           "flops_per_ray": flops / max(computed, 1),
           "peak_source": "measured now: mm_measure_peak FP32 FMA (8 fmaf chains per thread)"}
    if not irs and NCU_COUNTERS["sources_sha1"] == kernel_sources_sha1():
        # what bounds the kernel, from one ncu capture of the same sources on
        # the reduced profiling case: issue slots, not the FP32 pipe or atomics
        c = NCU_COUNTERS["k_shoot_ipm"]
        out["issue"] = {"issue_active_frac": c["issue_active"],
                        "warps_active_frac": c["warps_active"],
                        "alu_pipe_frac": c["alu_active"], "fma_pipe_frac": c["fma_active"],
                        "l2_red_frac_of_scattered_peak":
                            c["l2_red_requests_per_s"] / (peaks["l2_red_gops"] * 1e9),
                        "source": "ncu, " + NCU_COUNTERS["case"]}
    return out


def ipm_work(stats):
    """Mapping work of the timed run from the maps' statistics."""
    rays = sum(st["rays"] for st in stats)
    keys = ("triangles_clipped", "triangles_line", "triangles_quad", "triangles_box",
            "triangles_rows", "triangles_dropped", "triangles_near_critical")
    tot = {k[len("triangles_"):]: sum(st[k] for st in stats) for k in keys}
    tot["per_ray"] = {k: v / max(rays, 1) for k, v in tot.items()}
    return tot


def band_rows(st, n_stars, pairs_per_s=4e10, min_rays=1.05e6, max_rays=2e7):
    """A band of full-width cell rows through the grid's middle with at least
    ~1e6 rays, longer (up to 2e7 rays) where the plain FP64 path takes under
    ~1 s for it."""
    n0, n1 = st["params"]["n"]
    want = max(math.ceil(min_rays / n0), min(pairs_per_s / (n0 * max(n_stars, 1)),
                                             max_rays / n0))
    band = int(max(2, min(n1 - 1, want)))
    r0 = (n1 - 1) // 2 - band // 2
    return r0, r0 + band


def map_band_errors(mu, ref, mu_macro):
    """Band-map errors (pixels the band reaches only partly are measured
    against max(mu_ref, |mu_macro|))."""
    mu = np.asarray(mu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    pos = (ref > 0) | (mu > 0)
    if not pos.any():
        return 0.0, 0.0
    rel = np.abs(mu[pos] - ref[pos]) / np.maximum(ref[pos], abs(mu_macro))
    return float(np.quantile(rel, 0.999)), float(abs(mu.sum() - ref.sum()) / ref.sum())


def plain_and_error(mm, specs, hs, stats, stream, picks):
    """The plain FP64 path on row bands of the picked maps (same grids, same
    GPU): its pair rate, and the timed FP32 handles' maps of the same bands
    (mm_run_cells on the timed handle) against it."""
    rows, worst = [], [0.0, 0.0]
    pairs, secs = 0.0, 0.0
    for i in picks:
        sp, h, st = specs[i], hs[i], stats[i]
        r0, r1 = band_rows(st, len(sp.m))
        hp = mm.create(*sp.args(), mode=mm.MM_PLAIN_FP64, time_stages=True, row_begin=r0,
                       row_end=r1, npix_y=sp.npix_y)
        mm.run(hp, stream.cuda_stream)   # warm-up
        stream.synchronize()
        mm.run(hp, stream.cuda_stream)
        sp_st = mm.get_stats(hp)
        ref = mm.get_map(hp)
        mm.destroy(hp)
        n0 = st["params"]["n"][0]
        mm.run_cells(h, r0, r1, 0, n0 - 1, stream.cuda_stream)
        mu = mm.get_map(h)
        p999, mrel = map_band_errors(mu, ref, st["params"]["mu_macro"])
        worst = [max(worst[0], p999), max(worst[1], mrel)]
        pr = sp_st["rays"] * len(sp.m)
        pairs += pr
        secs += sp_st["ms_total"] * 1e-3
        rows.append({"map": i, "n_stars": len(sp.m), "rows": [r0, r1],
                     "rays": sp_st["rays"], "pairs_per_s": pr / (sp_st["ms_total"] * 1e-3),
                     "p999": p999, "mean_rel": mrel})
    return pairs / secs, rows, worst


def e2e_leg(mm, specs, name, args, tune_cache, stream, world, n_steps):
    """End to end through the C ABI with host buffers: per step, create
    every handle from pinned host star arrays (stars H2D, plan; tune choices
    from the cache), run, read every map back to pinned host memory and
    destroy the handles."""
    import torch
    pins = [(torch.from_numpy(np.ascontiguousarray(sp.m)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(sp.pos)).pin_memory()) for sp in specs]
    outs = [torch.empty((sp.npix_y or sp.npix, sp.npix), dtype=torch.float32).pin_memory()
            for sp in specs]
    from concurrent.futures import ThreadPoolExecutor
    times, parts = [], []
    # handles are created, read back and destroyed from 8 host threads (one
    # handle per thread at a time, as the ABI allows; ctypes releases the GIL)
    pool = ThreadPoolExecutor(max_workers=min(8, len(specs)))
    dev_index = torch.cuda.current_device()

    def create_on(d, sp):
        torch.cuda.set_device(d)   # mm_create uses the calling thread's device
        return create_handles(mm, [sp], name, args, tune_cache)[0]
    for k in range(2 + n_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = [dataclasses.replace(sp, m=mp.numpy(), pos=pp.numpy())
              for sp, (mp, pp) in zip(specs, pins)]
        hs = list(pool.map(lambda x: create_on(dev_index, x), s2))
        ta = time.perf_counter()
        if len(hs) > 1:
            mm.run_batch(hs, stream.cuda_stream)
        else:
            mm.run(hs[0], stream.cuda_stream)
        list(pool.map(lambda ho: mm.get_map(ho[0], ho[1].numpy()), zip(hs, outs)))
        tb = time.perf_counter()
        list(pool.map(mm.destroy, hs))
        t1 = time.perf_counter()
        if k >= 2:
            times.append(t1 - t0)
            parts.append((ta - t0, tb - ta, t1 - tb))
    pool.shutdown()
    return {"seconds": float(np.mean(times)),
            "h2d_bytes_per_step": int(sum(sp.m.nbytes + sp.pos.nbytes for sp in specs)),
            "d2h_bytes_per_step": int(sum(sp.npix * (sp.npix_y or sp.npix) * 4 for sp in specs)),
            "ms_create_run_destroy": [round(1e3 * float(np.mean([p[q] for p in parts])), 3)
                                      for q in range(3)]}


def single_rate(mm, name, stream, flush, n_steps=3):
    """Device-timed rays/s of one single-map workload (another config beside
    the headline): create, one warm-up run, n_steps timed runs."""
    import torch
    sp, wl = single_spec(name)
    h = mm.create(*sp.args(), fmm_order=sp.fmm_order, time_stages=True, npix_y=sp.npix_y)
    ms = []
    for k in range(1 + n_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mm.run(h, stream.cuda_stream)
            e1.record(stream)
        stream.synchronize()
        if k:
            ms.append(e0.elapsed_time(e1))
    st = mm.get_stats(h)
    mm.destroy(h)
    t = float(np.mean(ms))
    return {"value": st["rays"] / (t * 1e-3), "unit": UNIT, "ms_per_map": t,
            "rays": st["rays"], "rays_computed": rays_computed(st),
            "computed_rays_per_s": rays_computed(st) / (t * 1e-3), "steps": n_steps,
            "maps_per_s": 1e3 / t,
            "n_stars": len(sp.m), "npix": [sp.npix, sp.npix_y or sp.npix],
            "fmm_order": sp.fmm_order,
            "stages_ms": {k: st[k] for k in ("ms_tree", "ms_expansions", "ms_first_pass",
                                             "ms_second_pass", "ms_normalize")}}


# ---------------------------------------------------------------------------
# native path
# ---------------------------------------------------------------------------

def run_native(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2506_02114_gb300 as mm
    from paper_2506_02114_gb300 import shard
    mm.lib()

    peaks = measure_peaks(mm, local)
    name = args.workload
    specs = workload_specs(mm, name, args.rays_per_pixel)
    tune_cache = make_tune_cache(args)
    t0 = time.perf_counter()
    hs = create_handles(mm, specs, name, args, tune_cache, time_stages=True)
    s_create = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    sharded = args.shard == "one-map" and world > 1
    band = None
    if args.rows:
        n0, n1 = mm.get_stats(hs[0])["params"]["n"]
        r0 = max(0, (n1 - 1) // 2 - args.rows // 2)
        band = (r0, min(n1 - 1, r0 + args.rows), n0 - 1)

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)   # evict L2 (untimed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if sharded:
                shard.sharded_map(hs[0], rank, world)
            elif band:
                mm.run_cells(hs[0], band[0], band[1], 0, band[2], stream.cuda_stream)
            elif len(hs) > 1:
                mm.run_batch(hs, stream.cuda_stream)
            else:
                mm.run(hs[0], stream.cuda_stream)
            e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    events, first_ms = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            events.append(step())
            stream.synchronize()
            first_ms.append(mm.get_stats(hs[0])["ms_first_pass"])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in events]
    tot_ms = sum(ms)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_per_step = tot_ms / args.steps
    stats = [mm.get_stats(h) for h in hs]
    if band:   # the band's rays and cells (mm_get_stats counts the handle's)
        for st in stats:
            st["rays"] = (band[1] - band[0] + 1) * (band[2] + 1)
            st["cells"] = (band[1] - band[0]) * band[2]
    rays = sum(st["rays"] for st in stats)
    computed = sum(rays_computed(st) for st in stats)
    # replicas: every rank maps the whole workload; one sharded map: its rays once
    value = (1 if sharded else world) * rays / (ms_per_step * 1e-3)
    launches = sum(st["kernel_launches"] for st in stats)
    clocks = clk.summary()
    roof = roofline(stats, float(np.mean(first_ms)), peaks, args.irs)
    if rank != 0:
        for h in hs:
            mm.destroy(h)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    fp64_plain = e2e = workloads = map_error = cpu = None
    if not args.kernel_only:
        # plain FP64 on the same GPU: bands of the maps of smallest, median and
        # largest star count (the direct sum's pair rate does not depend on
        # the map), as rays/s of the whole workload; the timed handles' FP32
        # maps of the same bands against it
        order = sorted(range(len(specs)), key=lambda i: len(specs[i].m))
        picks = sorted({order[0], order[len(order) // 2], order[-1]})
        pps, bands, worst = plain_and_error(mm, specs, hs, stats, stream, picks)
        # the timed handles' device memory (the queues of a sweep hold ~100
        # GB) goes back to the pool before the end-to-end leg creates its own
        for h in hs:
            mm.destroy(h)
        hs = []
        ppr = pairs_per_ray(specs, [st["rays"] for st in stats])
        # the direct sum's inner loop issues 11 FP64 instructions per star-ray
        # pair (2 subtractions, a multiply and an FMA for |d|^2, the two
        # Newton-Raphson steps of the reciprocal (4 FMA), the mass multiply and
        # 2 FMA into the sum): its FP64-pipe load against the FMA-chain probe's
        # instruction rate (peak TFLOP/s / 2 flops per FMA)
        dp_rate = 11.0 * pps
        dp_peak = peaks["fp64_tflops"] * 1e12 / 2.0
        fp64_plain = {"value": pps / ppr, "unit": UNIT, "pairs_per_s": pps,
                      "pairs_per_ray": ppr, "bands": bands,
                      "speedup_fmm_fp32": value / world / (pps / ppr),
                      "fp64_pipe": {"dp_inst_per_pair": 11, "achieved_ginst_s": dp_rate / 1e9,
                                    "probe_ginst_s": dp_peak / 1e9, "frac": dp_rate / dp_peak}}
        map_error = {"p999": worst[0], "mean_rel": worst[1], "tol_p999": MAP_P999_TOL,
                     "tol_mean": MEAN_TOL,
                     "met": worst[0] <= MAP_P999_TOL and worst[1] <= MEAN_TOL,
                     "against": "plain FP64 direct sum + the same polygon mapping on the same "
                                "GPU, same grid bands (fp64_plain.bands)"}
        n_e2e = max(1, min(args.steps, 3))
        e = e2e_leg(mm, specs, name, args, tune_cache, stream, world, n_e2e)
        e2e = {"value": world * rays / e["seconds"], "unit": UNIT,
               "h2d_bytes_per_step": e["h2d_bytes_per_step"],
               "d2h_bytes_per_step": e["d2h_bytes_per_step"],
               "includes": "per map: mm_create (stars H2D from pinned host memory, plan, tune "
                           "choice from the cache) + one mm_run_batch (mm_run) + mm_get_map "
                           "(D2H to pinned host memory) + mm_destroy; creation, read-back and "
                           "destruction spread over 8 host threads",
               "steps": n_e2e, "ms_create_run_destroy": e["ms_create_run_destroy"]}
        if name == SWEEP and world == 1:
            workloads = {w: single_rate(mm, w, stream, flush) for w in SINGLE}
    for h in hs:
        mm.destroy(h)
    if not (args.no_cpu_baseline or args.kernel_only) and world == 1:
        cpu, _ = cpu_leg(specs, name, args.cpu_seconds, one_core=not args.no_one_core)
    if args.retune:
        out_dir = os.path.dirname(os.path.abspath(args.tune_out))
        os.makedirs(out_dir, exist_ok=True)
        shutil.copyfile(tune_cache, args.tune_out)
    os.unlink(tune_cache)

    tuned = [st["autotuned"] for st in stats]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": name, "maps": len(specs), "rays": rays,
                   "rays_computed": computed,
                   "npix": [min(sp.npix for sp in specs), max(sp.npix for sp in specs)],
                   "n_stars": [min(len(sp.m) for sp in specs), max(len(sp.m) for sp in specs)],
                   "fmm_order": sorted({st["fmm_order"] for st in stats}),
                   "eval_order": sorted({st["eval_order"] for st in stats}),
                   "leaf_size": sorted({st["leaf_size"] for st in stats}),
                   "sub_levels": sorted({st["sub_levels"] for st in stats}),
                   "rows_per_item": sorted({st["rows_per_item"] for st in stats}),
                   "tuned_from_cache": tuned.count(2), "tuned_by_timing": tuned.count(1),
                   "queue_gb": sum(st["queue_slots"] for st in stats) * 48 / 1e9,
                   "mapping": "irs" if args.irs else "ipm",
                   "band_rows": list(band[:2]) if band else None,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": ("one map, row bands over %d ranks + int64 all-reduce" % world
                                   if sharded else "replicas" if world > 1 else "single")},
        "step_ms": {"median": statistics.median(ms), "mean": float(np.mean(ms)),
                    "std": float(np.std(ms)), "min": min(ms), "max": max(ms)},
        "computed_rays_per_s": (1 if sharded else world) * computed / (ms_per_step * 1e-3),
        "maps_per_s": (1 if sharded else world) * len(specs) / (ms_per_step * 1e-3),
        "s_create": s_create,
        "stages_ms_lead": {k: stats[0][k] for k in ("ms_tree", "ms_expansions",
                                                    "ms_first_pass", "ms_second_pass",
                                                    "ms_normalize", "ms_total")},
        "ipm_work": ipm_work(stats),
        "map_error": map_error,
        "fp64_plain": fp64_plain,
        "roofline": roof,
        "peaks": peaks,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "workloads": workloads,
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
