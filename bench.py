"""Benchmark: rays/s of the FP32 FMM + IPM path on one magnification map.

Workload (synthetic, seeded): kappa = 0.5, gamma = 0.4, s = 0.5, Salpeter
masses 0.1-1 uniform in a disk of radius 212 (50 295 stars), 2000^2-pixel map
of half-width 10, 9 rays per pixel without lensing (~100 landing per pixel),
FMM order 25: a 12 803 x 115 219 ray grid (1.475e9 rays).

A step is one mm_run: Morton sort, quadtree, expansions, fused deflection +
inverse polygon mapping, normalisation, with the stars already on the device.
L2 is flushed (256 MiB write) before every timed step; steps are timed with
CUDA events on the stream they run on.  Multi-GPU (torchrun): every rank maps
its own replica of the workload (weak scaling, no collective on the data
path); value = rays of all ranks / the slowest rank's time.

Also reported: the plain FP64 direct-sum path on the same GPU (a band of grid
rows, rays/s), the end-to-end rate through the C ABI with host buffers, the
hot kernel's roofline, and the FP64 oracle on the host cores (cpu_baseline).
"""
import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

WORKLOAD = "fmm_fp32_salpeter_2000"
METRIC = "rays/s (FMM+IPM), FP32-batched vs FP64 plain, same GPU, at ≤1e-3 map error"
UNIT = "rays/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FMA lanes x 2 flops x max clock

# dram bytes per launch of k_shoot_ipm from one ncu capture (see profiles/),
# valid only for the kernel sources it was taken on (hash below)
NCU_TRAFFIC = {"sources_sha1": "ef45a235778aeee2d9ff0ac512bfa46407d5b75d",
               "bytes_per_launch": 68.97e6 + 3.36e9}


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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="--impl reference: oracle seconds per step (default: ~100 s "
                         "spread over the steps, 2 to 30 s each)")
    ap.add_argument("--no-one-core", action="store_true",
                    help="skip the one-core oracle run beside the all-core one")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named workload (the default is the one the metric is quoted on)")
    ap.add_argument("--rays-per-pixel", type=float, default=None,
                    help="override the workload's rays per pixel (smaller profiling cases)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the map steps only: no FP64 band, end-to-end or CPU legs")
    ap.add_argument("--irs", action="store_true",
                    help="inverse ray shooting (rays counted per pixel) instead of polygon "
                         "mapping, for the map steps; implies --kernel-only")
    ap.add_argument("--sweep", action="store_true",
                    help="the batched sweep: 128 maps (500^2-2000^2 px, ~100 rays landing per "
                         "pixel, 1e2-1e5 stars), each autotuned, run as one mm_run_batch")
    ap.add_argument("--autotune", action="store_true",
                    help="let mm_create choose leaf size, sub-cell levels and work-item rows "
                         "by timing (mm_options.autotune; no cache file)")
    a = ap.parse_args()
    if a.irs:
        a.kernel_only = True
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
# CPU oracle (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_rays_per_s(wl, m, pos, seconds, nthreads=None):
    """The FP64 oracle (direct sum + per-pixel clipping) on a band of cell rows
    of the same workload, sized to take ~`seconds`; returns (rays/s, info)."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    p = oracle.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, wl.npix,
                             rays_per_pixel=wl.rays_per_pixel)
    mid = (p.n[1] - 1) // 2
    t0 = time.perf_counter()
    oracle.magnification_map(p, m, pos, mid, mid + 1, nthreads=nthreads)
    t1 = time.perf_counter() - t0
    rows = int(max(1, min(256, round(seconds / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    oracle.magnification_map(p, m, pos, mid, mid + rows, nthreads=nthreads)
    dt = time.perf_counter() - t0
    rays = p.n[0] * (rows + 1)
    return rays / dt, {"cores": nthreads, "rows": rows, "rays": rays, "seconds": dt,
                       "sample": "%d cell rows x %d rays of the %s grid (full width, all %d stars)"
                                 % (rows, p.n[0], wl.name, len(m))}


def oracle_one_core(wl, m, pos):
    """The oracle on one host core over the smallest sample it takes (one
    cell row, full width): the per-core rate beside the all-core one."""
    import oracle
    p = oracle.derive_params(wl.kappa, wl.gamma, wl.s, m, wl.half_length, wl.npix,
                             rays_per_pixel=wl.rays_per_pixel)
    mid = (p.n[1] - 1) // 2
    t0 = time.perf_counter()
    oracle.magnification_map(p, m, pos, mid, mid + 1, nthreads=1)
    dt = time.perf_counter() - t0
    rays = 2 * p.n[0]
    return {"value": rays / dt, "unit": UNIT, "cores": 1, "pairs_per_s": rays * len(m) / dt,
            "sample": "1 cell row x %d rays (full width, all %d stars)" % (p.n[0], len(m))}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = synthetic.workload(WORKLOAD)
    m, pos = wl.stars()
    per_step = (args.ref_seconds if args.ref_seconds is not None
                else max(2.0, min(30.0, 100.0 / max(1, args.steps + args.warmup))))
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        v, info = oracle_rays_per_s(wl, m, pos, per_step)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * info["rays"] / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": info["sample"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                         "sample": info["sample"], "pairs_per_s": value * len(m)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


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
    mm.lib()

    wl = synthetic.workload(args.workload)
    if args.rays_per_pixel:
        wl = dataclasses.replace(wl, rays_per_pixel=args.rays_per_pixel)
    m, pos = wl.stars()
    args_map = (wl.kappa, wl.gamma, wl.s, m, pos, wl.half_length, wl.npix, wl.rays_per_pixel)
    stream = torch.cuda.Stream(device=dev)
    h = mm.create(*args_map, fmm_order=wl.fmm_order, time_stages=True, autotune=args.autotune,
                  mode=mm.MM_FMM_IRS if args.irs else mm.MM_FMM_FP32)
    st0 = mm.get_stats(h)
    # the end-to-end leg creates its handles with the settings chosen here
    tuned = (dict(leaf_size=st0["leaf_size"], sub_levels=st0["sub_levels"],
                  rows_per_item=st0["rows_per_item"]) if args.autotune else {})
    rays = st0["rays"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)   # evict L2 (untimed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mm.run(h, stream.cuda_stream)
            e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    events, shoot_ms, first_ms = [], [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e = step()
            events.append(e)
            stream.synchronize()
            s = mm.get_stats(h)
            shoot_ms.append(s["ms_shoot"])
            first_ms.append(s["ms_first_pass"])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in events]
    tot_ms = sum(ms)
    st = mm.get_stats(h)
    mu = mm.get_map(h)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_per_step = tot_ms / args.steps
    value = world * rays / (ms_per_step * 1e-3)

    fp64_plain, e2e = None, None
    if not args.kernel_only:
        # plain FP64 direct sum on the same GPU: a band of full-width rows of
        # at least ~1e6 rays, longer where that takes under ~1 s
        n0 = st["params"]["n"][0]
        pairs_per_s = 4e10
        band = int(max(2, min(st["params"]["n"][1] - 1,
                              max(math.ceil(1.05e6 / n0), pairs_per_s / (n0 * len(m))))))
        r0 = (st["params"]["n"][1] - 1) // 2 - band // 2
        hp = mm.create(*args_map, mode=mm.MM_PLAIN_FP64, time_stages=True, row_begin=r0,
                       row_end=r0 + band)
        mm.run(hp, stream.cuda_stream)  # warm-up
        stream.synchronize()
        mm.run(hp, stream.cuda_stream)
        sp = mm.get_stats(hp)
        mm.destroy(hp)
        plain_rays_s = sp["rays"] / (sp["ms_total"] * 1e-3)

        # end to end through the C ABI with host buffers: create (stars H2D),
        # run, map D2H, destroy
        m_pin = torch.from_numpy(np.ascontiguousarray(m)).pin_memory()
        pos_pin = torch.from_numpy(np.ascontiguousarray(pos)).pin_memory()
        out_pin = torch.empty((wl.npix, wl.npix), dtype=torch.float32).pin_memory()
        e2e_times, parts = [], []
        for k in range(2 + max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            he = mm.create(wl.kappa, wl.gamma, wl.s, m_pin.numpy(), pos_pin.numpy(), wl.half_length,
                           wl.npix, wl.rays_per_pixel, fmm_order=wl.fmm_order, **tuned)
            ta = time.perf_counter()
            mm.run(he, stream.cuda_stream)
            mm.get_map(he, out_pin.numpy())
            tb = time.perf_counter()
            mm.destroy(he)
            t1 = time.perf_counter()
            if k >= 2:
                e2e_times.append(t1 - t0)
                parts.append((ta - t0, tb - ta, t1 - tb))
        e2e_value = world * rays / float(np.mean(e2e_times))
        fp64_plain = {"value": plain_rays_s, "unit": UNIT, "rays": sp["rays"],
                      "sample": "%d cell rows, full width, same grid" % band,
                      "speedup_fmm_fp32": value / world / plain_rays_s}
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(m.nbytes + pos.nbytes),
               "d2h_bytes_per_step": int(wl.npix * wl.npix * 4),
               "includes": "mm_create (stars H2D, plan) + mm_run + mm_get_map (D2H) + mm_destroy",
               "ms_create_run_destroy": [round(1e3 * float(np.mean([p[q] for p in parts])), 3)
                                         for q in range(3)]}

    # roofline of the hot kernel, the fused deflection + first mapping pass
    # (FP32 ALU bound); the second pass deals the queued larger triangles
    p, pe = st["fmm_order"], st["eval_order"]
    # near field + local expansion (p_e terms about the sub-cell centre) + macro, then the
    # mapping: the polygon-mapping size test (~20) or the ray's pixel index (~4)
    flops_per_ray = (11.0 * st["mean_near_stars"] + 8.0 * (pe - 1) + 8.0
                     + (4.0 if args.irs else 20.0))
    shoot_s = float(np.mean(first_ms)) * 1e-3
    # vertices whose deflection culling proved unnecessary are not computed:
    # a culled warp row skips the 31 vertex columns of its work item
    computed = max(0, rays - 31 * st["rows_culled"])
    achieved = computed * flops_per_ray / shoot_s / 1e12
    # DRAM bytes of one full-size launch, taken by ncu for the polygon-mapping
    # kernel only; none recorded for the ray-counting kernel
    traffic = None
    if not args.irs and NCU_TRAFFIC["sources_sha1"] == kernel_sources_sha1():
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                "kernel": "k_shoot_irs" if args.irs else "k_shoot_ipm",
                "flops_per_ray": flops_per_ray,
                "rays_computed": computed,
                "kernel_ms": shoot_s * 1e3,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    clocks = clk.summary()
    if rank != 0:
        mm.destroy(h)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    cpu = None
    if not (args.no_cpu_baseline or args.kernel_only) and world == 1:
        v, info = oracle_rays_per_s(wl, m, pos, args.cpu_seconds)
        # a direct sum evaluates every star for every ray: pairs = rays x stars
        cpu = {"value": v, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
               "sample": info["sample"], "pairs_per_s": v * len(m)}
        # the one-core leg takes one full-width cell row; skipped where that
        # would take more than ~30 s at the all-core rate per core
        est_s = 2 * st["params"]["n"][0] / (v / info["cores"])
        if not args.no_one_core and est_s <= 30.0:
            cpu["one_core"] = oracle_one_core(wl, m, pos)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "kappa": wl.kappa, "gamma": wl.gamma, "s": wl.s,
                   "n_stars": len(m), "mass_function": wl.mass_fn.name, "npix": wl.npix,
                   "half_length": wl.half_length, "rays_per_pixel": wl.rays_per_pixel,
                   "ray_grid": st["params"]["n"], "rays": rays, "fmm_order": p,
                   "eval_order": pe, "sub_levels": st["sub_levels"],
                   "leaf_size": st["leaf_size"], "rows_per_item": st["rows_per_item"],
                   "autotuned": st["autotuned"], "mapping": "irs" if args.irs else "ipm",
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "step_ms": {"median": statistics.median(ms), "mean": float(np.mean(ms)),
                    "std": float(np.std(ms)), "min": min(ms), "max": max(ms)},
        "maps_per_s": world / (ms_per_step * 1e-3),
        "stages_ms": {k: st[k] for k in ("ms_tree", "ms_expansions", "ms_shoot", "ms_first_pass",
                                         "ms_second_pass", "ms_normalize", "ms_total")},
        "triangles": {k[len("triangles_"):]: st[k] for k in (
            "triangles_clipped", "triangles_line", "triangles_quad", "triangles_box",
            "triangles_rows", "triangles_dropped", "triangles_near_critical")},
        "fp64_plain": fp64_plain,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": st["kernel_launches"] * args.steps,
        "clocks": clocks,
        "map_mean": float(mu.mean()),
    }
    print(json.dumps(line), flush=True)
    mm.destroy(h)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


SWEEP_MAPS = 128


def sweep_maps(mm, n_maps):
    """The batched sweep's maps: (kappa, gamma, s, npix, half-length) as
    synthetic.batch_draws draws them, ~100 rays landing per pixel (rays per
    pixel without lensing 100 / |mu_macro|), Salpeter stars in a disk around
    the shooting region, 1e2 to 1e5 of them; draws whose stars do not span
    the ray grid are skipped."""
    out = []
    for d in synthetic.batch_draws(4000, 1 << 30):
        kappa, gamma, s = d["kappa"], d["gamma"], d["s"]
        rpp = 100.0 * abs((1 - kappa) ** 2 - gamma ** 2)
        p0 = mm.derive_params(kappa, gamma, s, np.ones(4), d["half_length"], d["npix"], rpp)
        R = 1.1 * math.hypot(p0.img_half[0], p0.img_half[1])
        n = synthetic.n_stars_for((1 - s) * kappa, R, synthetic.SALPETER_01_1)
        if n < 100 or n > 100000:
            continue
        m, pos = synthetic.star_field(d["seed"], n, R, synthetic.SALPETER_01_1)
        p = mm.derive_params(kappa, gamma, s, m, d["half_length"], d["npix"], rpp)
        if any(pos[:, k].min() > p.x0[k] or pos[:, k].max() < p.x0[k] + (p.n[k] - 1) * p.h[k]
               for k in (0, 1)):
            continue
        out.append((kappa, gamma, s, m, pos, d["half_length"], d["npix"], rpp))
        if len(out) == n_maps:
            return out
    return out


def run_sweep(args):
    """rays/s of the batched sweep: one mm_run_batch over all maps per step."""
    import tempfile
    import torch
    torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    import paper_2506_02114_gb300 as mm
    mm.lib()
    maps = sweep_maps(mm, SWEEP_MAPS)
    t0 = time.perf_counter()
    with tempfile.TemporaryDirectory() as tmp:
        cache = os.path.join(tmp, "tune.jsonl")
        # a 2^20-slot second-pass queue per map (48 MB); in a batch, batches
        # that do not fit are dealt by the first pass
        hs = [mm.create(*w, fmm_order=25, autotune=True, tune_cache=cache,
                        big_queue_slots=1 << 20) for w in maps]
    t_create = time.perf_counter() - t0
    sts = [mm.get_stats(h) for h in hs]
    rays = sum(st["rays"] for st in sts)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mm.run_batch(hs, stream.cuda_stream)
            e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    events = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            events.append(step())
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in events]
    ms_per_step = sum(ms) / len(ms)
    launches = sum(mm.get_stats(h)["kernel_launches"] for h in hs)
    for h in hs:
        mm.destroy(h)
    line = {
        "metric": METRIC, "value": rays / (ms_per_step * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "sweep_%d" % len(maps), "maps": len(maps), "rays": rays,
                   "npix": [min(w[6] for w in maps), max(w[6] for w in maps)],
                   "n_stars": [min(len(w[3]) for w in maps), max(len(w[3]) for w in maps)],
                   "fmm_order": 25, "autotune": "per map, one shared cache",
                   "leaf_size": sorted({st["leaf_size"] for st in sts}),
                   "sub_levels": sorted({st["sub_levels"] for st in sts}),
                   "rows_per_item": sorted({st["rows_per_item"] for st in sts}),
                   "l2": "flushed before every step (256 MiB write)", "parallelism": "single"},
        "maps_per_s": len(maps) / (ms_per_step * 1e-3),
        "s_create_and_autotune": t_create,
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
