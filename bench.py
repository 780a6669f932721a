"""Benchmark of the four-view matching stage (features, forward and inverse
fields, consistency/region filter, seeds) on one 1242x375 driving-shaped
quad per GPU.

Metric: matched pixels per second = W*H of the reference image L0 per step,
divided by the step time, summed over ranks (weak scaling: every rank matches
its own quad; no data-path collective).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sff|reference]

--impl reference times the CPU oracle (the plain C statement of the method)
on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen  # noqa: E402

WORKLOAD = "driving_1242x375"
SCENE_SEED = 2
MATCH_SEED = 2024
METRIC = "4-view matched px/s per GB300 (bit-exact), batched vs plain; serving p50/p99 ms"
L2_FLUSH_BYTES = 256 << 20
# Method parameters of both arms: the paper's k = 3 subscales, 12 iterations,
# tau_c = 1, s_c = 150 (Sec. 5) and the readings of the points it leaves open
PARAMS = dict(num_scales=4, iterations=12, tau_c=1, region_min=150, tau_r=1, quant_shift=4, knn_temporal=4,
              knn_epipolar=2)
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per unit of work of each kernel (units in `_units`):
#   k_iteration   per grid pixel and iteration (each pixel is updated once
#                 per iteration): own + written state 24 B, reference record
#                 48 B + norm 4 B, one 52 B target record per view = 232 B
#   k_features    per pixel and scale: packed smoothed pixel 4 B in, 48 B
#                 record + 4 B norm out
ALGO_BYTES = {"k_iteration": 24 + 52 + 3 * 52, "k_features": 8 + 52}
# Algorithmic integer work of the iteration kernel per grid pixel and
# iteration: 3 candidates (random search, 2 predecessors) x 3 views x one
# 48-element int8 dot product = 432 MACs = 108 dp4a.
ALGO_DP4A = {"k_iteration": 3 * 3 * 48 // 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sff", choices=["sff", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-quad batched and the serving measurements")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-paper-order", action="store_true",
                    help="skip the comparison with the paper's sequential propagation order")
    ap.add_argument("--no-interp", action="store_true", help="skip the dense interpolation measurement")
    ap.add_argument("--no-fill", action="store_true", help="skip the disparity fill (SGM) measurement")
    ap.add_argument("--no-sift", action="store_true", help="skip the SIFT-PCA cost measurement")
    ap.add_argument("--tuning-cache", default=None,
                    help="file of autotuned settings: read if present (no autotuning launches), written after "
                         "autotuning otherwise")
    ap.add_argument("--tuning", default="auto",
                    help="work distribution of the propagation kernels: 'auto' (autotune), L,TX,TY, or an "
                         "autotuner entry as JSON: {\"variants\": [4 x [lanes, slots, tile_x, tile_y, "
                         "min_ctas]], \"pair\": 0|1, \"alt\": bits, \"pdl\": bits, \"fuse\": bits}")
    ap.add_argument("--features-form", default="separable", choices=["separable", "tensor", "pairs"],
                    help="WHT features of the timed stage: separable butterflies through shared memory (the "
                         "default), the tensor-core form, or butterflies per pixel pair (identical features)")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="sff_tuning.overlap: the finer scales' features on a second stream while the K-NN "
                         "and the coarse scales match (1, the default) or every launch on one stream (0)")
    ap.add_argument("--tma", action="store_true",
                    help="scale 0 with TMA-staged reference records (sff_tuning.tma; the scale-0 variant must "
                         "have that form)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(scenegen.CONFIG_SIZES),
                    help="scene (profiling uses the small planes_256x80 case)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    return float(v["value"] if isinstance(v, dict) else v), "measured"
        except (ValueError, KeyError, TypeError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(kernel: str, launches_per_stage: float):
    """DRAM bytes per launch of `kernel`: its bytes per stage from
    profiles/dram_traffic.txt over its launches per stage, or None when missing
    or taken on a different version of the kernel's source."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p) or launches_per_stage <= 0:
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and f[0] == kernel and not line.startswith("#"):
            src = os.path.join(ROOT, "paper_1710_10096_gb300", "csrc", f[3])
            if os.path.exists(src) and hashlib.sha1(open(src, "rb").read()).hexdigest()[:12] == f[2]:
                return float(f[1]) / launches_per_stage
    return None


def _units(kernel: str, w: int, h: int, params) -> float:
    """Units of work of `kernel` in one step (summed over its launches)."""
    S, I = params.num_scales, params.iterations
    if kernel == "k_iteration":
        # 2 fields x per scale: I iterations, each updating every grid pixel once
        total = 0
        for s in range(S):
            n = 1 << s
            total += ((w + n - 1) // n) * ((h + n - 1) // n) * I
        return 2.0 * total
    if kernel == "k_features":
        return 4.0 * S * w * h
    return 0.0


def measured_peak_bf16():
    """Dense bf16 tensor peak (TFLOP/s) for a kernel timed alone: the burst
    figure of MEASURED_PEAKS.json, else the profiling fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if "bf16_tflops" in d:
                return float(d["bf16_tflops"]), "measured"
        except (ValueError, KeyError, TypeError):
            pass
    return 1900.0, "fallback"


def stage_rooflines(prof, steps, w, h, params, hbm_peak, bf16_peak, per_step_ms):
    """Roofline of every stage kernel of one quad step with its own bound and
    algorithmic work, and the stage's speed-of-light fraction: the sum over
    kernels of (work / peak) over the measured step time.  prof: {kernel:
    (launches, ms)} summed over `steps` steps.  Work per step (W x H = L0):
    - k_smooth: 4 images x (3 B read + 8 B x S scales written) per pixel;
    - k_features: 4 images x S scales x (8 B read + 48 B record + 4 B norm);
    - k_iteration: 232 B per grid pixel per iteration, both fields;
    - k_knn_tc: one pass of the coarsest grid's distance product, 2 fields x
      2 x gq^2 x 64 bf16 FLOP (the kernel makes two passes by design);
    - the consistency check (26 B per pixel, in k_cc_local) and the region
      filter (k_cc_*, 10 B per pixel; in the whole stage its last step, the
      removal of small joinable regions, runs inside k_block_best, and its
      bytes stay counted here); the seeds (k_block_best, k_write_seeds):
      16 B per pixel."""
    S = params.num_scales
    px = w * h
    nq = (1 << (S - 1))
    gq = ((w + nq - 1) // nq) * ((h + nq - 1) // nq)
    work = {"k_smooth": ("hbm", 4.0 * px * (3 + 8 * S)),
            "k_features": ("hbm", 4.0 * S * px * ALGO_BYTES["k_features"]),
            "k_features_tc": ("hbm", 4.0 * S * px * ALGO_BYTES["k_features"]),
            "k_features_sep": ("hbm", 4.0 * S * px * ALGO_BYTES["k_features"]),
            "k_iteration": ("hbm", ALGO_BYTES["k_iteration"] * _units("k_iteration", w, h, params)),
            "k_knn_tc": ("tensor", 2.0 * 2.0 * gq * gq * 64)}
    groups = {"consistency + region filter (k_cc_*)": (("k_cc_local", "k_cc_border", "k_cc_stats", "k_cc_remove"),
                                                       36.0 * px),
              "seeds (k_block_best, k_write_seeds)": (("k_block_best", "k_write_seeds"), 16.0 * px)}
    out, sol_ms = {}, 0.0
    for k, (bound, amount) in work.items():
        if k not in prof:
            continue
        ms = prof[k][1] / steps
        peak = hbm_peak * 1e9 if bound == "hbm" else bf16_peak * 1e12
        achieved = amount / (ms * 1e-3)
        out[k] = {"bound": bound, "ms_per_step": ms, "achieved": achieved / (1e9 if bound == "hbm" else 1e12),
                  "unit": "GB/s" if bound == "hbm" else "TFLOP/s", "frac": achieved / peak,
                  "work_per_step": amount}
        sol_ms += amount / peak * 1e3
    for name, (ks, amount) in groups.items():
        ms = sum(prof[k][1] for k in ks if k in prof) / steps
        if ms <= 0:
            continue
        out[name] = {"bound": "hbm", "ms_per_step": ms, "achieved": amount / (ms * 1e-3) / 1e9, "unit": "GB/s",
                     "frac": amount / (ms * 1e-3) / (hbm_peak * 1e9), "work_per_step": amount}
        sol_ms += amount / (hbm_peak * 1e9) * 1e3
    out["stage"] = {"speed_of_light_ms": sol_ms, "ms_per_step": per_step_ms, "frac": sol_ms / per_step_ms,
                    "what": "sum over the kernels above of work / peak, over the measured step time (kernels "
                            "without a work definition count as zero)"}
    return out


def merge_scales(prof):
    """Per-kernel totals {name: (launches, ms)} of a profile_collect(with_units=True)
    record, with the per-scale marks of a kernel ("name/s<scale>") summed under
    its name, and those per-scale entries separately: {name: {scale: (units, ms,
    launches)}}, units being iterations (a fused scale is one launch)."""
    merged, per_scale = {}, {}
    for name, (n, ms, units) in prof.items():
        base, sep, sc = name.partition("/s")
        if sep:
            per_scale.setdefault(base, {})[int(sc)] = (units, ms, n)
        a = merged.get(base, (0, 0.0))
        merged[base] = (a[0] + n, a[1] + ms)
    return merged, per_scale


def iteration_scales(per_scale, w, h, n_fields, peak, dp4a_peak=None):
    """Per-scale roofline of the propagation kernel: algorithmic bytes per
    iteration (ALGO_BYTES per grid pixel, every grid pixel of every field once
    per iteration) over the average time per iteration, and the same for its
    dp4a.  per_scale: {scale: (iterations, ms, launches)}; a scale whose
    iterations run as separate launches has one launch per iteration, a fused
    one a single launch."""
    out = []
    for s, (n, ms, launches) in sorted(per_scale.items()):
        st = 1 << s
        grid = ((w + st - 1) // st) * ((h + st - 1) // st)
        b = ALGO_BYTES["k_iteration"] * n_fields * grid
        us = 1e3 * ms / n
        r = {"scale": s, "grid_px": n_fields * grid, "iterations": n, "launches": launches,
             "avg_iteration_us": us, "algo_mb_per_iteration": b / 1e6, "achieved_gbs": b / (us * 1e-6) / 1e9,
             "frac": b / (us * 1e-6) / 1e9 / peak}
        if dp4a_peak:
            r["int_frac"] = ALGO_DP4A["k_iteration"] * n_fields * grid / (us * 1e-6) / dp4a_peak
        out.append(r)
    return out


def cpu_baseline(q, seed, target_s=12.0):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    px = q.width * q.height
    times, ref = [], None
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        ref = oracle.run_quad(*q.images(), seed=seed, params=oracle.default_params(**PARAMS))
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > target_s or len(times) >= 8:
            break
    return {"value": px / statistics.mean(times), "unit": "px/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} full {q.width}x{q.height} quads (features, both fields, filter, seeds), "
                      f"{cores} OpenMP threads, {statistics.mean(times):.2f} s each"}, ref


# The batched workload: 32 quads of uneven sizes, 8 each, scene seeds 100..131
BATCH_SIZES = [("driving", 1242, 375), ("driving", 1024, 436), ("planes", 640, 192), ("planes", 512, 160)]
BATCH_PER_SIZE = 8


def _gen_batch_quad(args):
    fam, w, h, seed = args
    q = scenegen.make_quad(fam, w, h, seed, supersample=1, with_gt=False)
    return q.L0, q.R0, q.L1, q.R1


def make_batch_quads():
    """The 32 quads, rendered in a spawn process pool (before any GPU work)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    jobs = [(fam, w, h, 100 + k * BATCH_PER_SIZE + j) for k, (fam, w, h) in enumerate(BATCH_SIZES)
            for j in range(BATCH_PER_SIZE)]
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_batch_quad, jobs)), [j[3] for j in jobs]


# Groups of the batch on concurrent streams (BatchMatcher.streams) tried by the bench
BATCH_STREAMS = (1, 2, 4)


def bench_batched(sff, torch, dev, quads, seeds, params, tuning, steps, warmup):
    """Matched px/s of the 32-quad batch: one CUDA graph of shared launches
    (sff_run_batch; the quads in 1, 2 or 4 groups on concurrent streams, the
    fastest kept) vs the plain per-quad form (one graph per quad, replayed one
    after the other); outputs compared for identity."""
    from paper_1710_10096_gb300 import tune
    sizes = [(im[0].shape[1], im[0].shape[0]) for im in quads]
    px = sum(w * h for w, h in sizes)
    bm = sff.BatchMatcher(sizes, params, device=dev, tuning=tuning)
    for k, im in enumerate(quads):
        bm.load(k, *im)
    # the batch's own scale-0 variant and schedules (autotuned on the batch);
    # the plain per-quad form below keeps the tuning passed in
    batch_tuning = tune.autotune_batch(bm, seeds)
    group_options = [ns for ns in BATCH_STREAMS if ns <= len(quads)]
    g_by = {}
    for ns in group_options:
        bm.streams = ns
        g_by[ns] = bm.capture(seeds)
    # plain: one matcher + graph per quad
    plain = []
    for k, im in enumerate(quads):
        m = sff.QuadMatcher(sizes[k][0], sizes[k][1], params, device=dev, tuning=tuning)
        for j in range(4):
            m.dev_in[j].copy_(torch.as_tensor(im[j]))
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s):
            m.run(*m.dev_in.unbind(0), seed=seeds[k], stream=s)
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                m.run(*m.dev_in.unbind(0), seed=seeds[k], stream=torch.cuda.current_stream(dev))
        plain.append((m, g))
    torch.cuda.synchronize(dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / steps / 1e3

    t_by = {ns: timed(g.replay) for ns, g in g_by.items()}
    best = min(t_by, key=t_by.get)
    t_batch = t_by[best]
    bm.streams = best
    g_by[best].replay()  # the outputs compared below
    t_plain = timed(lambda: [g.replay() for _, g in plain])
    # per-kernel (and per-scale) breakdown of the batched graph: one replay of
    # a second capture with event spans around the launches
    s = torch.cuda.Stream(device=dev)
    sff.profile_enable(True)
    try:
        gp = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gp, stream=s):
            bm.run(seeds, torch.cuda.current_stream(dev))
        gp.replay()
        s.synchronize()
        bprof, bscales = merge_scales(sff.profile_collect(with_units=True))
    finally:
        sff.profile_enable(False)
    del gp
    breakdown = {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(bprof.items(), key=lambda kv: -kv[1][1])}
    per_scale = {f"s{sc}": {"launches": nl, "iterations": n, "ms": ms, "avg_iteration_us": 1e3 * ms / n}
                 for sc, (n, ms, nl) in sorted(bscales.get("k_iteration", {}).items())}
    same = all(bq.seeds_numpy().tobytes() == m.buf.seeds_numpy().tobytes()
               and torch.equal(bq.fwd, m.fwd) and torch.equal(bq.inv, m.inv) for bq, (m, _) in zip(bm.quads, plain))
    out = {"workload": "32 quads: 8 x 1242x375 + 8 x 1024x436 (driving scenes), 8 x 640x192 + 8 x 512x160 "
                       "(planes scenes), scene seeds 100..131",
           "px_per_step": px, "value": px / t_batch, "unit": "px/s", "ms_per_step": 1e3 * t_batch,
           "plain_value": px / t_plain, "plain_ms_per_step": 1e3 * t_plain, "speedup_vs_plain": t_plain / t_batch,
           "identical_to_plain": bool(same), "cuda_graph": True, "streams": best,
           "by_streams": {str(ns): {"value": px / t, "ms_per_step": 1e3 * t} for ns, t in sorted(t_by.items())},
           "tuning": {"scale0": list(batch_tuning.scale_variants()[0]), "pair_fields": batch_tuning.pair_fields,
                      "alternate_order": batch_tuning.alternate_order,
                      "coarse": "derived from the batch's grid sizes",
                      "plain_per_quad": {"scale0": list(tuning.scale_variants()[0]), "pair_fields": tuning.pair_fields,
                                         "alternate_order": tuning.alternate_order,
                                         "coarse": "derived from each quad's grid sizes"}},
           "kernels_ms": breakdown, "k_iteration_per_scale": per_scale}
    del bm, plain, g_by
    torch.cuda.empty_cache()
    return out


SERVING_RATES = (10.0, 50.0, 200.0, 400.0)  # aggregate quads/s over 8 camera streams


def bench_serving(sff, torch, dev, quads, params, tuning, max_requests=240):
    """p50/p99 latency and sustained px/s of the continuous-batching server
    vs the plain per-request server, on Poisson arrivals from 8 streams over
    a pool of 24 quads (8 each of 1242x375, 1024x436, 640x192)."""
    from paper_1710_10096_gb300.serve import PlainServer, Server, poisson_arrivals, simulate, summarize
    pool = [tuple(im) for im in quads if im[0].shape[1] in (1242, 1024, 640)]
    out = {"pool": f"{len(pool)} quads: 8 x 1242x375, 8 x 1024x436, 8 x 640x192", "streams": 8,
           "requests": "min(240, 3 s of arrivals), at least 40 per rate"}
    srv = Server(params, tuning, device=dev, max_batch=32)
    for size in {(im[0].shape[1], im[0].shape[0]) for im in pool}:
        srv.reserve(size, 8)  # resident slots: no allocation while requests wait
    plain = PlainServer(params, tuning, device=dev)
    # warm-up: slots allocated, and every kernel variant the batch sizes pick
    # loaded once (a single-quad batch takes other per-scale variants than a
    # large one; CUDA loads a kernel at its first launch)
    for warm_rate in (400.0, 20.0):
        simulate(srv, poisson_arrivals(warm_rate, 24, 8, len(pool), seed=1), pool)
        simulate(plain, poisson_arrivals(warm_rate, 24, 8, len(pool), seed=1), pool)
    for rate in SERVING_RATES:
        n_requests = max(40, min(max_requests, int(3 * rate)))
        arr = poisson_arrivals(rate, n_requests, 8, len(pool), seed=7)
        r1, w1 = simulate(srv, arr, pool)
        r2, w2 = simulate(plain, arr, pool)
        a, b = summarize(r1, w1), summarize(r2, w2)
        same = all(x.seeds.tobytes() == y.seeds.tobytes() for x, y in zip(r1, r2))
        out[f"rate_{int(rate)}"] = {"continuous": a, "plain": b, "identical_results": bool(same)}
    return out


def bench_paper_order(sff, torch, dev, m, q, params, reps=3):
    """Matching of both fields of the quad in the paper's order (in-place
    raster sweeps, sff_match_views_sequential) against the checkerboard
    order (sff_match_views), on the same resident pyramids; CUDA events on
    one stream, L2 as left by the previous call."""
    w, h = q.width, q.height
    ws = torch.empty(sff.workspace_bytes(w, h, params), dtype=torch.uint8, device=dev)
    f = torch.empty((h, w, 4), dtype=torch.int16, device=dev)
    c = torch.empty((h, w), dtype=torch.int32, device=dev)
    L0, R0, L1, R1 = m.pyr
    stream = torch.cuda.Stream(device=dev)

    def both(fn):
        fn(L0, L1, R0, R1, w, h, 0, MATCH_SEED, f, c, ws, params, stream=stream)
        fn(R1, R0, L1, L0, w, h, 1, MATCH_SEED, f, c, ws, params, stream=stream)

    out = {}
    with torch.cuda.stream(stream):
        for name, fn in (("paper_order", sff.match_views_sequential), ("checkerboard", sff.match_views)):
            both(fn)  # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                both(fn)
            b.record(stream)
            stream.synchronize()
            out[name] = a.elapsed_time(b) / reps
    return {"what": "both fields of the quad matched from resident pyramids (initialisation, 4 scales x 12 "
                    "iterations, random search), ms per quad", "paper_order_ms": out["paper_order"],
            "checkerboard_ms": out["checkerboard"], "slowdown": out["paper_order"] / out["checkerboard"]}


# nominal dense FP64 rate of a GB300 (the double-precision fits are bound by it)
FP64_PEAK_GFLOPS = 1250.0


def field_quality(field, q):
    """Outlier rates of the dense field against the scene's ground truth on
    the pixels visible in all four views (the KITTI scene flow measures of
    Table 1: an estimate is an outlier when its error exceeds 3 px and 5 %
    of the true value; SF = any of D1, D2, Fl)."""
    m = ~q.occluded
    f = field[m].astype(np.float64)
    g = q.gt[m]
    e0, e1 = np.abs(f[:, 2] - g[:, 2]), np.abs(f[:, 3] - g[:, 3])
    ef = np.hypot(f[:, 0] - g[:, 0], f[:, 1] - g[:, 1])
    d1 = (e0 > 3) & (e0 > 0.05 * np.abs(g[:, 2]))
    d2 = (e1 > 3) & (e1 > 0.05 * np.abs(g[:, 3]))
    fl = (ef > 3) & (ef > 0.05 * np.hypot(g[:, 0], g[:, 1]))
    return {"D1": float(d1.mean()), "D2": float(d2.mean()), "Fl": float(fl.mean()), "SF": float((d1 | d2 | fl).mean()),
            "epe_flow": float(ef.mean()), "mae_d0": float(e0.mean()), "mae_d1": float(e1.mean()),
            "pixels": int(m.sum())}


def bench_interpolation(sff, torch, dev, m, q, params, steps, warmup, cpu: bool):
    """Dense interpolation (Sec. 3.2) of the quad's seeds on the GPU: the
    interpolation alone and the whole method (matching stage + interpolation)
    as one CUDA graph, both timed with CUDA events after an L2 flush; the
    per-kernel profile; the FP64 roofline of the model fits; the quality of
    the dense field; the oracle on a bounded sample."""
    w, h = q.width, q.height
    ip = sff.default_interp_params(w, h, q.focal, q.baseline)
    field = torch.empty((h, w, 4), dtype=torch.float32, device=dev)
    ws = torch.empty(sff.interp_workspace_bytes(w, h, m.capacity), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    dev_in = [torch.as_tensor(im).to(dev) for im in q.images()]

    def interp():
        sff.interpolate(m.seeds, m.count, m.capacity, w, h, ip, field, ws, stream=stream)

    with torch.cuda.stream(stream):
        m.run(*dev_in, seed=MATCH_SEED, stream=stream)
        for _ in range(max(1, warmup)):
            interp()
        stream.synchronize()
        sff.profile_enable(True)
        for _ in range(3):
            flush.zero_()
            interp()
        stream.synchronize()
        prof = sff.profile_collect()
        sff.profile_enable(False)
        g1, g2 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1, stream=stream):
            sff.interpolate(m.seeds, m.count, m.capacity, w, h, ip, field, ws, stream=torch.cuda.current_stream())
        with torch.cuda.graph(g2, stream=stream):
            m.run(*dev_in, seed=MATCH_SEED, stream=torch.cuda.current_stream())
            sff.interpolate(m.seeds, m.count, m.capacity, w, h, ip, field, ws, stream=torch.cuda.current_stream())
        times = {}
        for name, g in (("interp", g1), ("method", g2)):
            for _ in range(max(1, warmup)):
                g.replay()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                g.replay()
                b.record(stream)
            stream.synchronize()
            times[name] = statistics.mean(a.elapsed_time(b) for a, b in ev)
    status = sff.interp_status(ws, w, h, m.capacity)
    n = min(int(m.count.item()), m.capacity)
    out = {"what": "dense interpolation of the quad's GPU seeds (sff_interpolate) and the whole method "
                   "(matching stage + interpolation, one CUDA graph); ms per quad, L2 flushed before each",
           "seeds": n, "status": status, "interp_ms": times["interp"], "method_ms": times["method"],
           "interp_px_per_s": w * h / (times["interp"] / 1e3), "method_px_per_s": w * h / (times["method"] / 1e3),
           "params": {"k_geo": ip.k_geo, "k_motion": ip.k_motion, "alpha": ip.alpha, "dist_unit": ip.dist_unit,
                      "focal": ip.focal, "baseline": ip.baseline}}
    total = sum(v[1] for v in prof.values())
    out["kernels"] = {k: {"ms": v[1] / v[0], "share": v[1] / total}
                      for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    if "k_interp_models" in prof:
        # algorithmic FP64 work of the weighted normal equations: 20 flops per
        # plane neighbour, 53 per motion neighbour (centroid 7, centred sums 46)
        flops = n * (20 * ip.k_geo + 53 * ip.k_motion)
        t = prof["k_interp_models"][1] / prof["k_interp_models"][0] / 1e3
        out["roofline"] = {"bound": "fp64", "kernel": "k_interp_models", "achieved": flops / t / 1e9,
                           "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": flops / t / 1e9 / FP64_PEAK_GFLOPS,
                           "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                           "algo_flops_per_launch": flops, "avg_launch_us": t * 1e6}
    out["quality"] = field_quality(field.cpu().numpy(), q)
    if cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        oracle.set_threads(cores)
        seeds = sff.seeds_to_numpy(m.seeds.cpu().numpy(), n)
        op = oracle.interp_params(w, h, q.focal, q.baseline)
        rng = np.random.default_rng(0)
        which = rng.choice(n, size=min(n, 1024), replace=False)
        t0 = time.perf_counter()
        models = oracle.seed_models(seeds, op, which=which)
        tm = (time.perf_counter() - t0) * n / len(which)
        pix = np.stack([rng.integers(0, w, 16384), rng.integers(0, h, 16384)], 1)
        t0 = time.perf_counter()
        oracle.interpolate_pixels(seeds, op, pix, models=models)
        tp = (time.perf_counter() - t0) * w * h / len(pix)
        out["cpu_baseline"] = {"value": w * h / (tm + tp), "unit": "px/s", "cores": cores, "kind": "oracle",
                               "sample": f"models of {len(which)} of {n} seeds and 16384 of {w * h} pixels, "
                                         f"scaled to the whole field ({tm:.1f} s + {tp:.1f} s)"}
    return out


def bench_fill(sff, torch, dev, m, q, params, steps, warmup, cpu: bool):
    """Disparity fill (Sec. 3.1, last paragraph) on the quad: the SGM map of
    L0/R0 (sff_sgm, D = 128) and the seeds with disparity-only entries
    (sff_emit_seeds_geo), timed with CUDA events after an L2 flush; the
    per-kernel profile and the HBM roofline of the dominant kernel; the
    density and accuracy the fill adds, and what it does to the dense field;
    the oracle's SGM on the host cores."""
    w, h = q.width, q.height
    sp = sff.default_sgm_params()
    D = sp.max_disp
    stream = torch.cuda.Stream(device=dev)
    dev_in = [torch.as_tensor(im).to(dev) for im in q.images()]
    disp = torch.empty((h, w), dtype=torch.int16, device=dev)
    sws = torch.empty(sff.sgm_workspace_bytes(w, h, sp), dtype=torch.uint8, device=dev)
    cap = m.capacity
    gseeds = torch.zeros(20 * cap, dtype=torch.uint8, device=dev)
    gcount = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(sff.workspace_bytes(w, h, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def fill(s):
        sff.sgm(dev_in[0], dev_in[1], disp, sws, sp, stream=s)
        sff.emit_seeds_geo(m.fwd, m.fwd_cost, m.keep, m.cerr, disp, gseeds, cap, gcount, ws, params, stream=s)

    with torch.cuda.stream(stream):
        m.run(*dev_in, seed=MATCH_SEED, stream=stream)
        for _ in range(max(1, warmup)):
            fill(stream)
        stream.synchronize()
        sff.profile_enable(True)
        for _ in range(3):
            flush.zero_()
            fill(stream)
        stream.synchronize()
        prof = sff.profile_collect()
        sff.profile_enable(False)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fill(torch.cuda.current_stream())
        for _ in range(max(1, warmup)):
            g.replay()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            g.replay()
            b.record(stream)
        stream.synchronize()
    t_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    out = {"what": "SGM map of L0/R0 (D = 128, P1 10, P2 120) and the seeds with the disparity fill, one CUDA graph, "
                   "ms per quad, L2 flushed before each", "ms": t_ms, "px_per_s": w * h / (t_ms / 1e3)}
    prof = {k.split("<")[0]: v for k, v in prof.items()}
    total = sum(v[1] for v in prof.values())
    out["kernels"] = {k: {"ms": v[1] / v[0], "share": v[1] / total}
                      for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    # algorithmic bytes per pixel: k_sgm_paths reads the D cost bytes and
    # writes D bytes of path costs in each of the 8 directions; k_sgm_wta
    # reads the 8 D bytes and writes the 2-byte disparity; k_sgm_cost reads
    # the census words and writes D bytes
    algo = {"k_sgm_paths": 16 * D, "k_sgm_wta": 8 * D + 2, "k_sgm_cost": D + 16}
    dom = max((k for k in prof if k in algo), key=lambda k: prof[k][1], default=None)
    if dom:
        peak, peak_src = measured_peak_hbm()
        t = prof[dom][1] / prof[dom][0] / 1e3
        achieved = algo[dom] * w * h / t / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "peak_source": peak_src,
                           "algo_bytes_per_launch": algo[dom] * w * h, "avg_launch_us": t * 1e6}
    # what the fill adds, against the scene's ground truth (visible pixels)
    vis = ~q.occluded
    d_sgm = disp.cpu().numpy().astype(np.float64)
    fwd = m.fwd.cpu().numpy()
    keep = m.keep.cpu().numpy().astype(bool)
    valid = m.fwd_cost.cpu().numpy() != sff.EMPTY_COST
    gt0 = q.gt[..., 2]

    def d1(est, mask):
        e = np.abs(est[mask] - gt0[mask])
        return float(((e > 3) & (e > 0.05 * np.abs(gt0[mask]))).mean()) if mask.any() else None

    agree = valid & ~keep & (np.abs(fwd[..., 2] - d_sgm) <= params.tau_c)
    n_all = min(int(gcount.item()), cap)
    gs = sff.seeds_to_numpy(gseeds.cpu().numpy(), n_all)
    out["quality"] = {"sgm_D1": d1(d_sgm, vis), "joint_density": float((keep & vis).sum() / vis.sum()),
                      "joint_D1": d1(fwd[..., 2].astype(np.float64), keep & vis),
                      "fill_density": float(((keep | agree) & vis).sum() / vis.sum()),
                      "fill_only_D1": d1(fwd[..., 2].astype(np.float64), agree & vis),
                      "seeds_joint": int((gs["kind"] == 0).sum()), "seeds_disparity_only": int((gs["kind"] == 1).sum())}
    # the dense field from the seeds with the fill (geometry from every seed,
    # motion from the joint seeds)
    ip = sff.default_interp_params(w, h, q.focal, q.baseline)
    field = torch.empty((h, w, 4), dtype=torch.float32, device=dev)
    iws = torch.empty(sff.interp_workspace_bytes(w, h, cap), dtype=torch.uint8, device=dev)
    sff.interpolate(gseeds, gcount, cap, w, h, ip, field, iws)
    torch.cuda.synchronize()
    out["quality"]["field_with_fill"] = field_quality(field.cpu().numpy(), q)
    out["quality"]["field_with_fill"]["interp_status"] = sff.interp_status(iws, w, h, cap)
    if cpu:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        oracle.set_threads(cores)
        t0 = time.perf_counter()
        od = oracle.sgm(q.L0, q.R0, oracle.sgm_params(max_disp=D))
        tc = time.perf_counter() - t0
        out["bit_exact_sgm"] = bool(np.array_equal(od, disp.cpu().numpy()))
        out["cpu_baseline"] = {"value": w * h / tc, "unit": "px/s", "cores": cores, "kind": "oracle",
                               "sample": f"the whole {w}x{h} SGM map once ({tc:.2f} s), {cores} OpenMP threads "
                                         "(one per direction)"}
    return out


def bench_method(sff, torch, dev, m, q, params, steps, warmup):
    """The whole method without its trained parts, as one CUDA graph: the
    matching stage on one stream and the SGM map (which needs only L0 and R0)
    on a second stream at the same time, then the seeds with the disparity
    fill and the dense interpolation.  CUDA events around each replay, L2
    flushed before it."""
    w, h = q.width, q.height
    sp = sff.default_sgm_params()
    ip = sff.default_interp_params(w, h, q.focal, q.baseline)
    cap = m.capacity
    dev_in = [torch.as_tensor(im).to(dev) for im in q.images()]
    disp = torch.empty((h, w), dtype=torch.int16, device=dev)
    sws = torch.empty(sff.sgm_workspace_bytes(w, h, sp), dtype=torch.uint8, device=dev)
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(sff.workspace_bytes(w, h, params), dtype=torch.uint8, device=dev)
    field = torch.empty((h, w, 4), dtype=torch.float32, device=dev)
    iws = torch.empty(sff.interp_workspace_bytes(w, h, cap), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def method(a, b):
        fork = torch.cuda.Event()
        fork.record(a)
        b.wait_event(fork)
        sff.sgm(dev_in[0], dev_in[1], disp, sws, sp, stream=b)
        m.run(*dev_in, seed=MATCH_SEED, stream=a)
        join = torch.cuda.Event()
        join.record(b)
        a.wait_event(join)
        sff.emit_seeds_geo(m.fwd, m.fwd_cost, m.keep, m.cerr, disp, seeds, cap, count, ws, params, stream=a)
        sff.interpolate(seeds, count, cap, w, h, ip, field, iws, stream=a)

    with torch.cuda.stream(s1):
        for _ in range(max(1, warmup)):
            method(s1, s2)
        s1.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s1):
            method(torch.cuda.current_stream(), s2)
        for _ in range(max(1, warmup)):
            g.replay()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(s1)
            g.replay()
            b.record(s1)
        s1.synchronize()
    t_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    n = min(int(count.item()), cap)
    kinds = sff.seeds_to_numpy(seeds.cpu().numpy(), n)["kind"]
    return {"what": "matching stage || SGM map, then seeds with the disparity fill and the dense interpolation, "
                    "one CUDA graph with two streams, ms per quad, L2 flushed before each",
            "ms": t_ms, "px_per_s": w * h / (t_ms / 1e3), "seeds": n, "disparity_only_seeds": int((kinds == 1).sum()),
            "quality": field_quality(field.cpu().numpy(), q), "interp_status": sff.interp_status(iws, w, h, cap)}


def bench_sift(sff, torch, dev, m, q, params, steps, warmup):
    """The paper's own cost (Eq. 1 with SIFT-PCA features) against the WHT-SSD
    cost on the quad: the phi features of the four images and both fields
    with the SIFT cost (CUDA events, L2 flushed before each), and the
    accuracy of the forward field and of the filtered matches of both modes
    against the scene's ground truth."""
    w, h = q.width, q.height
    S = params.num_scales
    stream = torch.cuda.Stream(device=dev)
    dev_in = [torch.as_tensor(im).to(dev) for im in q.images()]
    phis = [torch.empty((S, h, w, 4), dtype=torch.float32, device=dev) for _ in range(4)]
    sws = torch.empty(sff.sift_workspace_bytes(w, h), dtype=torch.uint8, device=dev)
    ws = torch.empty(sff.workspace_bytes(w, h, params), dtype=torch.uint8, device=dev)
    f = [torch.empty((h, w, 4), dtype=torch.int16, device=dev) for _ in range(2)]
    c = [torch.empty((h, w), dtype=torch.int32, device=dev) for _ in range(2)]
    keep = torch.empty((h, w), dtype=torch.uint8, device=dev)
    cerr = torch.empty((h, w), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    L0, R0, L1, R1 = m.pyr
    pL0, pR0, pL1, pR1 = phis

    def feats():
        sff.sift_features(dev_in, phis, sws, params, stream=stream)

    def fields():
        sff.match_views_sift(L0, L1, R0, R1, pL0, pL1, pR0, pR1, w, h, 0, MATCH_SEED, f[0], c[0], ws, params,
                             stream=stream)
        sff.match_views_sift(R1, R0, L1, L0, pR1, pR0, pL1, pL0, w, h, 1, MATCH_SEED, f[1], c[1], ws, params,
                             stream=stream)

    times = {}
    with torch.cuda.stream(stream):
        m.run(*dev_in, seed=MATCH_SEED, stream=stream)
        for name, fn in (("features_ms", feats), ("fields_ms", fields)):
            for _ in range(max(1, warmup)):
                fn()
            ev = []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                ev.append((a, b))
            stream.synchronize()
            times[name] = statistics.mean(x.elapsed_time(y) for x, y in ev)
        sff.consistency_filter(f[0], c[0], f[1], c[1], keep, cerr, ws, params, stream=stream)
        stream.synchronize()
        sff.profile_enable(True)
        feats()
        fields()
        stream.synchronize()
        prof = sff.profile_collect()
        sff.profile_enable(False)
    vis = ~q.occluded
    gt = q.gt

    def accuracy(field, kept):
        e = np.abs(field.astype(np.float64) - gt)
        bad = (e > 3).any(axis=2)
        out = {"raw_outliers": float(bad[vis].mean()), "raw_epe_flow": float(np.hypot(e[..., 0], e[..., 1])[vis].mean())}
        k = kept & vis
        out["filtered_density"] = float(k.sum() / vis.sum())
        out["filtered_outliers"] = float(bad[k].mean()) if k.any() else None
        return out

    res = {"what": "the paper's SIFT-PCA cost (Eq. 1) against the WHT-SSD cost on the quad; times per quad with the "
                   "L2 flushed before each, accuracy against the scene's ground truth (visible pixels; an outlier has a "
                   "component off by more than 3 px)",
           "features_ms": times["features_ms"], "fields_ms": times["fields_ms"],
           "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
           "sift": accuracy(f[0].cpu().numpy(), keep.cpu().numpy().astype(bool)),
           "wht": accuracy(m.fwd.cpu().numpy(), m.keep.cpu().numpy().astype(bool))}
    return res


def combine_ranks(t_step: float, px_per_rank: int, world: int, device=None):
    """Whole-job throughput of `world` replicas: every rank matched its own
    quad; the job time is the slowest rank's (max over ranks), the pixels are
    summed.  Returns (max step time, px/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([t_step, float(px_per_rank)], dtype=torch.float64, device=device)
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        px = t[1:].clone()
        dist.all_reduce(px, op=dist.ReduceOp.SUM)
        return float(tmax.item()), float(px.item()) / float(tmax.item())
    return t_step, px_per_rank / t_step


def workload_config(workload, q, params, world):
    """The work of one step, identical in both arms' lines: what is matched,
    with which parameters and seeds, and the cache condition of the timing."""
    return {"workload": workload, "width": q.width, "height": q.height, "quads_per_step": 1,
            "parallelism": f"replicas{world}", "params": dict(params), "scene_seed": SCENE_SEED,
            "match_seed": MATCH_SEED, "scene_ranges": q.ranges(),
            "l2": "GPU arm: L2 flushed between timed steps (256 MB write outside the step events)"}


def summary(line):
    """The headline figures of the line, repeated at its end."""
    out = {"value_mpx_s": line["value"] / 1e6, "e2e_mpx_s": line["e2e"]["value"] / 1e6,
           "roofline_frac": (line.get("roofline") or {}).get("frac"),
           "per_scale_frac": [round(r["frac"], 3) for r in (line.get("roofline") or {}).get("per_scale", [])],
           "device_status": line.get("device_status"), "bit_exact": line.get("bit_exact")}
    st = line.get("stage_rooflines")
    if st:
        out["stage_speed_of_light_frac"] = st["stage"]["frac"]
        out["kernel_fracs"] = {k: round(v["frac"], 3) for k, v in st.items() if k not in ("stage", "peaks")}
    b = line.get("batched")
    if b:
        out.update(batched_mpx_s=b["value"] / 1e6, plain_per_quad_mpx_s=b["plain_value"] / 1e6,
                   batched_speedup=b["speedup_vs_plain"], batched_identical=b["identical_to_plain"])
    sv = line.get("serving")
    if sv:
        for rate in ("rate_400", "rate_50"):
            if rate in sv:
                r = sv[rate]
                out[f"serving_{rate[5:]}_p50_p99_ms"] = [r["continuous"]["p50_ms"], r["continuous"]["p99_ms"]]
                out[f"serving_{rate[5:]}_plain_p50_p99_ms"] = [r["plain"]["p50_ms"], r["plain"]["p99_ms"]]
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    q = scenegen.make_named(args.workload, SCENE_SEED)
    # the CUDA arm's parameters, passed explicitly
    op = oracle.default_params(**PARAMS)
    # calibrate on one warm-up; shrink each step to a band of rows if the whole
    # run would exceed about two minutes
    t0 = time.perf_counter()
    oracle.run_quad(*q.images(), seed=MATCH_SEED, params=op)
    t_full = time.perf_counter() - t0
    rows = q.height
    budget = 120.0
    if (args.steps + args.warmup) * t_full > budget:
        rows = max(48, int(q.height * budget / ((args.steps + args.warmup) * t_full)))
    imgs = [im[:rows].copy() for im in q.images()]
    for _ in range(max(0, args.warmup - 1)):
        oracle.run_quad(*imgs, seed=MATCH_SEED, params=op)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_quad(*imgs, seed=MATCH_SEED, params=op)
        times.append(time.perf_counter() - t0)
    px = q.width * rows
    value = px / statistics.mean(times)
    sample = (f"{'full quad' if rows == q.height else f'band of the first {rows} rows of'} {q.width}x{q.height} "
              f"per step, {cores} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "px/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": dict(workload_config(args.workload, q, PARAMS, 1), height=rows),
            "cpu_baseline": {"value": value, "unit": "px/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "px/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1710_10096_gb300 as sff

    rank, world, local = dist_info()
    batch = None if args.no_batch else make_batch_quads()  # CPU work before any GPU call
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sff.build()

    q = scenegen.make_named(args.workload, SCENE_SEED + rank)
    params = sff.default_params(**PARAMS)
    # work distribution of the propagation kernels: autotuned once per image
    # size (any setting gives bit-identical results)
    from paper_1710_10096_gb300 import tune
    if args.tuning == "auto":
        if args.tuning_cache:
            tune.load_cache(args.tuning_cache)
        probe = sff.QuadMatcher(q.width, q.height, params, device=dev)
        probe.run(*[torch.as_tensor(im).to(dev) for im in q.images()], seed=MATCH_SEED)
        tuning = tune.autotune(probe.pyr, q.width, q.height, params, reps=3)
        del probe
    elif args.tuning.lstrip().startswith("{"):
        tuning = tune._tuning_of(json.loads(args.tuning))
    else:
        tuning = sff.make_tuning(*(int(v) for v in args.tuning.split(",")))
    tuning.features_form = {"separable": 0, "tensor": 1, "pairs": 2}[args.features_form]
    tuning.overlap = args.overlap
    if args.tma:
        tuning.tma = 1
        if not sff.lib().sff_tuning_supported(ctypes.byref(tuning)):
            raise SystemExit(f"--tma: scale-0 variant {tuning.scale_variants()[0]} has no TMA form")
    # the batch and the server take the tuned scale-0 variant with the coarse
    # scales derived from their (much larger) launch sizes
    batch_tuning = sff.make_tuning(tuning.lanes_per_pixel, tuning.tile_x, tuning.tile_y, tuning.slots, None, 0,
                                   tuning.pair_fields, tuning.min_ctas, tuning.alternate_order & 1,
                                   overlap=args.overlap)
    m = sff.QuadMatcher(q.width, q.height, params, device=dev, tuning=tuning)
    stream = torch.cuda.Stream(device=dev)
    host_in = torch.empty((4, q.height, q.width, 3), dtype=torch.uint8).pin_memory()
    for k, im in enumerate(q.images()):
        host_in[k].copy_(torch.as_tensor(im))
    dev_in = host_in.to(dev)
    if args.tuning == "auto":
        # the coarse scales' fused form checked on the whole stage (beside the
        # overlapped features); a no-op for a tuning read from the cache
        tuning = tune.refine_stage(m, list(dev_in.unbind(0)), MATCH_SEED)
        if args.tuning_cache and rank == 0:
            tune.save_cache(args.tuning_cache)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # warm-up, then the per-kernel profile: a CUDA graph of prof_steps steps
    # (each after an L2 flush) with an event-record node around every kernel,
    # so that the kernels are timed as the timed graph below runs them
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            m.run(*dev_in.unbind(0), seed=MATCH_SEED, stream=stream)
        stream.synchronize()
        prof_steps = max(3, min(args.steps, 10))
        sff.profile_enable(True)
        pgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(pgraph, stream=stream):
            for _ in range(prof_steps):
                flush.zero_()
                m.run(*dev_in.unbind(0), seed=MATCH_SEED, stream=torch.cuda.current_stream())
        pgraph.replay()
        stream.synchronize()
        prof, prof_scales = merge_scales(sff.profile_collect(with_units=True))
        sff.profile_enable(False)
        del pgraph

    # the timed region: CUDA-graph replays of the whole stage on resident inputs
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        m.run(*dev_in.unbind(0), seed=MATCH_SEED, stream=stream)
        stream.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            m.run(*dev_in.unbind(0), seed=MATCH_SEED, stream=torch.cuda.current_stream())
        for _ in range(args.warmup):
            graph.replay()
        stream.synchronize()
    sff.device_status(stream, reset=True)  # conditions of the set-up runs (none expected) cleared
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()  # L2 flush, outside the step's events
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    px = q.width * q.height
    t_step, value = combine_ranks(statistics.mean(step_ms) / 1e3, px, world, dev)

    # end to end through the public host API: pinned host images in, seeds out
    e2e_times = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            dev_in.copy_(host_in, non_blocking=True)
            graph.replay()
            host_seeds = m.seeds.to("cpu", non_blocking=True)
            host_count = m.count.to("cpu", non_blocking=True)
            stream.synchronize()
            if k >= args.warmup:
                e2e_times.append(time.perf_counter() - t0)
    n_seeds = int(host_count.item())
    # device-side conditions of every run above (bounded waits, seed capacity)
    dev_status = sff.device_status(stream, reset=True)
    dev_timeouts = sff.device_timeouts(reset=True)
    e2e = {"value": combine_ranks(statistics.mean(e2e_times), px, world, dev)[1], "unit": "px/s",
           "h2d_bytes_per_step": int(host_in.numel()), "d2h_bytes_per_step": int(m.seeds.numel() + 4)}

    # integer peaks of this GPU, measured now (the other roofline of the
    # integer cost evaluations)
    int_peak = {"dp4a_per_s": sff.int_peak("dp4a", stream), "imad_per_s": sff.int_peak("imad", stream),
                "source": "measured in this run (sff_int_peak: 8 chains per thread, 8 x 256 threads per SM)"}
    # roofline of the dominant kernel (largest share of profiled time)
    launches_per_step = sum(v[0] for v in prof.values()) / prof_steps
    dom = max(prof, key=lambda k: prof[k][1])
    dom_launches, dom_ms = prof[dom]
    peak, peak_src = measured_peak_hbm()
    roof = None
    if dom in ALGO_BYTES:
        units = _units(dom, q.width, q.height, params) * prof_steps
        bytes_per_launch = ALGO_BYTES[dom] * units / dom_launches
        achieved = bytes_per_launch / (dom_ms / dom_launches / 1e3) / 1e9
        tr = ncu_traffic(dom, dom_launches / prof_steps)
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": tr, "peak_source": peak_src,
                "algo_bytes_per_launch": bytes_per_launch, "avg_launch_us": 1e3 * dom_ms / dom_launches}
        roof["hbm_frac"] = achieved / peak
        if dom in ALGO_DP4A:
            dp4a = ALGO_DP4A[dom] * units / dom_launches
            roof["int_peak"] = int_peak
            roof["int_frac"] = dp4a / (dom_ms / dom_launches / 1e3) / int_peak["dp4a_per_s"]
            roof["int_ops"] = f"{ALGO_DP4A[dom]} dp4a per grid pixel and iteration (3 candidates x 3 views x 48 MAC)"
            # the binding roofline is the larger fraction
            if roof["int_frac"] > roof["hbm_frac"]:
                roof.update(bound="int", frac=roof["int_frac"])
        if dom in prof_scales:
            sc = {s: (n / prof_steps, ms / prof_steps, nl / prof_steps) for s, (n, ms, nl) in prof_scales[dom].items()}
            roof["per_scale"] = iteration_scales(sc, q.width, q.height, 2, peak, int_peak["dp4a_per_s"])
    total_prof = sum(v[1] for v in prof.values())
    kernels = {k: {"launches_per_step": v[0] / prof_steps, "ms_per_step": v[1] / prof_steps,
                   "share": v[1] / total_prof} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    bf16_peak, bf16_src = measured_peak_bf16()
    stage_roof = stage_rooflines(prof, prof_steps, q.width, q.height, params, peak, bf16_peak, 1e3 * t_step)
    stage_roof["peaks"] = {"hbm_gbs": peak, "hbm_source": peak_src, "bf16_tflops": bf16_peak,
                           "bf16_source": bf16_src + " (burst)"}

    line = {"metric": METRIC, "value": value, "unit": "px/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": workload_config(args.workload, q, params.as_dict(), world),
            "launch": {"cuda_graph": True,
                       "tuning_per_scale": [list(v) for v in tuning.scale_variants()],
                       "tuning_fields": "(lanes per pixel, candidate slots, tile_x, tile_y, min CTAs per SM) of "
                                        "scales 0..3",
                       "pair_fields": tuning.pair_fields, "alternate_order_bits": tuning.alternate_order,
                       "pdl_bits": tuning.pdl, "fuse_bits": tuning.fuse, "tma": tuning.tma,
                       "overlap": tuning.overlap, "features_form": args.features_form},
            "roofline": roof, "stage_rooflines": stage_roof, "gpu_launches": int(round(launches_per_step * args.steps)),
            "e2e": e2e, "clocks": clk, "kernels": kernels, "seeds": n_seeds,
            "device_status": sff.lib().sff_status_string(dev_status).decode(), "device_timeouts": dev_timeouts}
    if not args.no_paper_order:
        line["paper_order"] = bench_paper_order(sff, torch, dev, m, q, params)
    if not args.no_interp:
        line["interpolation"] = bench_interpolation(sff, torch, dev, m, q, params, min(args.steps, 20),
                                                    max(3, args.warmup), rank == 0 and not args.no_cpu_baseline)
    if not args.no_fill:
        line["disparity_fill"] = bench_fill(sff, torch, dev, m, q, params, min(args.steps, 20), max(3, args.warmup),
                                            rank == 0 and not args.no_cpu_baseline)
    if not (args.no_fill or args.no_interp):
        line["method"] = bench_method(sff, torch, dev, m, q, params, min(args.steps, 20), max(3, args.warmup))
    if not args.no_sift:
        line["sift_cost"] = bench_sift(sff, torch, dev, m, q, params, 3, 1)
    if batch is not None:
        line["batched"] = bench_batched(sff, torch, dev, batch[0], batch[1], params, batch_tuning,
                                        min(args.steps, 20), max(1, args.warmup))
        if not args.no_serving:
            line["serving"] = bench_serving(sff, torch, dev, batch[0], params, batch_tuning)
    if rank == 0 and not args.no_cpu_baseline:
        cb, ref = cpu_baseline(q, MATCH_SEED)
        line["cpu_baseline"] = cb
        got = sff.seeds_to_numpy(host_seeds.numpy(), min(n_seeds, m.capacity))
        line["bit_exact"] = bool(got.tobytes() == ref["seeds"].tobytes() and n_seeds == len(ref["seeds"])
                                 and np.array_equal(m.fwd.cpu().numpy(), ref["fwd"])
                                 and np.array_equal(m.inv.cpu().numpy(), ref["inv"])
                                 and dev_status == sff.OK and dev_timeouts == 0)
    line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
