"""Autotuner of the propagation work distribution.

Every variant of the iteration kernel (lanes per pixel, candidate slots,
tile, resident CTAs; VARIANT_SPACE) is run at all scales of the caller's
pyramids, and the launches of each scale are timed as one span of CUDA events
inside a CUDA graph (sff_profile_enable), so that each scale gets its own
fastest variant.  Then the schedules are tried on those variants: a quad's two
fields alternating tile by tile (pair_fields), and, per scale, every other
launch visiting its tiles last-to-first (a bit of alternate_order) and
programmatic dependent launch (a bit of pdl).  A coarse scale may instead
run all its iterations in one cooperative launch (a bit of fuse) with the
fastest of FUSED_SPACE, and scale 0 may stage its reference records with
tensor copies (tma) when its variant is in TMA_SPACE.  All settings give bit-identical results (tested),
so the choice only affects speed.  Results are cached per image-size bucket.
"""
from __future__ import annotations

import json
import os

from . import (FUSED_SPACE, TMA_SPACE, VARIANT_SPACE, Tuning, default_params, default_tuning, make_tuning, match_quad_tuned,
               profile_collect, profile_enable, workspace_bytes)

_CACHE: dict = {}
# per cache key just measured by autotune(): {fused scale: (variant, alt, pdl)
# of its fastest separate launches}, for refine_stage()
_UNFUSED: dict = {}


def size_bucket(width: int, height: int) -> str:
    """Sizes that share a tuning: rounded up to multiples of 64 x 32."""
    return f"{(width + 63) // 64 * 64}x{(height + 31) // 32 * 32}"


def _tuning_of(entry) -> Tuning:
    """Tuning of a cache entry: {"variants": [4 x (lanes, slots, tile_x, tile_y, min_ctas)],
    "pair": 0 | 1, "alt": scale bits, "pdl": scale bits, "fuse": scale bits, "tma": 0 | 1,
    "overlap": 0 | 1 (absent: 1)}."""
    vs = entry["variants"]
    l, c, tx, ty, mb = vs[0]
    return make_tuning(l, tx, ty, c, vs[1:], 0, entry["pair"], mb, entry["alt"], 0, entry.get("pdl", 0),
                       entry.get("fuse", 0), entry.get("tma", 0), entry.get("overlap", 1))


def scale_times(pyramids, width: int, height: int, tuning: Tuning, params=None, reps: int = 3, stream=None) -> dict:
    """{scale: us per iteration} of the iteration kernel with `tuning`, timed
    as one span of events per scale in a CUDA graph of `reps` matching runs."""
    import torch
    params = params or default_params()
    dev = pyramids[0].device
    ws = torch.empty(workspace_bytes(width, height, params), dtype=torch.uint8, device=dev)
    out = [torch.empty((height, width, 4), dtype=torch.int16, device=dev) for _ in range(2)]
    cst = [torch.empty((height, width), dtype=torch.int32, device=dev) for _ in range(2)]
    s = stream or torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        match_quad_tuned(*pyramids, width, height, 1, tuning, out[0], cst[0], out[1], cst[1], ws, params, s)
        s.synchronize()
        profile_enable(True)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                for _ in range(reps):
                    match_quad_tuned(*pyramids, width, height, 1, tuning, out[0], cst[0], out[1], cst[1], ws, params,
                                     torch.cuda.current_stream(dev))
            g.replay()
            s.synchronize()
            prof = profile_collect(with_units=True)
        finally:
            profile_enable(False)
    res = {}
    for name, (_, ms, units) in prof.items():
        base, sep, sc = name.partition("/s")
        if base == "k_iteration" and sep:
            res[int(sc)] = 1e3 * ms / units
    return res


def autotune(pyramids, width: int, height: int, params=None, reps: int = 3, space=None, stream=None,
             verbose: bool = False) -> Tuning:
    """Fastest variant per scale, then the fastest schedules on them, for
    W x H, measured on the given L0/R0/L1/R1 pyramids."""
    params = params or default_params()
    key = (size_bucket(width, height), tuple(params.as_dict().values()))
    if key in _CACHE:
        return _tuning_of(_CACHE[key])
    S = params.num_scales
    best = [None] * 4
    best_us = [float("inf")] * 4
    for v in (space or VARIANT_SPACE):
        v = tuple(v)
        t = make_tuning(v[0], v[2], v[3], v[1], [v] * (S - 1), min_ctas=v[4])
        times = scale_times(pyramids, width, height, t, params, reps, stream)
        for s, us in times.items():
            if us < best_us[s]:
                best[s], best_us[s] = v, us
        if verbose:
            print(f"variant {v}: " + " ".join(f"s{s} {us:.2f} us" for s, us in sorted(times.items())))
    d = default_tuning().scale_variants()
    variants = [best[s] if s < S and best[s] is not None else (d[s] if s == 0 else (0,) * 5) for s in range(4)]
    # the fused form of the coarse scales: every scale >= 1 fused with one variant
    fused, fused_us = [None] * 4, [float("inf")] * 4
    coarse_bits = sum(1 << s for s in range(1, S))
    for v in (FUSED_SPACE if coarse_bits else []):
        t = make_tuning(variants[0][0], variants[0][2], variants[0][3], variants[0][1], [v] * (S - 1),
                        min_ctas=variants[0][4], fuse=coarse_bits)
        times = scale_times(pyramids, width, height, t, params, reps, stream)
        for s, us in times.items():
            if s >= 1 and us < fused_us[s]:
                fused[s], fused_us[s] = tuple(v), us
        if verbose:
            print(f"fused {tuple(v)}: " + " ".join(f"s{s} {us:.2f} us" for s, us in sorted(times.items())))
    # schedules on the chosen variants: pairing for the whole run, and per
    # scale the best of reversed order on / off x dependent launch on / off
    full = (1 << S) - 1
    combos = [(a, d) for a in (0, full) for d in (0, full)]
    sched = {}
    for pair in (0, 1):
        for alt, pdl in combos:
            t = _tuning_of({"variants": variants, "pair": pair, "alt": alt, "pdl": pdl})
            sched[(pair, alt, pdl)] = scale_times(pyramids, width, height, t, params, reps, stream)
            if verbose:
                print(f"pair {pair} alt {alt} pdl {pdl}: " +
                      " ".join(f"s{s} {us:.2f} us" for s, us in sorted(sched[(pair, alt, pdl)].items())))

    def best_combo(pair, s):
        return min(combos, key=lambda c: sched[(pair, c[0], c[1])][s])

    def scale_us(pair, s):
        return min(sched[(pair, *best_combo(pair, s))][s], fused_us[s])

    def total(pair):
        return sum(scale_us(pair, s) for s in range(S))

    pair = min((0, 1), key=total)
    fuse = sum(1 << s for s in range(1, S) if fused_us[s] < sched[(pair, *best_combo(pair, s))][s])
    # what each fused scale would run as separate launches, for refine_stage
    _UNFUSED[key] = {s: (tuple(variants[s]), *best_combo(pair, s)) for s in range(1, S) if (fuse >> s) & 1}
    for s in range(1, S):
        if (fuse >> s) & 1:
            variants[s] = fused[s]
    alt = sum(1 << s for s in range(S) if best_combo(pair, s)[0] and not (fuse >> s) & 1)
    pdl = sum(1 << s for s in range(S) if best_combo(pair, s)[1] and not (fuse >> s) & 1)
    entry = {"variants": variants, "pair": pair, "alt": alt, "pdl": pdl, "fuse": fuse, "tma": 0}
    # scale 0 with TMA-staged reference records, on the chosen schedule
    if tuple(variants[0]) in TMA_SPACE:
        plain = scale_times(pyramids, width, height, _tuning_of(entry), params, reps, stream)
        staged = scale_times(pyramids, width, height, _tuning_of(dict(entry, tma=1)), params, reps, stream)
        if verbose:
            print(f"scale 0 tma 0: {plain[0]:.2f} us, tma 1: {staged[0]:.2f} us")
        if staged[0] < plain[0]:
            entry["tma"] = 1
    _CACHE[key] = entry
    return _tuning_of(entry)


def _graph_ms(run, reps: int, flush, stream) -> float:
    """Median milliseconds of `reps` CUDA-graph replays of run(stream), each
    after an L2 flush (a write of `flush`) outside its events."""
    import statistics

    import torch
    run(stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        run(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        g.replay()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
    del g
    return statistics.median(ts)


def refine_stage(matcher, images, seed: int, reps: int = 7, verbose: bool = False) -> Tuning:
    """Whole-stage check of the coarse scales' fused form.  With the feature
    overlap the coarse scales run beside the features of the finer scales,
    which autotune()'s per-scale spans (matching alone) do not see.  Tries
    every subset of the tuned fuse bits -- a scale left unfused runs the
    variant and schedule bits autotune() found for its separate launches --
    on CUDA-graph replays of matcher.run on `images` (device tensors,
    L2 flushed between replays), and keeps the fastest if it beats the
    tuned setting by more than 1 % (differences below that are within the
    run-to-run spread of a stage), caching the result.  A no-op
    for a tuning that autotune() did not just measure (e.g. from a cache
    file).  Leaves matcher.tuning at the chosen setting."""
    import torch
    params = matcher.params
    key = (size_bucket(matcher.width, matcher.height), tuple(params.as_dict().values()))
    alts = _UNFUSED.pop(key, None)
    if not alts or key not in _CACHE:
        return matcher.tuning
    base = matcher.tuning
    stream = torch.cuda.Stream(device=matcher.device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=matcher.device)
    scales = sorted(alts)
    best, best_ms = None, float("inf")
    for mask in range(1 << len(scales)):
        e = dict(_CACHE[key], variants=list(_CACHE[key]["variants"]))
        for j, s in enumerate(scales):
            if (mask >> j) & 1:  # scale s as separate launches
                v, alt, pdl = alts[s]
                e["variants"][s] = v
                e["fuse"] &= ~(1 << s)
                e["alt"] |= (1 << s) if alt else 0
                e["pdl"] |= (1 << s) if pdl else 0
        t = _tuning_of(e)
        t.features_form, t.overlap, t.tma = base.features_form, base.overlap, base.tma
        matcher.tuning = t
        ms = _graph_ms(lambda st: matcher.run(*images, seed=seed, stream=st), reps, flush, stream)
        if verbose:
            print(f"stage fuse {e['fuse']}: {ms:.4f} ms")
        if mask == 0:
            best, best_ms = e, ms / 1.01  # the tuned setting, with the 1 % margin
        elif ms < best_ms:
            best, best_ms = e, ms
    _CACHE[key] = best
    matcher.tuning = _tuning_of(best)
    matcher.tuning.features_form, matcher.tuning.overlap, matcher.tuning.tma = \
        base.features_form, base.overlap, base.tma
    return matcher.tuning


def autotune_batch(batch, seeds, space=None, reps: int = 3, verbose: bool = False) -> Tuning:
    """Fastest scale-0 variant and schedules (pair_fields, alternate_order of
    scale 0) for the quads of `batch` (a BatchMatcher, its images loaded),
    timed on CUDA-graph replays of the whole batch; the coarse scales take the
    variants derived from the batch's grid sizes.  Leaves the batch with the
    chosen tuning."""
    import statistics

    import torch
    cands = space or [v for v in VARIANT_SPACE if v[0] == 1 and v[1] == 0]
    dev = batch.device
    s = torch.cuda.Stream(device=dev)
    best, best_ms = None, float("inf")
    for v in cands:
        for pair in (0, 1):
            for alt in (0, 1):
                batch.tuning = make_tuning(v[0], v[2], v[3], v[1], None, 0, pair, v[4], alt)
                g = batch.capture(seeds)
                with torch.cuda.stream(s):
                    g.replay()
                    s.synchronize()
                    ts = []
                    for _ in range(reps):
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(s)
                        g.replay()
                        b.record(s)
                        b.synchronize()
                        ts.append(a.elapsed_time(b))
                del g
                ms = statistics.median(ts)
                if verbose:
                    print(f"batch {tuple(v)} pair {pair} alt {alt}: {ms:.3f} ms")
                if ms < best_ms:
                    best, best_ms = batch.tuning, ms
    batch.tuning = best
    return best


def save_cache(path: str) -> None:
    with open(path, "w") as f:
        json.dump({f"{k[0]}|{','.join(map(str, k[1]))}": {"variants": [list(v) for v in e["variants"]],
                                                          "pair": e["pair"], "alt": e["alt"], "pdl": e.get("pdl", 0),
                                                          "fuse": e.get("fuse", 0), "tma": e.get("tma", 0)}
                   for k, e in _CACHE.items()}, f, indent=1)


def load_cache(path: str) -> int:
    """Adds the tunings of a file written by save_cache; entries that this
    build does not support (another build's variant space or format) are
    skipped.  Returns the number of entries taken."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        entries = json.load(f)
    taken = 0
    space = set(VARIANT_SPACE)
    fused_space = set(FUSED_SPACE)
    for k, e in entries.items():
        b, p = k.split("|")
        if not (isinstance(e, dict) and isinstance(e.get("variants"), list) and len(e["variants"]) == 4 and
                all(isinstance(v, list) and len(v) == 5 for v in e["variants"]) and e.get("pair") in (0, 1) and
                isinstance(e.get("alt"), int) and 0 <= e["alt"] <= 15 and isinstance(e.get("pdl", 0), int) and
                0 <= e.get("pdl", 0) <= 15 and isinstance(e.get("fuse", 0), int) and 0 <= e.get("fuse", 0) <= 14 and
                e.get("fuse", 0) % 2 == 0 and e.get("fuse", 0) & (e["alt"] | e.get("pdl", 0)) == 0 and
                e.get("tma", 0) in (0, 1)):
            continue
        vs = [tuple(v) for v in e["variants"]]
        fuse = e.get("fuse", 0)
        if vs[0] in space and all(v in space or v == (0,) * 5 for v in vs[1:]) and \
                all(vs[s] in fused_space or vs[s] == (0,) * 5 for s in range(1, 4) if (fuse >> s) & 1) and \
                (e.get("tma", 0) == 0 or vs[0] in set(TMA_SPACE)):
            _CACHE[(b, tuple(int(x) for x in p.split(",")))] = {"variants": vs, "pair": e["pair"], "alt": e["alt"],
                                                                "pdl": e.get("pdl", 0), "fuse": fuse,
                                                                "tma": e.get("tma", 0)}
            taken += 1
    return taken


__all__ = ["autotune", "autotune_batch", "refine_stage", "scale_times", "size_bucket", "save_cache", "load_cache",
           "default_tuning"]
