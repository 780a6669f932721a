"""Autotuner of the propagation work distribution.

Every variant of the iteration kernel (lanes per pixel, candidate slots,
tile; VARIANT_SPACE) is run at all scales of the caller's pyramids, and the
launches of each scale are timed as one span of CUDA events inside a CUDA
graph (sff_profile_enable), so that each scale gets its own fastest variant.
All variants give bit-identical results (tested), so the choice only affects
speed.  Results are cached per image-size bucket.
"""
from __future__ import annotations

import json
import os

from . import (VARIANT_SPACE, Tuning, default_params, default_tuning, make_tuning, match_quad_tuned, profile_collect,
               profile_enable, workspace_bytes)

_CACHE: dict = {}


def size_bucket(width: int, height: int) -> str:
    """Sizes that share a tuning: rounded up to multiples of 64 x 32."""
    return f"{(width + 63) // 64 * 64}x{(height + 31) // 32 * 32}"


def _tuning_of(per_scale) -> Tuning:
    l, c, tx, ty, mb = per_scale[0]
    return make_tuning(l, tx, ty, c, per_scale[1:], min_ctas=mb)


def scale_times(pyramids, width: int, height: int, variant, params=None, reps: int = 3, stream=None) -> dict:
    """{scale: us per launch} of the iteration kernel with `variant`
    (lanes, slots, tile_x, tile_y, min_ctas) at every scale, timed as one span
    of events per scale in a CUDA graph of `reps` matching runs."""
    import torch
    params = params or default_params()
    dev = pyramids[0].device
    ws = torch.empty(workspace_bytes(width, height, params), dtype=torch.uint8, device=dev)
    out = [torch.empty((height, width, 4), dtype=torch.int16, device=dev) for _ in range(2)]
    cst = [torch.empty((height, width), dtype=torch.int32, device=dev) for _ in range(2)]
    s = stream or torch.cuda.Stream(device=dev)
    l, c, tx, ty, mb = variant
    t = make_tuning(l, tx, ty, c, [variant] * (params.num_scales - 1), min_ctas=mb)
    with torch.cuda.stream(s):
        match_quad_tuned(*pyramids, width, height, 1, t, out[0], cst[0], out[1], cst[1], ws, params, s)
        s.synchronize()
        profile_enable(True)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                for _ in range(reps):
                    match_quad_tuned(*pyramids, width, height, 1, t, out[0], cst[0], out[1], cst[1], ws, params,
                                     torch.cuda.current_stream(dev))
            g.replay()
            s.synchronize()
            prof = profile_collect()
        finally:
            profile_enable(False)
    res = {}
    for name, (n, ms) in prof.items():
        base, sep, sc = name.partition("/s")
        if base == "k_iteration" and sep:
            res[int(sc)] = 1e3 * ms / n
    return res


def autotune(pyramids, width: int, height: int, params=None, reps: int = 3, space=None, stream=None,
             verbose: bool = False) -> Tuning:
    """Fastest variant per scale for W x H, measured on the given L0/R0/L1/R1 pyramids."""
    params = params or default_params()
    key = (size_bucket(width, height), tuple(params.as_dict().values()))
    if key in _CACHE:
        return _tuning_of(_CACHE[key])
    S = params.num_scales
    best = [None] * 4
    best_us = [float("inf")] * 4
    for v in (space or VARIANT_SPACE):
        times = scale_times(pyramids, width, height, tuple(v), params, reps, stream)
        for s, us in times.items():
            if us < best_us[s]:
                best[s], best_us[s] = tuple(v), us
        if verbose:
            print(f"variant {tuple(v)}: " + " ".join(f"s{s} {us:.2f} us" for s, us in sorted(times.items())))
    d = default_tuning().scale_variants()
    per_scale = [best[s] if s < S and best[s] is not None else (d[s] if s == 0 else (0,) * 5) for s in range(4)]
    _CACHE[key] = per_scale
    return _tuning_of(per_scale)


def save_cache(path: str) -> None:
    with open(path, "w") as f:
        json.dump({f"{k[0]}|{','.join(map(str, k[1]))}": [list(v) for v in vs] for k, vs in _CACHE.items()}, f,
                  indent=1)


def load_cache(path: str) -> int:
    """Adds the tunings of a file written by save_cache; entries that this
    build does not support (another build's variant space) are skipped.
    Returns the number of entries taken."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        entries = json.load(f)
    taken = 0
    space = set(VARIANT_SPACE)
    for k, vs in entries.items():
        b, p = k.split("|")
        if not (isinstance(vs, list) and len(vs) == 4 and all(isinstance(v, list) and len(v) == 5 for v in vs)):
            continue
        vs = [tuple(v) for v in vs]
        if tuple(vs[0]) in space and all(v in space or v == (0,) * 5 for v in vs[1:]):
            _CACHE[(b, tuple(int(x) for x in p.split(",")))] = vs
            taken += 1
    return taken


__all__ = ["autotune", "scale_times", "size_bucket", "save_cache", "load_cache", "default_tuning"]
