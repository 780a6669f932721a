"""Autotuner of the propagation work distribution.

Times every supported sff_tuning (lanes per pixel x tile shape) on the
caller's pyramids with CUDA events and keeps the fastest per image size.
All settings give bit-identical results (tested), so the choice only
affects speed.
"""
from __future__ import annotations

import json
import os

from . import (TUNING_SPACE, Tuning, default_params, default_tuning, make_tuning, match_quad_tuned,
               workspace_bytes)

_CACHE: dict = {}


def size_bucket(width: int, height: int) -> str:
    """Sizes that share a tuning: rounded up to multiples of 64 x 32."""
    return f"{(width + 63) // 64 * 64}x{(height + 31) // 32 * 32}"


def autotune(pyramids, width: int, height: int, params=None, reps: int = 3, space=None, stream=None,
             verbose: bool = False) -> Tuning:
    """Fastest tuning for W x H, measured on the given L0/R0/L1/R1 pyramids."""
    import torch
    params = params or default_params()
    key = (size_bucket(width, height), tuple(params.as_dict().values()))
    if key in _CACHE:
        return make_tuning(*_CACHE[key])
    dev = pyramids[0].device
    ws = torch.empty(workspace_bytes(width, height, params), dtype=torch.uint8, device=dev)
    out = [torch.empty((height, width, 4), dtype=torch.int16, device=dev) for _ in range(2)]
    cst = [torch.empty((height, width), dtype=torch.int32, device=dev) for _ in range(2)]
    s = stream or torch.cuda.current_stream(dev)
    best, best_ms, times = None, float("inf"), {}
    for cand in (space or TUNING_SPACE):
        t = make_tuning(*cand)
        with torch.cuda.stream(s):
            match_quad_tuned(*pyramids, width, height, 1, t, out[0], cst[0], out[1], cst[1], ws, params, s)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(reps):
                match_quad_tuned(*pyramids, width, height, 1, t, out[0], cst[0], out[1], cst[1], ws, params, s)
            b.record(s)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        times[cand] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    if verbose:
        for cand, ms in sorted(times.items(), key=lambda kv: kv[1]):
            print(f"tuning {cand}: {ms:.3f} ms")
    _CACHE[key] = best
    return make_tuning(*best)


def save_cache(path: str) -> None:
    with open(path, "w") as f:
        json.dump({f"{k[0]}|{','.join(map(str, k[1]))}": v for k, v in _CACHE.items()}, f, indent=1)


def load_cache(path: str) -> int:
    """Adds the tunings of a file written by save_cache; entries that this
    build does not support (another build's tuning space) are skipped.
    Returns the number of entries taken."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        entries = json.load(f)
    taken = 0
    for k, v in entries.items():
        b, p = k.split("|")
        if tuple(v) in TUNING_SPACE:
            _CACHE[(b, tuple(int(x) for x in p.split(",")))] = tuple(v)
            taken += 1
    return taken


__all__ = ["autotune", "size_bucket", "save_cache", "load_cache", "default_tuning"]
