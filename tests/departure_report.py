"""Match quality of each departure from the paper's own procedure.

Runs the oracle on rendered scenes with ground truth in five modes:
  built   -- the readings the CUDA path implements (bit-exact to it)
  D4      -- in-place sequential raster scans instead of checkerboard half-steps
  D3      -- approximate kD-tree leaves instead of exact nearest neighbours
  D5      -- one sequential random stream instead of counter-based Philox
  paper   -- all three together: the sequential-order run
and reports, for the filtered matches and for the seeds, the share of
visible pixels kept (density), the end-point error of the flow (EPE, px),
the mean absolute disparity error and the outlier rate (any component of
(u, v, d0, d1) off by more than 3 px).

python tests/departure_report.py [--full]   (--full adds the two 1242x375 /
1024x436 scenes; the default runs the 256x80 planes scene only)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import scenegen  # noqa: E402

MODES = [("built", 0), ("D4 sequential scans", oracle.SEQUENTIAL_SCAN), ("D3 kD-tree init", oracle.KDTREE_INIT),
         ("D5 sequential RNG", oracle.SEQUENTIAL_RNG),
         ("paper order (D3+D4+D5)", oracle.SEQUENTIAL_SCAN | oracle.KDTREE_INIT | oracle.SEQUENTIAL_RNG)]


def quality(q, r):
    vis = ~q.occluded
    keep = r["keep"].astype(bool) & vis
    err = np.abs(r["fwd"].astype(np.float64) - q.gt)
    sd = r["seeds"]
    sx, sy = sd["x"].astype(int), sd["y"].astype(int)
    svis = vis[sy, sx]
    serr = np.abs(np.stack([sd["u"], sd["v"], sd["d0"], sd["d1"]], -1).astype(np.float64) - q.gt[sy, sx])[svis]
    return {
        "density": keep.sum() / max(1, vis.sum()),
        "epe": float(np.hypot(err[..., 0], err[..., 1])[keep].mean()),
        "disp_err": float(err[..., 2:][keep].mean()),
        "outliers": float((err[keep].max(-1) > 3).mean()),
        "seeds": int(svis.sum()),
        "seed_outliers": float((serr.max(-1) > 3).mean()) if len(serr) else 0.0,
    }


def report(scenes, seed=1234):
    rows = []
    for name, q in scenes:
        for label, mode in MODES:
            r = oracle.run_quad(*q.images(), seed=seed, params=oracle.default_params(order_mode=mode))
            rows.append((name, label, quality(q, r)))
    return rows


def markdown(rows):
    out = ["| scene | mode | density | EPE px | disp err px | outliers >3px | seeds | seed outliers |",
           "|---|---|---|---|---|---|---|---|"]
    for name, label, m in rows:
        out.append(f"| {name} | {label} | {m['density']:.3f} | {m['epe']:.3f} | {m['disp_err']:.3f} | "
                   f"{100 * m['outliers']:.2f} % | {m['seeds']} | {100 * m['seed_outliers']:.2f} % |")
    return "\n".join(out)


def scenes(full: bool):
    out = [("planes 256x80 (seed 1)", scenegen.make_named("planes_256x80", 1))]
    if full:
        out.append(("driving 1242x375 (seed 2)", scenegen.make_named("driving_1242x375", 2)))
        out.append(("movie 1024x436 (seed 2)", scenegen.make_named("movie_1024x436", 2)))
    return out


if __name__ == "__main__":
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    print(markdown(report(scenes("--full" in sys.argv))))
