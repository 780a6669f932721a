"""Departures from the paper's procedure do not degrade match quality.

The oracle switches readings D3 (exact nearest neighbours instead of
approximate kD-trees), D4 (checkerboard half-steps instead of in-place
sequential scans) and D5 (counter-based instead of sequential random
numbers) back to the paper's own procedure one at a time; on a rendered
scene with ground truth, the matches of the built readings are as dense and
as accurate as those of the sequential-order run (Sec. 3.1; the paper's
matches row of Tab. 2 reports outliers and density of the same kind).
"""
import numpy as np

import departure_report as dr


def test_each_departure_changes_results_but_not_quality(orc):
    rows = dr.report(dr.scenes(full=False))
    by = {label: m for _, label, m in rows}
    built, paper = by["built"], by["paper order (D3+D4+D5)"]
    for label, m in by.items():
        assert m["density"] > 0.85, label
        assert m["outliers"] < 0.03, label
        assert m["epe"] < 0.8, label
    assert abs(built["outliers"] - paper["outliers"]) < 0.01
    assert abs(built["density"] - paper["density"]) < 0.03
    assert abs(built["epe"] - paper["epe"]) < 0.05


def test_paper_modes_really_differ(orc):
    import scenegen
    q = scenegen.make_named("planes_256x80", 1)
    ref = orc.run_quad(*q.images(), seed=3)
    for mode in (orc.SEQUENTIAL_SCAN, orc.KDTREE_INIT, orc.SEQUENTIAL_RNG):
        r = orc.run_quad(*q.images(), seed=3, params=orc.default_params(order_mode=mode))
        assert not np.array_equal(r["fwd"], ref["fwd"]), mode
