"""Pins of the oracle's initialisation and propagation (Sec. 3.1).

Propagation with random search is a heuristic without a closed-form result,
so it is pinned by what must hold for any correct implementation:
  - exhaustive nearest-neighbour initialisation on tiny images;
  - every final cost is the true cost of the final vector and is bounded
    below by the exhaustive minimum over all vectors;
  - costs never increase from one iteration to the next;
  - exact recovery of integer shifts and ground-truth recovery on a
    rendered scene;
  - results do not depend on the number of threads.
"""
import numpy as np
import pytest

import scenegen

EMPTY = np.iinfo(np.int32).max


def _feats(orc, imgs, params):
    return [orc.features(im, params)[0] for im in imgs]


def _ssd(a, b):
    d = a.astype(np.int64) - b.astype(np.int64)
    return (d * d).sum(-1)


def test_init_exhaustive(orc):
    # 16x16 image, scales {0, 1}: the coarsest grid G_1 has 64 points; with
    # K_T = 64 every temporal point is a leaf, so the initial vector is the
    # exhaustive argmin of the cost with ties resolved by leaf rank.
    imgs = scenegen.random_images(16, 16, 21)
    p = orc.default_params(num_scales=2, iterations=0, knn_temporal=64, knn_epipolar=2)
    Fall = _feats(orc, imgs, p)  # images L0, R0, L1, R1
    for mirror in (0, 1):
        sg = -1 if mirror else 1
        roles = (0, 2, 1, 3) if not mirror else (3, 1, 2, 0)  # ref, temporal, stereo, cross
        fld, cost = orc.match_views(*(Fall[i] for i in roles), mirror, 1, p)
        ref, tmp, ste, crs = (Fall[i][1] for i in roles)  # scale-1 features
        grid = [(x, y) for y in range(0, 16, 2) for x in range(0, 16, 2)]
        for (px, py) in grid:
            a = ref[py, px]
            best = None
            for (tx, ty) in grid:
                dT = int(_ssd(a, tmp[ty, tx]))
                for sx in range(0, 16, 2):
                    if sg * (px - sx) < 0:
                        continue
                    dS = int(_ssd(a, ste[py, sx]))
                    for cx in range(0, 16, 2):
                        if sg * (tx - cx) < 0:
                            continue
                        dX = int(_ssd(a, crs[ty, cx]))
                        key = (dT + dS + dX, dT, ty * 16 + tx, dS, py * 16 + sx, dX, ty * 16 + cx)
                        vec = (tx - px, ty - py, sg * (px - sx), sg * (tx - cx))
                        if best is None or key < best[0]:
                            best = (key, vec)
            assert tuple(int(v) for v in fld[py, px]) == best[1], (mirror, px, py)
        # non-grid points of the finest scale stay empty without iterations
        assert (cost[1::2, :] == EMPTY).all() and (cost[:, 1::2] == EMPTY).all()


def test_init_ties_go_to_the_first_combination(orc):
    # a constant image: every feature is the same, so every combination
    # costs 0.  The nearest-neighbour lists then hold the lowest raster
    # indices, and the first combination wins: the temporal point (0, 0),
    # the stereo and cross points of lowest x that the sign of d allows
    # (x = 0 for the left-reference pass, x = px / tx for the mirrored one)
    img = np.full((16, 20, 3), 90, np.uint8)
    p = orc.default_params(num_scales=2, iterations=0)
    F = orc.features(img, p)[0]
    for mirror in (0, 1):
        fld, cost = orc.match_views(F, F, F, F, mirror, 1, p)
        for py in range(0, 16, 2):
            for px in range(0, 20, 2):
                want = (-px, -py, 0 if mirror else px, 0)
                assert tuple(int(v) for v in fld[py, px]) == want, (mirror, px, py)
                assert cost[py, px] == 0


def _constant_cost_fill(H, W, mirror, iters):
    """The propagation when every cost ties (constant features): a vector
    moves only into an empty pixel, which takes its first non-empty
    predecessor, (x - dx n, y) before (x, y - dy n), as of the start of its
    half-step; the colour-0 pixels ((x + y) / n even) go first; the
    iterations take the directions (1, 1), (-1, -1), (1, -1), (-1, 1) in
    turn.  Two scales: the coarsest grid (n = 2) holds its first
    combinations and keeps them; at n = 1 its points keep their vectors and
    every other pixel starts empty.  Random search never wins a tie."""
    vec = {(x, y): (-x, -y, 0 if mirror else x, 0) for y in range(0, H, 2) for x in range(0, W, 2)}
    dirs = [(1, 1), (-1, -1), (1, -1), (-1, 1)]
    for it in range(iters):
        dx, dy = dirs[it % 4]
        for colour in (0, 1):
            snap = dict(vec)
            for y in range(H):
                for x in range(W):
                    if (x + y) % 2 != colour or (x, y) in snap:
                        continue
                    for q in ((x - dx, y), (x, y - dy)):
                        if q in snap:
                            vec[(x, y)] = snap[q]
                            break
    return vec


@pytest.mark.parametrize("iters", [1, 2, 3, 4])
def test_propagation_order_on_tied_costs(orc, iters):
    # pins the checkerboard colours, each iteration's predecessors and
    # direction, the candidates' order, strict improvement in propagation and
    # random search, and which points carry over from the coarser scale
    H, W = 9, 10
    p = orc.default_params(num_scales=2, iterations=iters)
    F = orc.features(np.full((H, W, 3), 90, np.uint8), p)[0]
    for mirror in (0, 1):
        fld, cost = orc.match_views(F, F, F, F, mirror, 1, p)
        want = _constant_cost_fill(H, W, mirror, iters)
        for y in range(H):
            for x in range(W):
                if (x, y) in want:
                    assert tuple(int(v) for v in fld[y, x]) == want[(x, y)] and cost[y, x] == 0, (mirror, x, y)
                else:
                    assert cost[y, x] == EMPTY, (mirror, x, y)
        if iters == 1:
            assert sum((x, y) not in want for y in range(H) for x in range(W)) == 20  # the (odd, odd) pixels


def _rs_offset(r, n):
    # reading D5: j = mulhi(r, 4 n), offset = floor((j + 1) / 2) - n
    j = (int(r) * 4 * n) >> 32
    return (j + 1) // 2 - n


def _first_accepted(orc, seed, scale, mirror, iters, need):
    """Offsets of the first random-search draw of pixel 0 whose u offset is
    at least `need` (counter = (pixel 0, iteration, scale + 4 pass, 0), key =
    the seed's two words), with d0, d1 clamped at 0; None if no iteration's is."""
    key = np.array([seed & 0xffffffff, seed >> 32], np.uint32)
    n = 1 << scale
    for it in range(iters):
        o = [_rs_offset(r, n) for r in orc.philox4x32_10(np.array([0, it, scale + 4 * mirror, 0], np.uint32), key)]
        if o[0] >= need:
            return (o[0], o[1], max(0, o[2]), max(0, o[3]))
    return None


@pytest.mark.parametrize("seed", [1, 2, 3, 12345, 2 ** 40 + 7])
def test_random_search_draws(orc, seed):
    # a 2 x 1 image, two scales.  The coarsest grid holds only pixel 0, which
    # has no predecessors, and its best temporal target (x = 1, cost 0; x = 0
    # costs 100) is off that grid: only random search can move it, and it
    # does at the first draw that reaches x = 1, with all four offsets of
    # that draw.  At full resolution pixel 1 then copies pixel 0.  When no
    # coarse draw reaches x = 1, pixel 1 takes pixel 0's initial vector
    # (target x = 1 from there) and pixel 0 waits for a full-resolution draw.
    ref = np.zeros((2, 1, 2, 48), np.int8)
    ref[..., 0] = 10
    tmp = np.zeros((2, 1, 2, 48), np.int8)
    tmp[:, :, 1, 0] = 10
    for mirror in (0, 1):
        for iters in (1, 3, 12):
            p = orc.default_params(num_scales=2, iterations=iters)
            fld, cost = orc.match_views(ref, tmp, ref, ref, mirror, seed, p)
            got = [tuple(int(v) for v in fld[0, x]) for x in range(2)]
            coarse = _first_accepted(orc, seed, 1, mirror, iters, 1)
            if coarse is not None:
                assert got == [coarse, coarse], (mirror, iters)
                assert list(cost[0]) == [0, 0]
                continue
            fine = _first_accepted(orc, seed, 0, mirror, iters, 1)
            assert got == [fine or (0, 0, 0, 0), (0, 0, 0, 0)], (mirror, iters)
            assert list(cost[0]) == [0 if fine else 100, 0]


def test_init_knn_leaves(orc):
    # with K_T = 4 the chosen temporal match is one of the 4 nearest grid points
    imgs = scenegen.random_images(40, 24, 22)
    p = orc.default_params(num_scales=2, iterations=0)
    F = _feats(orc, imgs, p)
    fld, _ = orc.match_views(F[0], F[2], F[1], F[3], 0, 1, p)
    ref, tmp = F[0][1], F[2][1]
    gy, gx = np.mgrid[0:24:2, 0:40:2]
    for py in range(0, 24, 2):
        for px in range(0, 40, 2):
            d = _ssd(ref[py, px][None, None], tmp[0:24:2, 0:40:2])
            order = sorted(zip(d.ravel().tolist(), (gy * 40 + gx).ravel().tolist()))[:4]
            t = (py + int(fld[py, px, 1])) * 40 + px + int(fld[py, px, 0])
            assert t in [i for _, i in order]


def test_costs_are_true_costs_and_bounded_below(orc):
    imgs = scenegen.random_images(20, 14, 23)
    p = orc.default_params(num_scales=1, iterations=12)
    F = _feats(orc, imgs, p)
    fld, cost = orc.match_views(F[0], F[2], F[1], F[3], 0, 77, p)
    ref, ste, tmp, crs = (f[0] for f in F)
    h, w = 14, 20
    hits = 0
    for py in range(h):
        for px in range(w):
            c = int(cost[py, px])
            assert c != EMPTY
            assert c == orc.cost(ref, tmp, ste, crs, 0, px, py, fld[py, px])
            a = ref[py, px]
            dS = min(int(_ssd(a, ste[py, sx])) for sx in range(0, px + 1))
            dTX = min(int(_ssd(a, tmp[ty, tx])) + min(int(_ssd(a, crs[ty, cx])) for cx in range(0, tx + 1))
                      for ty in range(h) for tx in range(w))
            assert c >= dS + dTX
            hits += c == dS + dTX
    assert hits > 0


def test_monotone_over_iterations(orc):
    imgs = scenegen.random_images(48, 32, 24)
    prev = None
    for it in range(0, 9):
        p = orc.default_params(num_scales=1, iterations=it, knn_temporal=4)
        F = _feats(orc, imgs, p)
        _, cost = orc.match_views(F[0], F[2], F[1], F[3], 0, 5, p)
        if prev is not None:
            assert (cost.astype(np.int64) <= prev).all()
        prev = cost.astype(np.int64)


def test_threads_do_not_change_results(orc):
    q = scenegen.make_named("planes_256x80", 3)
    before = orc.get_threads()
    try:
        orc.set_threads(1)
        r1 = orc.run_quad(*q.images(), seed=99)
        orc.set_threads(4)
        r4 = orc.run_quad(*q.images(), seed=99)
    finally:
        orc.set_threads(before)
    for k in ("fwd", "fwd_cost", "inv", "inv_cost", "keep", "cerr"):
        assert np.array_equal(r1[k], r4[k]), k
    assert np.array_equal(r1["seeds"], r4["seeds"])


@pytest.mark.parametrize("uvdd", [(3, -2, 5, 4), (-6, 3, 2, 9), (11, 0, 14, 12)])
def test_exact_recovery_of_integer_shifts(orc, uvdd):
    u, v, d0, d1 = uvdd
    q = scenegen.make_shift_quad(160, 96, 31, u=u, v=v, d0=d0, d1=d1)
    r = orc.run_quad(*q.images(), seed=3)
    fwd = r["fwd"].astype(np.int64)
    m = 40
    interior = fwd[m:-m, m:-m]
    assert (interior == np.array(uvdd)).all()
    # inverse field recovers the true inverse vector
    iu = np.array([-(u - d1 + d0), -v, d1, d0])
    assert (r["inv"].astype(np.int64)[m:-m, m:-m] == iu).all()
    # the interior is kept by the filter and its seeds are exact
    assert r["keep"][m:-m, m:-m].all()
    sd = r["seeds"]
    inner = (sd["x"] >= m) & (sd["x"] < 160 - m) & (sd["y"] >= m) & (sd["y"] < 96 - m)
    assert inner.sum() > 0
    assert (sd["u"][inner] == u).all() and (sd["d1"][inner] == d1).all()


def test_ground_truth_recovery_planes(orc):
    q = scenegen.make_named("planes_256x80", 1)
    r = orc.run_quad(*q.images(), seed=1234)
    vis = ~q.occluded
    keep = r["keep"].astype(bool) & vis
    err = np.abs(r["fwd"].astype(np.float64) - q.gt).max(-1)
    assert keep.sum() / vis.sum() > 0.8        # density of kept matches
    assert (err[keep] > 3).mean() < 0.03       # outliers among kept matches
