"""Pins of the interpolation oracle (Sec. 3.2): closed forms it must reproduce,
independent of its own formulas."""
import math

import numpy as np
import pytest

import oracle


def _seeds(rows):
    s = np.zeros(len(rows), oracle.SEED_DTYPE)
    for k, (x, y, u, v, d0, d1) in enumerate(rows):
        s[k]["x"], s[k]["y"], s[k]["u"], s[k]["v"], s[k]["d0"], s[k]["d1"] = x, y, u, v, d0, d1
    return s


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def _plane_motion_seeds(w, h, step=3, jitter_seed=1):
    # seeds sampled from a known scene: plane d0 = 40 + x - y, 3D motion
    # x1 = 0.5 x0 + (B/2, 0, 0): in the image u = d0, v = 0, d1 = 2 d0 (exact
    # integers at integer positions)
    rng = np.random.default_rng(jitter_seed)
    rows = []
    for by in range(0, h, step):
        for bx in range(0, w, step):
            x = min(w - 1, bx + int(rng.integers(0, step)))
            y = min(h - 1, by + int(rng.integers(0, step)))
            d0 = 40 + x - y
            rows.append((x, y, d0, 0, d0, 2 * d0))
    return _seeds(rows)


def test_exact_plane_and_affine_motion_are_reproduced_everywhere():
    w, h, f, B = 48, 30, 300.0, 0.5
    s = _plane_motion_seeds(w, h)
    p = oracle.interp_params(w, h, f, B, k_geo=40, k_motion=24)
    out = oracle.interpolate(s, w, h, p)
    ys, xs = np.mgrid[0:h, 0:w]
    d0 = 40.0 + xs - ys
    assert np.allclose(out[..., 2], d0, atol=1e-3)      # plane
    assert np.allclose(out[..., 0], d0, atol=1e-3)      # u = d0 from the X translation
    assert np.allclose(out[..., 1], 0.0, atol=1e-3)     # v
    assert np.allclose(out[..., 3], 2 * d0, atol=1e-3)  # d1 from Z halved


def test_weighted_plane_of_a_symmetric_star():
    # the seed at (10, 10) with d0 = 0 and four neighbours 3 px away with
    # d0 = 6: by symmetry the plane is flat at the weighted mean
    # 4 * 6 w / (1 + 4 w), w = exp(-alpha * 3 / dist_unit)
    s = _seeds([(10, 10, 0, 0, 0, 0), (13, 10, 0, 0, 6, 0), (7, 10, 0, 0, 6, 0), (10, 13, 0, 0, 6, 0),
                (10, 7, 0, 0, 6, 0)])
    p = oracle.interp_params(32, 32, 300.0, 0.5, k_geo=5, k_motion=5)
    plane, _, _ = oracle.seed_models(s, p)
    wgt = math.exp(-2.2 * 3 / 20.0)
    want = 24 * wgt / (1 + 4 * wgt)
    assert plane[0][0] == pytest.approx(0.0, abs=1e-6)  # slopes (coordinates centred at the seed)
    assert plane[0][1] == pytest.approx(0.0, abs=1e-6)
    assert plane[0][2] == pytest.approx(want, abs=1e-6)


def test_neighbourhood_on_a_lattice_and_ties():
    # seeds on a 3-px lattice: the 5 nearest to a lattice point are itself and
    # its 4 axis neighbours; with k = 3 the tie at distance 3 goes to the lower
    # seed indices (raster order: the upper, then the left neighbour)
    rows = [(x, y, 0, 0, 5, 5) for y in range(0, 15, 3) for x in range(0, 15, 3)]
    s = _seeds(rows)
    centre = rows.index((6, 6, 0, 0, 5, 5))
    idx, d2 = oracle.nearest_seeds(s, 6, 6, 5)
    assert idx[0] == centre and d2[0] == 0
    assert sorted((rows[i][0], rows[i][1]) for i in idx[1:]) == [(3, 6), (6, 3), (6, 9), (9, 6)]
    assert list(d2[1:]) == [9, 9, 9, 9]
    idx3, _ = oracle.nearest_seeds(s, 6, 6, 3)
    assert [(rows[i][0], rows[i][1]) for i in idx3] == [(6, 6), (6, 3), (3, 6)]


def _circle_offsets(r2):
    """The lattice points (dx, dy) with dx^2 + dy^2 = r2."""
    r = math.isqrt(r2)
    return [(dx, dy) for dx in range(-r, r + 1) for dy in range(-r, r + 1) if dx * dx + dy * dy == r2]


def test_more_than_32_seeds_tied_at_the_kth_distance():
    # 5525 = 5^2 * 13 * 17 is a sum of two squares in 48 ways (4 (3 * 2 * 2)
    # lattice points), so a seed at the centre of that circle sees 48 seeds
    # tied at its k-th distance; listed in a shuffled order, the neighbourhood
    # is the centre and the k - 1 tied seeds of lowest index, by brute force
    circle = _circle_offsets(5525)
    assert len(circle) == 48
    rng = np.random.default_rng(5525)
    rows = [(85 + dx, 80 + dy, 0, 0, 20, 20) for dx, dy in circle] + [(85, 80, 0, 0, 20, 20)]
    rows = [rows[i] for i in rng.permutation(len(rows))]
    s = _seeds(rows)
    d2 = (s["x"].astype(np.int64) - 85) ** 2 + (s["y"].astype(np.int64) - 80) ** 2
    brute = np.lexsort((np.arange(len(s)), d2))
    for k in (1, 2, 10, 33, 48, 49):
        idx, dk = oracle.nearest_seeds(s, 85, 80, k)
        assert list(idx) == list(brute[:k])
        assert list(dk) == list(d2[brute[:k]])
        assert sorted(idx[1:]) == list(idx[1:])  # the tied seeds in index order


def test_reprojection_at_unit_disparity():
    # every seed at d0 = d1 = 1 (depth f B) moving 3 px right: the 3D motion
    # is the translation (3 B, 0, 0) and the plane d0 = 1, so every pixel is
    # reprojected at max(d0, 1) = 1 and moves by exactly (3, 0) with d1 = 1
    rows = [(x, y, 3, 0, 1, 1) for y in range(1, 24, 3) for x in range(1, 30, 3)]
    s = _seeds(rows)
    out = oracle.interpolate(s, 30, 24, oracle.interp_params(30, 24, 400.0, 0.5, k_geo=12, k_motion=8))
    np.testing.assert_allclose(out[..., 0], 3.0, atol=1e-6)
    np.testing.assert_allclose(out[..., 1], 0.0, atol=1e-6)
    np.testing.assert_allclose(out[..., 2], 1.0, atol=1e-6)
    np.testing.assert_allclose(out[..., 3], 1.0, atol=1e-6)
    # a plane that falls below 1: seed A (5, 10) at d0 = 1 moving 3 px, seed B
    # (15, 10) at d0 = 3 tilts A's plane to 1 + 0.2 (x - 5), 0.4 at x = 2;
    # the reprojection uses max(d0, 1) = 1, so A's translation still moves the
    # pixel by exactly 3 px with d1 = 1 (at depth f B / 0.4 it would be 1.2 px)
    s2 = _seeds([(5, 10, 3, 0, 1, 1), (15, 10, 0, 0, 3, 3)])
    p2 = oracle.interp_params(21, 21, 300.0, 0.5, k_geo=2, k_motion=1)
    o2, closest = oracle.interpolate_pixels(s2, p2, [[2, 10]])
    assert list(closest) == [0]
    np.testing.assert_allclose(o2[0], [3.0, 0.0, 0.4, 1.0], atol=1e-5)


def test_points_moved_behind_the_camera_get_no_flow():
    # seed A at (5, 10) with d0 = 2 and d1 = 40 (depth f B / 2 -> f B / 40:
    # its own translation is -0.475 f B in Z); seed B at (15, 10) with d0 = 12
    # tilts A's plane to d0 = 2 + (x - 5).  At x = 9, closest to A, the plane
    # gives d0 = 6, depth f B / 6 < 0.475 f B: the moved point is behind the
    # camera, so u = v = 0 and d1 = d0 there; at x = 5 it is A's own motion
    s = _seeds([(5, 10, 0, 0, 2, 40), (15, 10, 0, 0, 12, 13)])
    f, B = 300.0, 0.5
    p = oracle.interp_params(21, 21, f, B, k_geo=2, k_motion=1)
    out, closest = oracle.interpolate_pixels(s, p, [[9, 10], [5, 10]])
    assert list(closest) == [0, 0]
    np.testing.assert_allclose(out[0], [0.0, 0.0, 6.0, 6.0], atol=1e-5)
    np.testing.assert_allclose(out[1], [0.0, 0.0, 2.0, 40.0], atol=1e-5)


def test_motion_neighbourhood_skips_seeds_that_cannot_be_triangulated():
    s = _seeds([(5, 5, 0, 0, 4, 4), (6, 5, 0, 0, 0, 4), (7, 5, 0, 0, 4, 0), (9, 5, 0, 0, 3, 3)])
    idx, _ = oracle.nearest_seeds(s, 5, 5, 4, motion_only=True)
    assert list(idx) == [0, 3]
    _, _, motion = oracle.seed_models(s, oracle.interp_params(16, 16, 300.0, 0.5))
    assert list(motion) == [2, 2, 2, 2]


def test_closest_seed_ties_go_to_the_lower_index():
    s = _seeds([(2, 4, 0, 0, 7, 7), (6, 4, 0, 0, 9, 9)])
    p = oracle.interp_params(9, 9, 300.0, 0.5, k_geo=1, k_motion=1)
    out, closest = oracle.interpolate_pixels(s, p, [[4, 4], [5, 4], [3, 4]])
    assert list(closest) == [0, 1, 0]
    # one neighbour: a flat plane at the seed's own disparity (the ridge on
    # the slopes keeps the system solvable)
    assert out[0][2] == pytest.approx(7.0, abs=1e-4)
    assert out[1][2] == pytest.approx(9.0, abs=1e-4)


def test_no_motion_neighbours_gives_zero_flow_and_equal_disparities():
    s = _seeds([(4, 4, 3, 1, 6, 0)])  # d1 = 0: not a motion seed
    p = oracle.interp_params(8, 8, 300.0, 0.5)
    out, _ = oracle.interpolate_pixels(s, p, [[4, 4]])
    assert out[0][0] == 0 and out[0][1] == 0
    assert out[0][3] == pytest.approx(out[0][2])


def test_single_motion_neighbour_is_a_translation():
    # one motion seed: A defaults to the identity, the map is the seed's 3D
    # translation; the pixel at the seed itself moves exactly like the seed
    s = _seeds([(6, 5, 3, -2, 8, 10)])
    p = oracle.interp_params(16, 12, 300.0, 0.5)
    out, _ = oracle.interpolate_pixels(s, p, [[6, 5]])
    assert out[0] == pytest.approx([3.0, -2.0, 8.0, 10.0], abs=1e-4)


def test_models_of_listed_seeds_equal_the_full_fit():
    s = _plane_motion_seeds(40, 28, jitter_seed=3)
    s["d0"][::5] += 3  # not an exact plane any more
    p = oracle.interp_params(40, 28, 300.0, 0.5, k_geo=25, k_motion=12)
    full = oracle.seed_models(s, p)
    which = [0, 7, 7, len(s) - 1, 30]
    part = oracle.seed_models(s, p, which=which)
    for a, b in zip(full, part):
        assert np.array_equal(a[sorted(set(which))], b[sorted(set(which))])
    rest = np.setdiff1d(np.arange(len(s)), which)
    assert (part[0][rest] == 0).all() and (part[2][rest] == 0).all()


def test_synthetic_seeds_have_the_structure_of_sparse_matches():
    import scenegen
    gt, occ, f, B = scenegen.ground_truth("driving", 121, 47, 2)
    s = scenegen.sparse_seeds(gt, occ, 4, keep=0.7, noise=1.0, outliers=0.1)
    assert s.dtype.itemsize == 20 and s.dtype == oracle.SEED_DTYPE
    blk = (s["y"] // 3) * (-(-121 // 3)) + s["x"] // 3
    assert (np.diff(blk) > 0).all()  # one per 3x3 block, block raster order
    assert (s["x"] >= 0).all() and (s["x"] < 121).all() and (s["y"] >= 0).all() and (s["y"] < 47).all()
    assert (s["d0"] >= 0).all() and (s["d1"] >= 0).all()
    assert not occ[s["y"], s["x"]].any()
    exact = scenegen.sparse_seeds(gt, occ, 4, keep=0.7)
    assert np.array_equal(exact["d0"], np.rint(gt[exact["y"], exact["x"], 2]))


def test_fits_agree_with_weighted_least_squares():
    # random non-degenerate seeds: the ridge (1e-9 of the trace) is negligible,
    # so every seed's plane and affine map are numpy's weighted least-squares
    # solutions over the same neighbours with the same weights
    rng = np.random.default_rng(7)
    rows = []
    for by in range(0, 36, 3):
        for bx in range(0, 48, 3):
            if rng.random() < 0.7:
                x, y = bx + int(rng.integers(0, 3)), by + int(rng.integers(0, 3))
                rows.append((x, y, int(rng.integers(-9, 10)), int(rng.integers(-5, 6)), int(rng.integers(5, 60)),
                             int(rng.integers(5, 60))))
    s = _seeds(rows)
    f, B = 400.0, 0.5
    p = oracle.interp_params(48, 36, f, B, k_geo=25, k_motion=15)
    plane, affine, motion = oracle.seed_models(s, p)
    cx, cy = p.cx, p.cy

    def tri(x, y, d):
        Z = f * B / d
        return np.array([(x - cx) * Z / f, (y - cy) * Z / f, Z])

    for i in rng.choice(len(s), 25, replace=False):
        sx, sy = int(s["x"][i]), int(s["y"][i])
        idx, d2 = oracle.nearest_seeds(s, sx, sy, 25)
        w = np.exp(-2.2 * np.sqrt(d2.astype(np.float64)) / 20.0)
        A = np.stack([s["x"][idx] - sx, s["y"][idx] - sy, np.ones(len(idx))], 1).astype(np.float64)
        sol = np.linalg.lstsq(A * np.sqrt(w)[:, None], s["d0"][idx] * np.sqrt(w), rcond=None)[0]
        assert np.allclose(plane[i], sol, rtol=1e-7, atol=1e-7)
        idx, d2 = oracle.nearest_seeds(s, sx, sy, 15, motion_only=True)
        w = np.exp(-2.2 * np.sqrt(d2.astype(np.float64)) / 20.0)
        X0 = np.array([tri(s["x"][j], s["y"][j], s["d0"][j]) for j in idx])
        X1 = np.array([tri(s["x"][j] + s["u"][j], s["y"][j] + s["v"][j], s["d1"][j]) for j in idx])
        c = (w[:, None] * X0).sum(0) / w.sum()
        D = np.concatenate([X0 - c, np.ones((len(idx), 1))], 1)
        # normal equations with the ridge of the reading (1e-9 trace / 4 on the
        # linear part, towards A = I), solved by numpy: with depths of 3-40 m
        # the ridge moves A by ~1e-5 relative, so it is part of the check
        N = (D * w[:, None]).T @ D
        R = (D * w[:, None]).T @ X1  # [4, 3]
        lam = 1e-9 * np.trace(N) / 4
        for a in range(3):
            N[a, a] += lam
            R[a, a] += lam
        At = np.linalg.solve(N, R)  # [4, 3]: rows of A^T, then t
        assert motion[i] == len(idx)
        assert np.allclose(affine[i][12:], c, rtol=1e-10, atol=1e-10)
        assert np.allclose(affine[i][:12].reshape(3, 4), At.T, rtol=1e-8, atol=1e-8)
        # and without the ridge the weighted least-squares solution is within
        # the ridge's reach
        Aw = np.linalg.lstsq(D * np.sqrt(w)[:, None], X1 * np.sqrt(w)[:, None], rcond=None)[0]
        assert np.allclose(affine[i][:12].reshape(3, 4), Aw.T, rtol=1e-3, atol=1e-3)
