"""Pins of the oracle of the paper's own matching cost (Eq. 1 with SIFT-PCA
features): closed forms of the descriptor, the principal axes of data with
known variance directions, the cost's zero at the true vector, and the
matching on integer-shift scenes."""
import math

import numpy as np
import pytest

import oracle
import scenegen


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def test_orientation_bins():
    rays = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    for k, (dx, dy) in enumerate(rays):
        assert oracle.orientation_bin(3 * dx, 3 * dy) == k  # on a sector's first ray
    rng = np.random.default_rng(0)
    for dx, dy in rng.integers(-500, 500, (2000, 2)):
        a = math.degrees(math.atan2(dy, dx)) % 360.0
        if dx == 0 and dy == 0 or abs(a / 45.0 - round(a / 45.0)) < 1e-9:
            continue
        assert oracle.orientation_bin(dx, dy) == int(a // 45.0)


def test_descriptor_closed_forms():
    h, w = 40, 50
    assert (oracle.sift_descriptors(np.full((h, w, 3), 77, np.uint8), 0) == 0).all()
    ys, xs = np.mgrid[0:h, 0:w]
    for s, axis, k in ((0, "x", 0), (1, "x", 0), (0, "y", 2)):
        n = 1 << s
        g = (4 * (xs if axis == "x" else ys)).astype(np.uint8)
        img = np.repeat(g[..., None], 3, axis=2)
        d = oracle.sift_descriptors(img, s)
        # interior: every sample has the same gradient (8 n along the axis), so
        # every cell holds 9 * 8 n in one bin: 16 equal entries of 1/4, clipped
        # to 0.2, renormalised to 1/4, quantised to 128
        want = np.zeros(128, np.uint8)
        want[k::8] = 128
        m = 6 * n + n
        assert (d[m:h - m, m:w - m] == want).all()


def test_descriptor_cell_layout_on_a_ramp_that_ends_inside_a_cell():
    # grey 4 min(x, 21): at pixel (20, 20) the sample columns are 14..25 and
    # the gradient dx = g(q + 1) - g(q - 1) is 8 for q <= 20, 4 at q = 21 and
    # 0 beyond, dy = 0 (sector 0).  Cell columns 0..3 then hold 72, 72, 36
    # and 0 in every cell row: norm 216, so 1/3 (clipped to 0.2) and 1/6;
    # renormalised by sqrt(8 * 0.04 + 4 / 36), quantised to 156 and 130
    h, w = 40, 40
    g = np.repeat((4 * np.minimum(np.arange(w), 21)).astype(np.uint8)[None, :], h, axis=0)
    d = oracle.sift_descriptors(np.repeat(g[..., None], 3, axis=2), 0)[20, 20]
    want = np.zeros(128, np.uint8)
    for cy in range(4):
        for cx, val in enumerate((156, 156, 130, 0)):
            want[(cy * 4 + cx) * 8] = val
    assert np.array_equal(d, want)
    # the same edge seen along y: the cells' roles move from columns to rows
    dt = oracle.sift_descriptors(np.repeat(g.T[..., None], 3, axis=2), 0)[20, 20]
    want_t = np.zeros(128, np.uint8)
    for cy, val in enumerate((156, 156, 130, 0)):
        for cx in range(4):
            want_t[(cy * 4 + cx) * 8 + 2] = val
    assert np.array_equal(dt, want_t)


def test_principal_axes_of_known_variances():
    # a full factorial design: the three varying coordinates are exactly
    # uncorrelated, so the principal axes are the unit vectors, ordered by
    # variance
    a, b, c = np.meshgrid(np.arange(-60, 61, 20), np.arange(-30, 31, 10), np.arange(-10, 11, 5), indexing="ij")
    q = np.full((a.size, 128), 100, np.int32)
    q[:, 9], q[:, 0], q[:, 5] = 100 + a.ravel(), 100 + b.ravel(), 100 + c.ravel()
    desc = q.astype(np.uint8)
    mean, axes = oracle.sift_pca(desc)
    assert np.array_equal(mean, np.full(128, 100.0))
    want = np.zeros((3, 128))
    want[0, 9] = want[1, 0] = want[2, 5] = 1.0
    assert np.allclose(axes, want, atol=1e-12)
    phi = oracle.sift_project(desc, mean, axes)
    assert np.array_equal(phi[:, :3], np.stack([a.ravel(), b.ravel(), c.ravel()], 1).astype(np.float32))
    assert (phi[:, 3] == 0).all()


def test_principal_axes_agree_with_an_eigensolver():
    rng = np.random.default_rng(1)
    base = rng.integers(0, 60, (5000, 128))
    mix = rng.normal(size=(128, 128)) * (rng.random(128) < 0.05)
    desc = np.clip(base + (base @ mix) * 0.5, 0, 255).astype(np.uint8)
    mean, axes = oracle.sift_pca(desc)
    vals, vecs = np.linalg.eigh(np.cov(desc.T.astype(np.float64), bias=True))
    top = vecs[:, ::-1][:, :3].T
    for k in range(3):
        v = top[k] * np.sign(top[k][np.argmax(np.abs(top[k]))])
        assert np.allclose(axes[k], v, atol=1e-6), k
    phi = oracle.sift_project(desc, mean, axes)
    assert np.allclose(phi[:, :3], (desc - mean) @ axes.T, atol=2e-3)


def test_cost_is_zero_at_the_true_vector_and_clamps():
    q = scenegen.make_shift_quad(96, 64, 3, u=5, v=-2, d0=4, d1=7)
    phis, _, _ = oracle.sift_phi(q.images(), num_scales=1)
    L0, R0, L1, R1 = (p[0] for p in phis)
    truth = np.array([5, -2, 4, 7], np.int16)
    # interior pixels: every window pixel sees the same features in all views
    for px, py in ((40, 30), (60, 25), (30, 40)):
        assert oracle.sift_cost(L0, L1, R0, R1, 1, 0, px, py, truth) == 0.0
        assert oracle.sift_cost(L0, L1, R0, R1, 1, 0, px, py, truth + np.array([1, 0, 0, 0], np.int16)) > 0.0
    # far outside the image every position clamps to the same border pixels
    c1 = oracle.sift_cost(L0, L1, R0, R1, 1, 0, 40, 30, np.array([500, 0, 0, 0], np.int16))
    c2 = oracle.sift_cost(L0, L1, R0, R1, 1, 0, 40, 30, np.array([900, 0, 0, 0], np.int16))
    assert c1 == c2


def test_cost_sums_three_distances_over_a_7x7_window_at_stride_n():
    h, w = 40, 48
    zero = np.zeros((h, w, 4), np.float32)

    def const(a, b, c):
        x = np.zeros((h, w, 4), np.float32)
        x[..., :3] = (a, b, c)
        return x

    # constant features: every window pixel adds |(3, 4, 0)| = 5 (temporal),
    # |(0, 0, 2)| = 2 (stereo) and |(1, 2, 2)| = 3 (cross), exactly
    u = np.array([2, -1, 3, 5], np.int16)
    for n in (1, 2):
        assert oracle.sift_cost(zero, const(3, 4, 0), const(0, 0, 2), const(1, 2, 2), n, 0, 20, 20, u) == 49.0 * 10
    # one marked pixel in the temporal view, vector 0: it counts only where it
    # lies on the window's grid, offsets -3n .. 3n at stride n
    for n in (1, 2):
        for (ox, oy), hits in (((3 * n, -3 * n), 1), ((-3 * n, 2 * n), 1), ((4 * n, 0), 0), ((0, -4 * n), 0),
                               ((n + 1, 0), 1 if n == 1 else 0)):
            tmp = zero.copy()
            tmp[20 + oy, 24 + ox, :3] = (3.0, 4.0, 0.0)
            c = oracle.sift_cost(zero, tmp, zero, zero, n, 0, 24, 20, np.zeros(4, np.int16))
            assert c == 5.0 * hits, (n, ox, oy)


def test_matching_with_the_sift_cost_recovers_integer_shifts():
    q = scenegen.make_shift_quad(128, 96, 5, u=-3, v=2, d0=6, d1=4)
    p = oracle.default_params()
    feats = [oracle.features(im, p) for im in q.images()]
    phis, _, _ = oracle.sift_phi(q.images(), num_scales=p.num_scales)
    h, w = q.height, q.width
    (f0, _), (r0, _), (f1, _), (r1, _) = feats
    field, cost = oracle.match_views_sift(f0, f1, r0, r1, phis[0], phis[2], phis[1], phis[3], w, h, 0, 9, p)
    inner = field[20:-20, 20:-20].reshape(-1, 4)
    assert (inner == np.array([-3, 2, 6, 4])).all(axis=1).mean() > 0.99
    assert (cost.view(np.float32)[20:-20, 20:-20] >= 0).all()
