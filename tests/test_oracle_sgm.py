"""Pins of the disparity-fill oracle (Sec. 3.1, last paragraph): semi-global
matching of L0/R0 and the disparity-only seeds, against closed forms, brute
force and special cases that reduce to a library routine."""
import itertools

import numpy as np
import pytest

import oracle
import scenegen


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def _window_bits(pred):
    """Census word with the bits of the 9x7 window positions (i, j) for which
    pred(i, j) holds, in row-major window order with the centre skipped."""
    bits, k = 0, 0
    for j in range(-3, 4):
        for i in range(-4, 5):
            if i == 0 and j == 0:
                continue
            if pred(i, j):
                bits |= 1 << k
            k += 1
    return bits


def test_grey_and_census_closed_forms():
    rgb = np.zeros((20, 30, 3), np.uint8)
    rgb[..., 0], rgb[..., 1], rgb[..., 2] = 10, 20, 30
    assert (oracle.grey(rgb) == (10 + 40 + 30 + 2) >> 2).all()
    assert (oracle.census(oracle.grey(rgb)) == 0).all()  # nothing darker than the centre
    ys, xs = np.mgrid[0:20, 0:30]
    ramp_x = (5 * xs).astype(np.uint8)
    c = oracle.census(ramp_x)
    assert (c[3:-3, 4:-4] == _window_bits(lambda i, j: i < 0)).all()  # the left half is darker
    assert (c[:, 0] == 0).all()  # clamped: no neighbour is darker at the left border
    ramp_y = (7 * ys).astype(np.uint8)
    assert (oracle.census(ramp_y)[3:-3, 4:-4] == _window_bits(lambda i, j: j < 0)).all()


def test_census_depends_on_the_order_of_grey_values_only():
    g = np.random.default_rng(1).integers(0, 120, (25, 33)).astype(np.uint8)
    mono = (2 * g.astype(np.int32) + 7).astype(np.uint8)  # strictly increasing map
    assert np.array_equal(oracle.census(g), oracle.census(mono))


def _brute_path(C, p1, p2):
    """Minimum over all disparity sequences along a line of the summed costs
    plus penalties (0 / P1 / P2 for a change of 0 / 1 / more), per end
    disparity; C [n, D]."""
    n, D = C.shape
    best = np.full(D, np.iinfo(np.int64).max)
    for seq in itertools.product(range(D), repeat=n):
        c = sum(int(C[t, seq[t]]) for t in range(n))
        for t in range(1, n):
            step = abs(seq[t] - seq[t - 1])
            c += 0 if step == 0 else (p1 if step == 1 else p2)
        best[seq[-1]] = min(best[seq[-1]], c)
    return best


def test_a_single_preference_travels_along_the_eight_rays():
    # a flat cost volume with one pixel q0 that prefers d* = 5: only the path
    # of direction r reaches q0 + k r through q0, so the sum over the 8
    # directions prefers d* exactly on the 8 rays from q0 (and at q0); every
    # other pixel sees flat sums and takes the lowest disparity, 0
    H, W, D, dstar = 21, 23, 8, 5
    C = np.full((H, W, D), 6, np.uint8)
    qy, qx = 10, 11
    C[qy, qx] = 30
    C[qy, qx, dstar] = 0
    disp = oracle.sgm_from_cost(C, 10, 120)
    want = np.zeros((H, W), np.int16)
    for rx, ry in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]:
        k = 0
        while 0 <= qx + k * rx < W and 0 <= qy + k * ry < H:
            want[qy + k * ry, qx + k * rx] = dstar
            k += 1
    assert np.array_equal(disp, want)


@pytest.mark.parametrize("rx,ry", [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)])
def test_path_costs_are_shortest_paths(rx, ry):
    # L_r(p, .) equals the brute-force minimum over disparity sequences along
    # the line ending at p, up to a constant per pixel (the subtracted minima)
    rng = np.random.default_rng(3 * (rx + 1) + (ry + 1))
    H, W, D, p1, p2 = 4, 5, 3, 3, 8
    C = rng.integers(0, 12, (H, W, D)).astype(np.uint8)
    L = oracle.path_costs(C, p1, p2, rx, ry).astype(np.int64)
    for y in range(H):
        for x in range(W):
            line = [(x, y)]
            while 0 <= line[-1][0] - rx < W and 0 <= line[-1][1] - ry < H:
                line.append((line[-1][0] - rx, line[-1][1] - ry))
            line = line[::-1]
            b = _brute_path(np.array([C[yy, xx] for xx, yy in line]), p1, p2)
            assert np.array_equal(L[y, x] - L[y, x].min(), b - b.min()), (x, y)
            # the exact normalised values: the brute-force minimum ending at p
            # less the one ending at p - r (C itself at the first pixel)
            prev = _brute_path(np.array([C[yy, xx] for xx, yy in line[:-1]]), p1, p2).min() if len(line) > 1 else 0
            assert np.array_equal(L[y, x], b - prev), (x, y)


def test_no_penalties_is_winner_takes_all():
    C = np.random.default_rng(3).integers(0, 9, (6, 11, 16)).astype(np.uint8)
    assert np.array_equal(oracle.sgm_from_cost(C, 0, 0), np.argmin(C, axis=2))


@pytest.mark.parametrize("d0", [0, 5, 23])
def test_integer_shift_is_recovered(d0):
    q = scenegen.make_shift_quad(120, 60, 10 + d0, u=1, v=0, d0=d0, d1=d0)
    disp = oracle.sgm(q.L0, q.R0, oracle.sgm_params(max_disp=32))
    assert (disp[3:-3, d0 + 4:-4] == d0).all()


def _blocks():
    # a 9 x 6 image, blocks (0, 0) (1, 0) (2, 0) on top, (0, 1) (1, 1) (2, 1) below
    h, w = 6, 9
    fwd = np.zeros((h, w, 4), np.int16)
    fwd[..., 0], fwd[..., 1], fwd[..., 3] = 3, -1, 12
    fwd[..., 2] = 10
    cost = np.full((h, w), 500, np.int32)
    keep = np.zeros((h, w), np.uint8)
    cerr = np.zeros((h, w), np.uint8)
    sgm = np.full((h, w), 30, np.int16)  # disagrees everywhere unless set
    keep[1, 1], cerr[1, 1] = 1, 2         # block (0, 0): a joint seed
    sgm[0, 0] = 10                        # ... whose disparity-only pixel is ignored
    sgm[0, 4], sgm[2, 3] = 11, 10         # block (1, 0): |d| 1 at (4, 0), 0 at (3, 2) -> (3, 2)
    sgm[1, 7] = 12                        # block (2, 0): |d| 2 > tau_c -> no seed
    sgm[4, 0], sgm[5, 2] = 9, 11          # block (0, 1): both |d| 1, cost decides -> (2, 5)
    cost[5, 2] = 400
    sgm[3, 4], sgm[4, 3] = 10, 10         # block (1, 1): tie in |d| and cost -> raster first (4, 3)
    cost[3:6, 6:9] = 2147483647           # block (2, 1): no vectors although sgm agrees
    sgm[3:6, 6:9] = 10
    return fwd, cost, keep, cerr, sgm


def test_disparity_only_seeds_on_hand_built_blocks():
    fwd, cost, keep, cerr, sgm = _blocks()
    s = oracle.emit_seeds_geo(fwd, cost, keep, cerr, sgm, tau_c=1)
    got = [(int(r["x"]), int(r["y"]), int(r["kind"]), int(r["u"]), int(r["d0"]), int(r["d1"]), int(r["cerr"]))
           for r in s]
    assert got == [(1, 1, 0, 3, 10, 12, 2), (3, 2, 1, 0, 10, 0, 0), (2, 5, 1, 0, 10, 0, 1), (4, 3, 1, 0, 10, 0, 0)]


def test_without_agreement_the_joint_seeds_remain():
    q = scenegen.make_named("planes_256x80", 1)
    ref = oracle.run_quad(*q.images(), seed=1)
    never = np.full(ref["fwd_cost"].shape, -100, np.int16)
    s = oracle.emit_seeds_geo(ref["fwd"], ref["fwd_cost"], ref["keep"], ref["cerr"], never, tau_c=1)
    assert s.tobytes() == ref["seeds"].tobytes()
    # with the fill, every block that had a joint seed keeps it, and more blocks get one
    disp = oracle.sgm(q.L0, q.R0, oracle.sgm_params(max_disp=64))
    g = oracle.emit_seeds_geo(ref["fwd"], ref["fwd_cost"], ref["keep"], ref["cerr"], disp, tau_c=1)
    assert g[g["kind"] == 0].tobytes() == ref["seeds"].tobytes()
    assert (g["kind"] == 1).sum() > 0
    assert (g[g["kind"] == 1][["u", "v", "d1"]].tolist() == [(0, 0, 0)] * int((g["kind"] == 1).sum()))
