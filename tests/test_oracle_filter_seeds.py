"""Pins of the oracle's consistency check, region filter (Sec. 3.1) and
3x3 sparsification (Sec. 3.2): closed-form fields, invariants, and scipy /
numpy restatements of connected components and block argmins."""
import numpy as np
import pytest

EMPTY = np.iinfo(np.int32).max


def _const_fields(h, w, u, v, d0, d1):
    fwd = np.broadcast_to(np.array([u, v, d0, d1], np.int16), (h, w, 4)).copy()
    inv = np.broadcast_to(np.array([-(u - d1 + d0), -v, d1, d0], np.int16), (h, w, 4)).copy()
    c = np.zeros((h, w), np.int32)
    return fwd, c, inv, c.copy()


def test_exact_inverse_passes(orc):
    h, w = 30, 50
    fwd, fc, inv, ic = _const_fields(h, w, 3, -2, 5, 4)
    keep, cerr = orc.consistency_check(fwd, fc, inv, ic)
    ys, xs = np.mgrid[0:h, 0:w]
    qx, qy = xs + 3 - 4, ys - 2
    inside = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
    assert np.array_equal(keep.astype(bool), inside)
    assert (cerr[inside] == 0).all() and (cerr[~inside] == 255).all()


@pytest.mark.parametrize("comp", [0, 1, 2, 3])
@pytest.mark.parametrize("delta", [1, 2, -2])
def test_perturbation_threshold(orc, comp, delta):
    h, w = 20, 24
    fwd, fc, inv, ic = _const_fields(h, w, 2, 1, 4, 3)
    inv[..., comp] += delta
    keep, cerr = orc.consistency_check(fwd, fc, inv, ic)
    ys, xs = np.mgrid[0:h, 0:w]
    inside = (xs + 2 - 3 >= 0) & (xs + 2 - 3 < w) & (ys + 1 < h)
    assert np.array_equal(keep.astype(bool), inside & (abs(delta) <= 1))
    assert (cerr[inside] == abs(delta)).all()


def test_consistency_error_saturates_at_255(orc):
    # cerr is the sum of the four absolute round-trip differences, saturated
    # to a byte: one component off by 200 gives 200, by 300 gives 255
    h, w = 12, 16
    for delta, want in ((200, 200), (254, 254), (255, 255), (300, 255)):
        fwd, fc, inv, ic = _const_fields(h, w, 1, 0, 2, 2)
        inv[..., 0] += delta
        keep, cerr = orc.consistency_check(fwd, fc, inv, ic)
        assert not keep.any()
        # column 0's cross match (x + u - d1 = -1) is outside: 255 untested
        assert (cerr[:, 1:] == want).all() and (cerr[:, 0] == 255).all(), delta


def test_empty_vectors_rejected(orc):
    h, w = 10, 12
    fwd, fc, inv, ic = _const_fields(h, w, 0, 0, 1, 1)
    fc[2, 3] = EMPTY
    ic[5, 4] = EMPTY  # R1 pixel (x=4, y=5), the cross match of L0 pixel (x=5, y=5)
    keep, cerr = orc.consistency_check(fwd, fc, inv, ic)
    assert keep[2, 3] == 0 and cerr[2, 3] == 255
    assert keep[5, 5] == 0 and cerr[5, 5] == 255


def _expected_region_filter(fwd_piece, keep0, rejected, smin):
    """Components of kept pixels within one piece (vectors of different
    pieces differ by more than tau_r), by scipy.ndimage.label."""
    import scipy.ndimage as ndi
    keep = keep0.copy()
    h, w = keep.shape
    for pid in np.unique(fwd_piece):
        lab, n = ndi.label(keep0 & (fwd_piece == pid))
        for k in range(1, n + 1):
            m = lab == k
            grown = ndi.binary_dilation(m, structure=ndi.generate_binary_structure(2, 1))
            joinable = (grown & ~m & rejected & (fwd_piece == pid)).any()
            if joinable and m.sum() < smin:
                keep[m] = False
    return keep


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_region_filter_matches_component_labelling(orc, seed):
    rng = np.random.default_rng(seed)
    h, w = 60, 80
    # piecewise-constant field from random rectangles; pieces differ by 3 in u
    piece = np.zeros((h, w), np.int64)
    for k in range(1, 12):
        y0, x0 = rng.integers(0, h), rng.integers(0, w)
        piece[y0:y0 + rng.integers(3, 30), x0:x0 + rng.integers(3, 40)] = k
    fwd = np.zeros((h, w, 4), np.int16)
    fwd[..., 0] = 3 * piece
    fc = np.zeros((h, w), np.int32)
    fc[rng.random((h, w)) < 0.02] = EMPTY
    keep0 = (rng.random((h, w)) > 0.15) & (fc != EMPTY)
    rejected = ~keep0 & (fc != EMPTY)
    p = orc.default_params(region_min=40)
    got = orc.region_filter(fwd, fc, keep0.astype(np.uint8), p).astype(bool)
    exp = _expected_region_filter(piece, keep0, rejected, 40)
    assert np.array_equal(got, exp)
    assert not (got & ~keep0).any()  # filtering never adds pixels


def test_region_filter_hand_built(orc):
    h, w = 40, 40
    fwd = np.zeros((h, w, 4), np.int16)
    fc = np.zeros((h, w), np.int32)
    keep = np.zeros((h, w), np.uint8)
    # A: 5x5 region, vector (9,0,0,0), next to rejected pixels with the same vector -> removed
    fwd[2:9, 2:9, 0] = 9
    keep[3:8, 3:8] = 1
    # B: 5x5 region, vector (20,..), rejected neighbours differ by 2 -> kept
    fwd[12:19, 2:9, 0] = 22
    fwd[13:18, 3:8, 0] = 20
    keep[13:18, 3:8] = 1
    # C: 13x13 = 169 >= 150 region with joinable rejected neighbours -> kept
    fwd[20:40, 20:40, 0] = 5
    keep[22:35, 22:35] = 1
    # D: 5x5 region with vector (30,..) surrounded by EMPTY pixels only -> kept
    fwd[2:9, 20:27, 0] = 30
    fc[2:9, 20:27] = EMPTY
    fc[3:8, 21:26] = 0
    keep[3:8, 21:26] = 1
    out = orc.region_filter(fwd, fc, keep, orc.default_params()).astype(bool)
    assert not out[3:8, 3:8].any()
    assert out[13:18, 3:8].all()
    assert out[22:35, 22:35].all()
    assert out[3:8, 21:26].all()


def test_region_of_exactly_s_c_pixels_is_kept(orc):
    # two regions with joinable rejected neighbours: 10 x 15 = 150 = s_c
    # pixels (kept) and the same less one corner, 149 pixels (removed)
    h, w = 40, 60
    fwd = np.zeros((h, w, 4), np.int16)
    fc = np.zeros((h, w), np.int32)
    keep = np.zeros((h, w), np.uint8)
    fwd[1:14, 1:19, 0] = 7
    keep[2:12, 2:17] = 1
    fwd[20:33, 30:48, 0] = 11
    keep[21:31, 31:46] = 1
    keep[21, 31] = 0
    assert keep[2:12, 2:17].sum() == 150 and keep[21:31, 31:46].sum() == 149
    out = orc.region_filter(fwd, fc, keep, orc.default_params()).astype(bool)
    assert out[2:12, 2:17].all()
    assert not out[21:31, 31:46].any()


def test_seeds_block_argmin(orc):
    rng = np.random.default_rng(4)
    for (h, w) in [(30, 45), (31, 47), (7, 8), (3, 3), (10, 10)]:
        fwd = rng.integers(-50, 50, (h, w, 4)).astype(np.int16)
        cost = rng.integers(0, 5, (h, w)).astype(np.int32)
        keep = (rng.random((h, w)) > 0.4).astype(np.uint8)
        cerr = rng.integers(0, 3, (h, w)).astype(np.uint8)
        sd = orc.emit_seeds(fwd, cost, keep, cerr)
        exp = []
        for by in range(0, h, 3):
            for bx in range(0, w, 3):
                cands = [(int(cerr[y, x]), int(cost[y, x]), y * w + x, x, y)
                         for y in range(by, min(by + 3, h)) for x in range(bx, min(bx + 3, w)) if keep[y, x]]
                if cands:
                    exp.append(min(cands))
        assert len(sd) == len(exp)
        for s, e in zip(sd, exp):
            x, y = e[3], e[4]
            assert (s["x"], s["y"]) == (x, y)
            assert (s["u"], s["v"], s["d0"], s["d1"]) == tuple(fwd[y, x])
            assert s["cost"] == cost[y, x] and s["cerr"] == cerr[y, x]


def test_filter_never_adds(orc):
    import scenegen
    q = scenegen.make_named("planes_256x80", 2)
    r = orc.run_quad(*q.images(), seed=5)
    k0, _ = orc.consistency_check(r["fwd"], r["fwd_cost"], r["inv"], r["inv_cost"])
    assert not (r["keep"].astype(bool) & ~k0.astype(bool)).any()
    assert (r["cerr"][r["keep"].astype(bool)] <= 4).all()
