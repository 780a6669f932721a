"""Pins of the oracle's scale space and Walsh-Hadamard features (Sec. 3.1).

The oracle builds the sequency-ordered Walsh matrix by sorting Sylvester
Hadamard rows by their sign changes; here it is checked against the
independent closed form (row k of the sequency order is natural Hadamard row
bitreverse(gray(k))), against transform identities on hand-built patches, and
against numpy/scipy restatements of the smoothing and of H P H^T.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def walsh_closed_form():
    """Sequency-ordered Walsh matrix: natural Hadamard row bitrev3(gray(k))."""
    def bitrev3(x):
        return ((x & 1) << 2) | (x & 2) | ((x >> 2) & 1)
    W = np.zeros((8, 8), np.int64)
    for k in range(8):
        m = bitrev3(k ^ (k >> 1))
        for j in range(8):
            W[k, j] = -1 if bin(m & j).count("1") % 2 else 1
    return W


def golden_order():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "wht_coef_order.txt")) if l.strip() and l[0] != "#"]
    return np.array([[int(a), int(b)] for _, a, b in rows])


def test_walsh_matrix_closed_form(orc):
    W = orc.walsh_matrix().astype(np.int64)
    assert np.array_equal(W, walsh_closed_form())
    assert np.array_equal(W @ W.T, 8 * np.eye(8, dtype=np.int64))
    for k in range(8):  # sequency: row k changes sign exactly k times
        assert int(np.sum(W[k, 1:] != W[k, :-1])) == k


def test_2d_basis_orthogonality(orc):
    # HH^T = 64 I for the 2-D (Kronecker) basis of 8x8 patches
    W = walsh_closed_form()
    K = np.kron(W, W)
    assert np.array_equal(K @ K.T, 64 * np.eye(64, dtype=np.int64))


def test_coef_order_golden(orc):
    ky, kx = orc.coef_order()
    assert np.array_equal(np.stack([ky, kx], 1), golden_order())


@pytest.mark.parametrize("c", [0, 1, 77, 255])
def test_constant_patch(orc, c):
    T = orc.wht8x8(np.full((8, 8), c))
    exp = np.zeros((8, 8), np.int64)
    exp[0, 0] = 64 * c
    assert np.array_equal(T, exp)


@pytest.mark.parametrize("ky,kx", [(0, 1), (1, 0), (3, 5), (7, 7), (4, 2)])
def test_walsh_basis_patch(orc, ky, kx):
    W = walsh_closed_form()
    patch = 128 + 63 * np.outer(W[ky], W[kx])
    T = orc.wht8x8(patch).astype(np.int64)
    exp = np.zeros((8, 8), np.int64)
    exp[0, 0] = 64 * 128
    exp[ky, kx] = 63 * 64
    assert np.array_equal(T, exp)


def test_parseval_and_matmul(orc):
    rng = np.random.default_rng(0)
    W = walsh_closed_form()
    for _ in range(50):
        P = rng.integers(0, 256, (8, 8)).astype(np.int64)
        T = orc.wht8x8(P).astype(np.int64)
        assert np.array_equal(T, W @ P @ W.T)
        assert (T ** 2).sum() == 64 * (P ** 2).sum()


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_box_smoothing(orc, s):
    import scipy.ndimage as ndi
    rng = np.random.default_rng(s)
    img = rng.integers(0, 256, (23, 37, 3)).astype(np.uint8)
    out = orc.smooth(img, s)
    n = 1 << s
    if s == 0:
        assert np.array_equal(out, img)
        return
    # window -n/2 .. n/2-1 with edge replication == scipy's centred even window, mode 'nearest'
    sums = ndi.uniform_filter(img.astype(np.float64) * n * n, size=(n, n, 1), mode="nearest")
    sums = np.rint(sums).astype(np.int64)
    exp = (sums + n * n // 2) // (n * n)
    assert np.array_equal(out, exp.astype(np.uint8))
    # a constant image stays constant
    assert np.all(orc.smooth(np.full((9, 11, 3), 200, np.uint8), s) == 200)


def features_numpy(img, s, qshift, x, y):
    """Feature vector of pixel (x, y) at scale s by the definition, numpy."""
    import scipy.ndimage as ndi
    h, w, _ = img.shape
    n = 1 << s
    if s:
        sums = np.rint(ndi.uniform_filter(img.astype(np.float64) * n * n, size=(n, n, 1), mode="nearest")).astype(np.int64)
        sm = (sums + n * n // 2) // (n * n)
    else:
        sm = img.astype(np.int64)
    W = walsh_closed_form()
    order = golden_order()
    out = []
    for c in range(3):
        P = np.array([[sm[min(max(y + n * (i - 3), 0), h - 1), min(max(x + n * (j - 3), 0), w - 1), c]
                       for j in range(8)] for i in range(8)])
        T = W @ P @ W.T
        for ky, kx in order:
            out.append(min(max(T[ky, kx] >> qshift, -128), 127))  # numpy >> floors
    return np.array(out)


def test_features_definition(orc):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (29, 41, 3)).astype(np.uint8)
    for qs in (0, 4):
        p = orc.default_params(quant_shift=qs)
        feat, norm = orc.features(img, p)
        assert feat.shape == (4, 29, 41, 48)
        for s in range(4):
            for (x, y) in [(0, 0), (40, 28), (5, 17), (20, 0), (0, 13), (37, 26)] + \
                          [tuple(rng.integers(0, (41, 29))) for _ in range(8)]:
                exp = features_numpy(img, s, qs, x, y)
                assert np.array_equal(feat[s, y, x].astype(np.int64), exp), (s, x, y)
        assert np.array_equal(norm, (feat.astype(np.int64) ** 2).sum(-1))


def test_feature_quantisation_floor(orc):
    # one darker pixel in the positive half of w_1 makes T(0,1) = -34:
    # floor(-34 / 16) = -3, where truncating division would give -2
    W = walsh_closed_form()
    patch = np.full((8, 8), 100, np.int64)
    patch[0, 0] -= 34
    T = W @ patch @ W.T
    assert T[0, 1] == -34
    img = np.repeat(patch.astype(np.uint8)[:, :, None], 3, axis=2)
    feat, _ = orc.features(img, orc.default_params(quant_shift=4))
    # pixel (3, 3): offsets -3..+4 cover the whole 8x8 image without clamping
    got = feat[0, 3, 3, :16].astype(np.int64)
    order = golden_order()
    exp = np.array([min(max(int(np.floor(T[a, b] / 16)), -128), 127) for a, b in order])
    assert got[0] == -3
    assert np.array_equal(got, exp)


def test_feature_saturation(orc):
    # a maximal-contrast basis patch saturates at 127 / -128
    W = walsh_closed_form()
    patch = np.where(np.outer(W[0], W[1]) > 0, 255, 0).astype(np.uint8)
    img = np.repeat(patch[:, :, None], 3, axis=2)
    feat, _ = orc.features(img, orc.default_params(quant_shift=4))
    assert feat[0, 3, 3, 0] == 127  # (ky, kx) = (0, 1) is feature 0
    inv = np.repeat((255 - patch)[:, :, None], 3, axis=2)
    feat2, _ = orc.features(inv, orc.default_params(quant_shift=4))
    assert feat2[0, 3, 3, 0] == -128
