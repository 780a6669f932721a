"""Pins of the oracle's random-search generator and matching cost.

Philox4x32-10 (Salmon et al., SC'11) is pinned by the published known-answer
vectors; the shape of its round function and key schedule is also checked
against numpy's independent Philox4x64-10.  The offset mapping is pinned by
exact enumeration.  The cost (Eq. 1 with SSD of WHT features) is pinned by
the closed form "zero at the true correspondence" on integer-shift scenes and
by an int64 restatement with clamped positions.
"""
import os

import numpy as np
import pytest

import scenegen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def _philox_py(ctr, key, bits, rounds=10):
    """Philox4xW round function + Weyl key schedule, word size `bits`."""
    if bits == 64:
        M0, M1, W0, W1 = 0xD2E7470EE14C6C93, 0xCA5A826395121157, 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B
    else:
        M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    mask = (1 << bits) - 1
    c, k = list(ctr), list(key)
    for r in range(rounds):
        if r:
            k = [(k[0] + W0) & mask, (k[1] + W1) & mask]
        p0, p1 = M0 * c[0], M1 * c[2]
        c = [(p1 >> bits) ^ c[1] ^ k[0], p1 & mask, (p0 >> bits) ^ c[3] ^ k[1], p0 & mask]
    return c


def test_philox_structure_against_numpy(orc):
    # numpy's Philox (4x64, 10 rounds) emits block(counter + 1) first
    rng = np.random.default_rng(7)
    for _ in range(5):
        key = [int(x) for x in rng.integers(0, 2**63, 2)]
        ctr = [int(x) for x in rng.integers(0, 2**63, 4)]
        bg = np.random.Philox(key=key, counter=ctr)
        raw = [int(bg.random_raw()) for _ in range(4)]
        assert raw == _philox_py([ctr[0] + 1] + ctr[1:], key, 64)
    # the same structure with 32-bit words is what the oracle computes
    for _ in range(200):
        key = [int(x) for x in rng.integers(0, 2**32, 2)]
        ctr = [int(x) for x in rng.integers(0, 2**32, 4)]
        assert [int(x) for x in orc.philox4x32_10(ctr, key)] == _philox_py(ctr, key, 32)


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_rs_offset_distribution(orc, n):
    # r enumerated on a uniform grid of 2^16 points: the offset is the nearest
    # integer to a uniform value on ]-n, n[ -> -n and n get half weight
    counts = {}
    step = 1 << 16
    for r in range(0, 1 << 32, step):
        o = orc.rs_offset(r, n)
        counts[o] = counts.get(o, 0) + 1
    assert sorted(counts) == list(range(-n, n + 1))
    total = (1 << 32) // step
    unit = total // (4 * n)
    for o, c in counts.items():
        assert c == (unit if abs(o) == n else 2 * unit), (o, c)


def test_philox_uniformity(orc):
    # chi-square of the top 4 bits over 4096 counters x 4 words
    vals = np.concatenate([orc.philox4x32_10([i, 3, 5, 0], [11, 13]) for i in range(4096)])
    hist = np.bincount(vals >> 28, minlength=16)
    exp = len(vals) / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45  # 15 dof, p ~ 1e-4


def _shift_feats(orc, u, v, d0, d1, w=128, h=112, seed=2):
    q = scenegen.make_shift_quad(w, h, seed, u=u, v=v, d0=d0, d1=d1)
    return q, [orc.features(im)[0] for im in q.images()]


@pytest.mark.parametrize("uvdd", [(3, -2, 5, 4), (-4, 1, 0, 2), (0, 0, 7, 7)])
def test_cost_zero_at_truth(orc, uvdd):
    u, v, d0, d1 = uvdd
    q, (fL0, fR0, fL1, fR1) = _shift_feats(orc, u, v, d0, d1)
    h, w = q.height, q.width
    # patch reach at scale 3 (-3n..+4n, smoothing -n/2..n/2-1) plus the motion
    m = 4 * 8 + 4 + abs(u) + abs(v) + d0 + d1
    for s in range(4):
        for y in range(m, h - m, 3):
            for x in range(m, w - m, 3):
                c = orc.cost(fL0[s], fL1[s], fR0[s], fR1[s], 0, x, y, [u, v, d0, d1])
                assert c == 0, (s, x, y, c)
        # a wrong vector costs more somewhere
        wrong = sum(orc.cost(fL0[s], fL1[s], fR0[s], fR1[s], 0, x, y, [u + 1, v, d0, d1])
                    for y in range(m, h - m, 5) for x in range(m, w - m, 5))
        assert wrong > 0


def test_cost_zero_at_truth_mirrored(orc):
    # inverse field: reference R1, temporal R0, stereo L1, cross L0; the true
    # inverse vector of (u, v, d0, d1) is (-(u - d1 + d0), -v, d1, d0)
    u, v, d0, d1 = 3, -2, 5, 4
    q, (fL0, fR0, fL1, fR1) = _shift_feats(orc, u, v, d0, d1)
    iu = [-(u - d1 + d0), -v, d1, d0]
    h, w = q.height, q.width
    m = 4 * 8 + 4 + 14
    for s in range(4):
        for y in range(m, h - m, 4):
            for x in range(m, w - m, 4):
                assert orc.cost(fR1[s], fR0[s], fL1[s], fL0[s], 1, x, y, iu) == 0


def test_cost_restated_with_clamping(orc):
    rng = np.random.default_rng(5)
    imgs = scenegen.random_images(23, 17, 9)
    feats = [orc.features(im)[0][1] for im in imgs]  # scale 1
    h, w = 17, 23
    F = [f.astype(np.int64) for f in feats]
    for mirror in (0, 1):
        sg = -1 if mirror else 1
        for _ in range(300):
            x, y = int(rng.integers(0, w)), int(rng.integers(0, h))
            u = [int(a) for a in rng.integers(-40, 40, 2)] + [int(a) for a in rng.integers(0, 40, 2)]
            cl = lambda a, n: min(max(a, 0), n - 1)
            a = F[0][y, x]
            exp = (((a - F[1][cl(y + u[1], h), cl(x + u[0], w)]) ** 2).sum()
                   + ((a - F[2][y, cl(x - sg * u[2], w)]) ** 2).sum()
                   + ((a - F[3][cl(y + u[1], h), cl(x + u[0] - sg * u[3], w)]) ** 2).sum())
            assert orc.cost(*feats, mirror, x, y, u) == exp
