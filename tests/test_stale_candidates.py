"""The stale-candidate skip of the iteration kernels, checked on the CPU.

The kernels skip a predecessor candidate whose vector has not changed since
the pixel last took a candidate from the same neighbour (change stamps: 0
before the scale's first iteration, 2 it + 1 for a colour-0 change in the
first half-step of iteration it, 2 it + 2 for a colour-1 change in the
second).  The claim is that such a candidate can never be strictly lower
than the pixel's cost, so the skip leaves every result unchanged.  This test
replays the oracle's checkerboard iteration (two synchronous half-steps per
iteration over a snapshot, then the random search) in numpy on a rendered
scene, applies the skip with the same stamp bookkeeping and thresholds, and
checks:
  - the replay without any skip reproduces the oracle's fields exactly (so the
    replay is the oracle's procedure);
  - every skipped candidate's cost is at least the pixel's cost at the moment
    it would have been compared (so it could not have been taken);
  - the fields with the skip equal the oracle's, and the skip fires.
"""
import numpy as np

import scenegen

EMPTY = np.iinfo(np.int32).max
DIRS = [(1, 1), (-1, -1), (1, -1), (-1, 1)]


def _philox(c0, c1, c2, key):
    """Philox4x32-10 (Salmon et al., SC'11) on arrays of counters (c0, c1, c2, 0)."""
    M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    c = [c0.astype(np.uint32), np.full(c0.shape, c1, np.uint32), np.full(c0.shape, c2, np.uint32),
         np.zeros(c0.shape, np.uint32)]
    k0, k1 = key
    for r in range(10):
        if r:
            k0, k1 = (k0 + 0x9E3779B9) & 0xFFFFFFFF, (k1 + 0xBB67AE85) & 0xFFFFFFFF
        p0 = M0 * c[0].astype(np.uint64)
        p1 = M1 * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), p0.astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), p1.astype(np.uint32)
        c = [hi1 ^ c[1] ^ np.uint32(k0), lo1, hi0 ^ c[3] ^ np.uint32(k1), lo0]
    return c


def _offset(r, n):
    j = ((r.astype(np.uint64) * np.uint64(4 * n)) >> np.uint64(32)).astype(np.int64)
    return (j + 1) // 2 - n


def _replay(feats, mirror, seed, init_field, init_valid, skip, iters=12):
    """Both colours' half-steps and the search of every iteration of every
    scale; returns the final field and cost (image layout) and the number of
    skipped candidates.  skip: apply the stale-candidate rule (asserting the
    invariant for every skipped candidate)."""
    fr, ft, fs, fc = feats
    S, h, w = fr.shape[0], fr.shape[1], fr.shape[2]
    sigma = -1 if mirror else 1
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    skipped = 0
    vec = cst = None
    for s in range(S - 1, -1, -1):
        n = 1 << s
        gw, gh = (w + n - 1) // n, (h + n - 1) // n
        R, T, St, C = (f[s].astype(np.int32) for f in (fr, ft, fs, fc))
        gy, gx = np.mgrid[0:gh, 0:gw]
        X, Y = gx * n, gy * n
        ref = R[Y, X]

        def cost(V, mask):
            idx = np.nonzero(mask)
            x, y = X[idx], Y[idx]
            u, v, d0, d1 = (V[..., k][idx] for k in range(4))
            a = ref[idx]
            tx, ty = np.clip(x + u, 0, w - 1), np.clip(y + v, 0, h - 1)
            sx = np.clip(x - sigma * d0, 0, w - 1)
            cx = np.clip(x + u - sigma * d1, 0, w - 1)
            out = np.full(mask.shape, EMPTY, np.int64)
            out[idx] = (((a - T[ty, tx]) ** 2).sum(-1) + ((a - St[y, sx]) ** 2).sum(-1)
                        + ((a - C[ty, cx]) ** 2).sum(-1))
            return out

        if s == S - 1:  # the initialisation (the oracle's, read from a run without iterations)
            vec = init_field[Y, X].astype(np.int64)
            valid = init_valid[Y, X]
            vec[~valid] = 0
            cst = np.where(valid, cost(vec, valid), EMPTY)
        else:  # inheritance: coarser grid points keep their vector, rescored; the rest empty
            pvec, pcst = vec, cst
            coarse = ((gx % 2) == 0) & ((gy % 2) == 0)
            m = coarse & (pcst[np.minimum(gy // 2, pcst.shape[0] - 1), np.minimum(gx // 2, pcst.shape[1] - 1)] != EMPTY)
            vec = np.zeros((gh, gw, 4), np.int64)
            vec[m] = pvec[(gy // 2)[m], (gx // 2)[m]]
            cst = np.where(m, cost(vec, m), EMPTY)
        colour = (gx + gy) & 1
        stamp = np.zeros((gh, gw), np.int64)
        for it in range(iters):
            dx, dy = DIRS[it % 4]
            ih, iv = it - 2, (it - 3 if it & 1 else it - 1)
            for col in (0, 1):
                sv, sc, sst = vec.copy(), cst.copy(), stamp.copy()  # the snapshot of the half-step
                own = colour == col
                ax, by = gx - dx, gy - dy
                ha, hb = own & (ax >= 0) & (ax < gw), own & (by >= 0) & (by < gh)
                axc, byc = np.clip(ax, 0, gw - 1), np.clip(by, 0, gh - 1)
                va, vb = sv[gy, axc], sv[byc, gx]
                ca, cb = np.where(ha, sc[gy, axc], EMPTY), np.where(hb, sc[byc, gx], EMPTY)
                own_valid = sc != EMPTY
                same = lambda p, q: (p == q).all(-1)
                do_a = own & (ca != EMPTY) & ~(own_valid & same(va, sv))
                do_b = own & (cb != EMPTY) & ~(own_valid & same(vb, sv)) & ~((ca != EMPTY) & same(vb, va))
                lim_h = 2 * ih + col if ih >= 0 else -1
                lim_v = 2 * iv + col if iv >= 0 else -1
                stale_a = skip & (sst[gy, axc] <= lim_h)
                stale_b = skip & (sst[byc, gx] <= lim_v)
                bc, bv = sc.copy(), sv.copy()
                for go, stale, cand in ((do_a, stale_a, va), (do_b, stale_b, vb)):
                    if skip:
                        gone = go & stale
                        # invariant: a skipped candidate could not be strictly lower
                        assert not (gone & (cost(cand, gone) < bc)).any()
                        skipped += int(gone.sum())
                        go = go & ~stale
                    cc = cost(cand, go)
                    better = go & (cc < bc)
                    bc = np.where(better, cc, bc)
                    bv[better] = cand[better]
                changed = own & (bc != sc)
                vec = np.where(own[..., None], bv, vec)
                cst = np.where(own, bc, cst)
                stamp = np.where(changed, 2 * it + 1 + col, stamp)
            # the random search of every non-empty grid pixel
            r = _philox((Y * w + X).astype(np.uint32), it, s + 4 * mirror, key)
            cand = np.stack([vec[..., k] + _offset(r[k], n) for k in range(4)], -1)
            cand[..., 2:] = np.maximum(cand[..., 2:], 0)
            cand = cand.astype(np.int16).astype(np.int64)
            go = (cst != EMPTY) & ~(cand == vec).all(-1)
            cc = cost(cand, go)
            better = go & (cc < cst)
            cst = np.where(better, cc, cst)
            vec[better] = cand[better]
            # a colour-0 change is seen from the next iteration's first half-step
            # (time 2 it + 2), a colour-1 change from the same point (2 it + 1)
            stamp = np.where(better, np.where(colour == 0, 2 * it + 3, 2 * it + 2), stamp)
    field = np.zeros((h, w, 4), np.int16)
    field[Y, X] = vec
    cost_out = np.full((h, w), EMPTY, np.int32)
    cost_out[Y, X] = cst
    return field, cost_out, skipped


def test_stale_candidate_skip_leaves_the_fields_unchanged(orc):
    q = scenegen.make_quad("planes", 160, 64, 3)
    P = orc.default_params()
    P0 = orc.default_params(iterations=0)
    f = [orc.features(im, P)[0] for im in (q.L0, q.R0, q.L1, q.R1)]
    fL0, fR0, fL1, fR1 = f
    seed = 77
    total = 0
    for mirror, views in ((0, (fL0, fL1, fR0, fR1)), (1, (fR1, fR0, fL1, fL0))):
        want_f, want_c = orc.match_views(*views, mirror, seed, P)
        init_f, init_c = orc.match_views(*views, mirror, seed, P0)
        valid = init_c != EMPTY
        plain_f, plain_c, _ = _replay(views, mirror, seed, init_f, valid, skip=False)
        assert np.array_equal(plain_f, want_f) and np.array_equal(plain_c, want_c)
        got_f, got_c, k = _replay(views, mirror, seed, init_f, valid, skip=True)
        assert np.array_equal(got_f, want_f) and np.array_equal(got_c, want_c)
        total += k
    assert total > 0
