"""Dense interpolation of the seeds (Sec. 3.2) on the GPU vs the CPU oracle,
through the C ABI.

Both sides fit and evaluate in double precision with the same neighbour
order and ridge; they differ only in the order of the floating-point sums
(the GPU reduces across the lanes of a warp), so the fitted models agree to
about 1e-13 relative.  The Cholesky solves amplify that by at most the
condition number the ridge allows (1e9 for the linear part) and the output
is rounded to float32 (half an ulp: 6e-8 relative), hence the bound
|gpu - oracle| <= 1e-3 px + 1e-5 |oracle| used below.  The closest seed of a
pixel is an integer decision taken on integer squared distances on both
sides, so a wrong choice would show as a difference of whole pixels.
"""
import os

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_1710_10096_gb300 as sff
    sff.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    return torch, sff, oracle


def _gpu_interp(env, seeds, w, h, f, B, capacity=None, count=None, **over):
    torch, sff, _ = env
    n = len(seeds)
    capacity = n if capacity is None else capacity
    count = n if count is None else count
    raw = np.zeros(20 * max(capacity, n, 1), np.uint8)
    raw[:20 * n] = np.frombuffer(np.ascontiguousarray(seeds).tobytes(), np.uint8)
    dseeds = torch.as_tensor(raw).cuda()
    dcount = torch.tensor([count], dtype=torch.int32, device="cuda")
    p = sff.default_interp_params(w, h, f, B, **over)
    field = torch.full((h, w, 4), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.empty(sff.interp_workspace_bytes(w, h, capacity), dtype=torch.uint8, device="cuda")
    sff.interpolate(dseeds, dcount, capacity, w, h, p, field, ws)
    torch.cuda.synchronize()
    return field.cpu().numpy(), sff.interp_status(ws, w, h, capacity)


def _oracle_interp(orc, seeds, w, h, f, B, **over):
    return orc.interpolate(np.ascontiguousarray(seeds, orc.SEED_DTYPE), w, h, orc.interp_params(w, h, f, B, **over))


def _scene_seeds(family, w, h, scene_seed, seed, **kw):
    gt, occ, f, B = scenegen.ground_truth(family, w, h, scene_seed)
    return scenegen.sparse_seeds(gt, occ, seed, **kw), f, B


@pytest.mark.parametrize("w,h,frac,over", [
    (1242, 375, 0.6, {}),                                  # the driving size, default neighbourhoods
    (400, 160, 0.85, dict(k_geo=40, k_motion=80)),         # motion seeds in one corner strip only
])
def test_far_motion_neighbours_equal_oracle(env, w, h, frac, over):
    # dense geometry seeds everywhere, motion seeds only right of frac * W
    # (the disparity fill's seeds carry d1 = 0: no motion): the motion
    # neighbours of the seeds on the left are far, the rings that reach them
    # hold many candidates, and the candidate buffer is compacted on the
    # way; the field still equals the unbounded oracle's
    gt, occ, f, B = scenegen.ground_truth("driving", w, h, 2)
    seeds = scenegen.sparse_seeds(gt, occ, 5, keep=1.0)
    left = seeds["x"] < int(frac * w)
    seeds["u"][left] = 0
    seeds["v"][left] = 0
    seeds["d1"][left] = 0
    seeds["kind"][left] = 1
    assert left.sum() > 1000 and (~left).sum() > 100
    got, status = _gpu_interp(env, seeds, w, h, f, B, **over)
    want = _oracle_interp(env[2], seeds, w, h, f, B, **over)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


@pytest.mark.parametrize("family,w,h,keep,noise,outl,over", [
    ("planes", 96, 64, 0.6, 0.5, 0.05, {}),                          # defaults: 160 / 80 neighbours
    ("driving", 37, 23, 1.0, 0.0, 0.0, dict(k_geo=20, k_motion=10)),  # ragged, dense
    ("movie", 130, 70, 0.3, 1.0, 0.1, dict(k_geo=40, k_motion=24)),   # outliers, large motion
    ("planes", 200, 120, 0.04, 0.0, 0.0, {}),                         # sparse: fewer seeds than k
    ("driving", 200, 120, 0.04, 0.5, 0.0, dict(k_geo=30, k_motion=12, alpha=0.0)),  # sparse, far rings, flat weights
    ("planes", 200, 120, 1.0, 0.5, 0.0, dict(k_geo=400, k_motion=300)),  # more candidates than registers hold
])
def test_field_equals_oracle(env, family, w, h, keep, noise, outl, over):
    seeds, f, B = _scene_seeds(family, w, h, 3, w + h, keep=keep, noise=noise, outliers=outl)
    assert len(seeds) > 0
    got, status = _gpu_interp(env, seeds, w, h, f, B, **over)
    want = _oracle_interp(env[2], seeds, w, h, f, B, **over)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


def test_lattice_ties(env):
    # seeds at the centres of the 3x3 blocks: every pixel and every seed has
    # shells of equidistant seeds, and k cuts through them, so the order of
    # equal distances (the lower seed index first) decides the neighbourhoods
    w, h = 61, 40
    ys, xs = np.mgrid[1:h:3, 1:w:3]
    s = np.zeros(xs.size, scenegen.SEED_RECORD)
    s["x"], s["y"] = xs.ravel(), ys.ravel()
    s["d0"] = 20 + (s["x"] // 7)
    s["d1"] = s["d0"] + 3
    s["u"] = 2 + (s["y"] // 5)
    s["v"] = -1
    for kg, km in ((13, 7), (5, 3), (1, 1)):
        got, status = _gpu_interp(env, s, w, h, 500.0, 0.3, k_geo=kg, k_motion=km)
        want = _oracle_interp(env[2], s, w, h, 500.0, 0.3, k_geo=kg, k_motion=km)
        assert status == 0
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


def test_more_than_32_seeds_tied_at_the_kth_distance(env):
    # 48 seeds on one lattice circle (dx^2 + dy^2 = 5525) around a centre
    # seed, in a shuffled order and with random values: the centre's k-th
    # neighbour is a 48-way tie, more than a warp ranks in registers, so the
    # index threshold comes from the bisection over seed indices; a wrong
    # choice of tied seeds changes the centre's fits and the field around it
    r = 74
    circle = [(dx, dy) for dx in range(-r, r + 1) for dy in range(-r, r + 1) if dx * dx + dy * dy == 5525]
    assert len(circle) == 48
    w, h, cx, cy = 170, 160, 85, 80
    rng = np.random.default_rng(48)
    s = np.zeros(len(circle) + 1, scenegen.SEED_RECORD)
    s["x"] = [cx + dx for dx, _ in circle] + [cx]
    s["y"] = [cy + dy for _, dy in circle] + [cy]
    s["d0"] = rng.integers(20, 60, len(s))
    s["d1"] = s["d0"] + rng.integers(-3, 4, len(s))
    s["u"] = rng.integers(-10, 11, len(s))
    s["v"] = rng.integers(-5, 6, len(s))
    s["d1"][rng.choice(len(circle), 8, replace=False)] = 0  # 40 tied motion seeds
    s = s[rng.permutation(len(s))]
    for kg, km in ((10, 5), (40, 30), (48, 40)):
        got, status = _gpu_interp(env, s, w, h, 500.0, 0.3, k_geo=kg, k_motion=km)
        want = _oracle_interp(env[2], s, w, h, 500.0, 0.3, k_geo=kg, k_motion=km)
        assert status == 0
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


def _rows(rows):
    s = np.zeros(len(rows), scenegen.SEED_RECORD)
    for k, (x, y, u, v, d0, d1) in enumerate(rows):
        s[k]["x"], s[k]["y"], s[k]["u"], s[k]["v"], s[k]["d0"], s[k]["d1"] = x, y, u, v, d0, d1
    return s


@pytest.mark.parametrize("rows,w,h,kg,km", [
    # every seed at unit disparity: the reprojection at max(d0, 1) = 1
    ([(x, y, 3, 0, 1, 1) for y in range(1, 24, 3) for x in range(1, 30, 3)], 30, 24, 12, 8),
    # a plane that falls below d0 = 1 left of the first seed
    ([(5, 10, 3, 0, 1, 1), (15, 10, 0, 0, 3, 3)], 21, 21, 2, 1),
    # a seed whose translation moves its near plane behind the camera
    ([(5, 10, 0, 0, 2, 40), (15, 10, 0, 0, 12, 13)], 21, 21, 2, 1),
])
def test_reprojection_edge_cases(env, rows, w, h, kg, km):
    s = _rows(rows)
    got, status = _gpu_interp(env, s, w, h, 300.0, 0.5, k_geo=kg, k_motion=km)
    want = _oracle_interp(env[2], s, w, h, 300.0, 0.5, k_geo=kg, k_motion=km)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


def test_end_to_end_after_the_matching_stage(env):
    # the seeds of the whole matching stage, each side on its own: the GPU
    # interpolates the GPU's seeds, the oracle the oracle's
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 1)
    m = sff.QuadMatcher(q.width, q.height)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    dseeds, dcount = m.run(*dev, seed=1)
    p = sff.default_interp_params(q.width, q.height, q.focal, q.baseline)
    field = torch.empty((q.height, q.width, 4), dtype=torch.float32, device="cuda")
    ws = torch.empty(sff.interp_workspace_bytes(q.width, q.height, m.capacity), dtype=torch.uint8, device="cuda")
    sff.interpolate(dseeds, dcount, m.capacity, q.width, q.height, p, field, ws)
    torch.cuda.synchronize()
    ref = orc.run_quad(*q.images(), seed=1)
    assert len(ref["seeds"]) > 100
    want = orc.interpolate(ref["seeds"], q.width, q.height, orc.interp_params(q.width, q.height, q.focal, q.baseline))
    assert sff.interp_status(ws, q.width, q.height, m.capacity) == 0
    np.testing.assert_allclose(field.cpu().numpy(), want, rtol=RTOL, atol=ATOL)


def test_full_size_sampled_pixels(env):
    # 1242 x 375 with about 25k seeds: the oracle evaluates a sample of pixels
    # (the tail row and column included), fitting only their closest seeds
    torch, sff, orc = env
    w, h = 1242, 375
    seeds, f, B = _scene_seeds("driving", w, h, 2, 11, keep=0.6, noise=0.5, outliers=0.05)
    got, status = _gpu_interp(env, seeds, w, h, f, B)
    assert status == 0
    rng = np.random.default_rng(5)
    pix = np.concatenate([np.stack([rng.integers(0, w, 1500), rng.integers(0, h, 1500)], 1),
                          [[w - 1, h - 1], [0, 0], [w - 1, 0], [0, h - 1]]]).astype(np.int32)
    p = orc.interp_params(w, h, f, B)
    sd = np.ascontiguousarray(seeds, orc.SEED_DTYPE)
    _, closest = orc.interpolate_pixels(sd, p, pix, models=(np.zeros((len(sd), 3)), np.zeros((len(sd), 15)),
                                                             np.zeros(len(sd), np.int32)))
    models = orc.seed_models(sd, p, which=closest)
    want, closest2 = orc.interpolate_pixels(sd, p, pix, models=models)
    assert np.array_equal(closest, closest2)
    np.testing.assert_allclose(got[pix[:, 1], pix[:, 0]], want, rtol=RTOL, atol=ATOL)


def test_lone_seed_in_a_hole(env):
    # a dense lattice with a 480 x 480 px hole holding one seed: that seed's
    # neighbourhoods lie on the far side of the hole (833 candidates for
    # k = 160, more than the registers hold); pixels in and around the hole
    torch, sff, orc = env
    w, h = 600, 600
    ys, xs = np.mgrid[0:200, 0:200]
    keep = (np.maximum(np.abs(xs - 100), np.abs(ys - 100)) >= 80) | ((xs == 100) & (ys == 100))
    d = np.zeros(int(keep.sum()), scenegen.SEED_RECORD)
    d["x"], d["y"] = 3 * xs[keep], 3 * ys[keep]
    d["d0"] = 20 + d["x"] // 40
    d["d1"] = d["d0"] + 2 + d["y"] // 100
    d["u"], d["v"] = 3 + d["y"] // 60, -2
    got, status = _gpu_interp(env, d, w, h, 400.0, 0.5)
    assert status == 0
    rng = np.random.default_rng(3)
    pix = np.concatenate([np.stack([rng.integers(40, 560, 600), rng.integers(40, 560, 600)], 1),
                          [[300, 300], [301, 299], [0, 599]]]).astype(np.int32)
    p = orc.interp_params(w, h, 400.0, 0.5)
    sd = np.ascontiguousarray(d, orc.SEED_DTYPE)
    zero = (np.zeros((len(sd), 3)), np.zeros((len(sd), 15)), np.zeros(len(sd), np.int32))
    _, closest = orc.interpolate_pixels(sd, p, pix, models=zero)
    want, _ = orc.interpolate_pixels(sd, p, pix, models=orc.seed_models(sd, p, which=closest))
    np.testing.assert_allclose(got[pix[:, 1], pix[:, 0]], want, rtol=RTOL, atol=ATOL)


def test_no_seeds_and_capacity(env):
    w, h = 50, 31
    seeds, f, B = _scene_seeds("planes", w, h, 4, 8, keep=0.5)
    got, status = _gpu_interp(env, seeds[:0], w, h, f, B, capacity=0, count=0)
    assert status == 0 and (got == 0).all()
    got, status = _gpu_interp(env, seeds, w, h, f, B, count=0)  # count 0 with room
    assert status == 0 and (got == 0).all()
    # a count above the capacity: the first `capacity` seeds are used
    cap = len(seeds) // 2
    got, status = _gpu_interp(env, seeds, w, h, f, B, capacity=cap, count=len(seeds))
    want = _oracle_interp(env[2], seeds[:cap], w, h, f, B)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)
    # one seed: a constant disparity and a translation everywhere
    got, status = _gpu_interp(env, seeds[:1], w, h, f, B)
    want = _oracle_interp(env[2], seeds[:1], w, h, f, B)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)


def test_invalid_seed_sets_are_reported(env):
    w, h = 40, 30
    s = np.zeros(3, scenegen.SEED_RECORD)
    s["x"], s["y"], s["d0"], s["d1"] = [4, 5, 20], [4, 3, 20], 10, 10  # the first two share block (1, 1)
    got, status = _gpu_interp(env, s, w, h, 300.0, 0.5)
    assert status & 1 and (got == 0).all()
    s["x"], s["y"] = [4, 45, 20], [4, 3, 20]  # x = 45 is outside the image
    got, status = _gpu_interp(env, s, w, h, 300.0, 0.5)
    assert status & 1 and (got == 0).all()



def test_candidates_beyond_the_slots_are_compacted(env):
    # more candidates than the 6 k + 256 slots: a lone seed in the middle of a
    # 480 x 480 px hole in a dense lattice (8151 candidates for k = 1024).  The
    # buffer is compacted to the candidates within the k-th distances so far
    # whenever it would overflow, and the field equals the unbounded oracle's
    w, h = 600, 600
    ys, xs = np.mgrid[0:200, 0:200]
    keep = (np.maximum(np.abs(xs - 100), np.abs(ys - 100)) >= 80) | ((xs == 100) & (ys == 100))
    d = np.zeros(int(keep.sum()), scenegen.SEED_RECORD)
    d["x"], d["y"], d["d0"], d["d1"] = 3 * xs[keep], 3 * ys[keep], 30, 31
    got, status = _gpu_interp(env, d, w, h, 300.0, 0.5, k_geo=1024, k_motion=4)
    want = _oracle_interp(env[2], d, w, h, 300.0, 0.5, k_geo=1024, k_motion=4)
    assert status == 0
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)
