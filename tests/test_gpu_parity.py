"""CUDA path vs the CPU oracle, bit for bit, through the C ABI.

Every output of the stage is integer: features, vectors, costs, keep masks,
consistency errors and seeds must be identical.  Sizes span several CTAs
and ragged tails (widths not multiples of the 128-thread rows or of the
scale strides), the minimum 8x8 image, and the full 1242x375 and 1024x436
workloads in the launch configuration the benchmark times.
"""
import os

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


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


def _oparams(orc, p):
    return orc.default_params(**p.as_dict())


def _gpu_features(torch, sff, img, p):
    h, w, _ = img.shape
    pyr = torch.empty(sff.pyramid_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.features(torch.as_tensor(img).cuda(), pyr, ws, p)
    torch.cuda.synchronize()
    feat, norm = sff.split_pyramid(pyr, w, h, p)
    return pyr, (feat.cpu().numpy(), norm.cpu().numpy())


@pytest.mark.parametrize("size", [(8, 8), (37, 23), (130, 70), (256, 80), (300, 9), (40, 410), (1242, 375)])
@pytest.mark.parametrize("qshift", [4, 0])
def test_features_bit_exact(env, size, qshift):
    # sff_features (the separable form: tiles of 32 columns x 24 rows of one
    # residue class of rows mod n; 40 x 410 gives several tiles per residue at
    # every scale, 8 x 8 a single partial tile)
    torch, sff, orc = env
    w, h = size
    img = scenegen.random_images(w, h, seed=w * 1000 + h, n=1)[0]
    p = sff.default_params(quant_shift=qshift)
    _, (gfeat, gnorm) = _gpu_features(torch, sff, img, p)
    feat, norm = orc.features(img, _oparams(orc, p))
    assert np.array_equal(gfeat, feat)
    assert np.array_equal(gnorm, norm)


@pytest.mark.parametrize("size", [(8, 8), (37, 23), (130, 70), (256, 80), (300, 9), (1242, 375)])
@pytest.mark.parametrize("qshift", [4, 0])
def test_features_tensor_core_bit_exact(env, size, qshift):
    # the transform as a tensor-core matrix product (sff_features_tc): every
    # record and norm equals the oracle's (and so the butterfly form's)
    torch, sff, orc = env
    w, h = size
    img = scenegen.random_images(w, h, seed=w * 1000 + h + 7, n=1)[0]
    p = sff.default_params(quant_shift=qshift)
    pyr = torch.empty(sff.pyramid_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.device_status(reset=True)
    sff.features(torch.as_tensor(img).cuda(), pyr, ws, p, tensor=True)
    assert sff.device_status(reset=True) == sff.OK
    gfeat, gnorm = (a.cpu().numpy() for a in sff.split_pyramid(pyr, w, h, p))
    feat, norm = orc.features(img, _oparams(orc, p))
    assert np.array_equal(gfeat, feat)
    assert np.array_equal(gnorm, norm)


@pytest.mark.parametrize("size", [(8, 8), (37, 23), (130, 70), (256, 80), (300, 9), (1242, 375)])
@pytest.mark.parametrize("qshift", [4, 0])
def test_features_pixel_pairs_bit_exact(env, size, qshift):
    # the earlier form (sff_features_pairs: one thread per vertical pixel
    # pair, 9 row transforms folded into both): every record and norm equals
    # the oracle's
    torch, sff, orc = env
    w, h = size
    img = scenegen.random_images(w, h, seed=w * 1000 + h + 11, n=1)[0]
    p = sff.default_params(quant_shift=qshift)
    pyr = torch.empty(sff.pyramid_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.features(torch.as_tensor(img).cuda(), pyr, ws, p, form=2)
    torch.cuda.synchronize()
    gfeat, gnorm = (a.cpu().numpy() for a in sff.split_pyramid(pyr, w, h, p))
    feat, norm = orc.features(img, _oparams(orc, p))
    assert np.array_equal(gfeat, feat)
    assert np.array_equal(gnorm, norm)


def _match_both(env, imgs, p, seed):
    torch, sff, orc = env
    h, w, _ = imgs[0].shape
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in imgs]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    op = _oparams(orc, p)
    feats = [orc.features(im, op)[0] for im in imgs]
    out = []
    for mirror, roles in ((0, (0, 2, 1, 3)), (1, (3, 1, 2, 0))):
        field = torch.empty((h, w, 4), dtype=torch.int16, device="cuda")
        cost = torch.empty((h, w), dtype=torch.int32, device="cuda")
        sff.match_views(*(pyrs[i] for i in roles), w, h, mirror, seed, field, cost, ws, p)
        torch.cuda.synchronize()
        of, oc = orc.match_views(*(feats[i] for i in roles), mirror, seed, op)
        out.append((field.cpu().numpy(), cost.cpu().numpy(), of, oc))
    return out


@pytest.mark.parametrize("size,params", [
    ((64, 48), {}),
    ((37, 23), {}),
    ((8, 8), {}),
    ((130, 70), {"iterations": 5}),
    ((96, 40), {"num_scales": 1, "iterations": 3}),
    ((96, 40), {"num_scales": 2, "iterations": 0}),
    ((96, 40), {"num_scales": 3, "knn_temporal": 1, "knn_epipolar": 1}),
    ((150, 66), {"knn_temporal": 8, "knn_epipolar": 8}),
])
def test_match_views_random_images(env, size, params):
    torch, sff, orc = env
    w, h = size
    imgs = scenegen.random_images(w, h, seed=7 + w + h)
    p = sff.default_params(**params)
    for gf, gc, of, oc in _match_both(env, imgs, p, seed=0x1234567890ABCDEF):
        assert np.array_equal(gc, oc)
        assert np.array_equal(gf, of)


@pytest.mark.parametrize("size,params", [
    ((64, 48), {}),
    ((37, 23), {"iterations": 5}),
    ((96, 40), {"num_scales": 2, "iterations": 3}),
    ((600, 520), {"iterations": 2}),  # scale-0 diagonals longer than one round of 512 pixel groups
])
def test_match_views_sequential_equals_oracle_scan_order(env, size, params):
    # the paper's in-place raster sweeps (departure D4 switched back): both
    # fields bit-exact to the oracle's sequential-scan mode
    torch, sff, orc = env
    w, h = size
    imgs = scenegen.random_images(w, h, seed=11 + w + h)
    p = sff.default_params(**params)
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in imgs]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    op = _oparams(orc, p)
    op.order_mode = orc.SEQUENTIAL_SCAN
    feats = [orc.features(im, op)[0] for im in imgs]
    for mirror, roles in ((0, (0, 2, 1, 3)), (1, (3, 1, 2, 0))):
        field = torch.empty((h, w, 4), dtype=torch.int16, device="cuda")
        cost = torch.empty((h, w), dtype=torch.int32, device="cuda")
        sff.match_views_sequential(*(pyrs[i] for i in roles), w, h, mirror, 77, field, cost, ws, p)
        torch.cuda.synchronize()
        of, oc = orc.match_views(*(feats[i] for i in roles), mirror, 77, op)
        assert np.array_equal(cost.cpu().numpy(), oc)
        assert np.array_equal(field.cpu().numpy(), of)


def test_match_views_sequential_on_scene(env):
    # a rendered scene, full parameters: the paper order matches the oracle's
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 5)
    w, h = q.width, q.height
    p = sff.default_params()
    imgs = q.images()
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in imgs]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    op = _oparams(orc, p)
    op.order_mode = orc.SEQUENTIAL_SCAN
    feats = [orc.features(im, op)[0] for im in imgs]
    field = torch.empty((h, w, 4), dtype=torch.int16, device="cuda")
    cost = torch.empty((h, w), dtype=torch.int32, device="cuda")
    sff.match_views_sequential(pyrs[0], pyrs[2], pyrs[1], pyrs[3], w, h, 0, 9, field, cost, ws, p)
    torch.cuda.synchronize()
    of, oc = orc.match_views(feats[0], feats[2], feats[1], feats[3], 0, 9, op)
    assert np.array_equal(cost.cpu().numpy(), oc)
    assert np.array_equal(field.cpu().numpy(), of)
    # and it differs from the checkerboard order (the two orders are not the same method)
    fc = torch.empty_like(field)
    cc = torch.empty_like(cost)
    sff.match_views(pyrs[0], pyrs[2], pyrs[1], pyrs[3], w, h, 0, 9, fc, cc, ws, p)
    torch.cuda.synchronize()
    assert not np.array_equal(fc.cpu().numpy(), of)


@pytest.mark.parametrize("size,params", [((256, 80), {}), ((37, 23), {}), ((96, 40), {"num_scales": 2}),
                                         ((130, 70), {"iterations": 3, "knn_temporal": 8})])
def test_match_quad_equals_two_match_views(env, size, params):
    # both fields in shared launches == the two single-field calls (and the oracle)
    torch, sff, orc = env
    w, h = size
    imgs = scenegen.random_images(w, h, seed=3 * w + h)
    p = sff.default_params(**params)
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in imgs]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
    cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
    sff.match_quad(*pyrs, w, h, 99, out[0], cst[0], out[1], cst[1], ws, p)
    torch.cuda.synchronize()
    (f0, c0, of0, oc0), (f1, c1, of1, oc1) = _match_both(env, imgs, p, seed=99)
    assert np.array_equal(out[0].cpu().numpy(), f0) and np.array_equal(cst[0].cpu().numpy(), c0)
    assert np.array_equal(out[1].cpu().numpy(), f1) and np.array_equal(cst[1].cpu().numpy(), c1)
    assert np.array_equal(f0, of0) and np.array_equal(f1, of1)


@pytest.mark.parametrize("seed", [1, 2])
def test_match_views_planes_scene(env, seed):
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", seed)
    p = sff.default_params()
    for gf, gc, of, oc in _match_both(env, list(q.images()), p, seed=seed * 31):
        assert np.array_equal(gc, oc)
        assert np.array_equal(gf, of)


def _run_gpu_quad(torch, sff, q, seed, p=None, mode="batch"):
    m = sff.QuadMatcher(q.width, q.height, p, mode=mode)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    seeds, count = m.run(*dev, seed=seed)
    torch.cuda.synchronize()
    n = int(count.item())
    return m, sff.seeds_to_numpy(seeds.cpu().numpy(), min(n, m.capacity)), n


def _assert_quad_equal(m, got_seeds, n, ref):
    assert np.array_equal(m.fwd_cost.cpu().numpy(), ref["fwd_cost"])
    assert np.array_equal(m.fwd.cpu().numpy(), ref["fwd"])
    assert np.array_equal(m.inv_cost.cpu().numpy(), ref["inv_cost"])
    assert np.array_equal(m.inv.cpu().numpy(), ref["inv"])
    assert np.array_equal(m.cerr.cpu().numpy(), ref["cerr"])
    assert np.array_equal(m.keep.cpu().numpy(), ref["keep"])
    assert n == len(ref["seeds"])
    assert got_seeds.tobytes() == ref["seeds"].tobytes()


@pytest.mark.parametrize("name,seed,mode", [("planes_256x80", 1, "batch"), ("planes_256x80", 5, "batch"),
                                            ("planes_256x80", 5, "calls")])
def test_full_stage_small(env, name, seed, mode):
    torch, sff, orc = env
    q = scenegen.make_named(name, seed)
    m, got, n = _run_gpu_quad(torch, sff, q, seed=seed, mode=mode)
    ref = orc.run_quad(*q.images(), seed=seed)
    _assert_quad_equal(m, got, n, ref)


def test_full_stage_shift_scene(env):
    torch, sff, orc = env
    q = scenegen.make_shift_quad(160, 96, 31, u=-6, v=3, d0=2, d1=9)
    m, got, n = _run_gpu_quad(torch, sff, q, seed=3)
    ref = orc.run_quad(*q.images(), seed=3)
    _assert_quad_equal(m, got, n, ref)
    assert (m.fwd.cpu().numpy()[40:-40, 40:-40] == np.array([-6, 3, 2, 9])).all()


@pytest.mark.parametrize("name", ["driving_1242x375", "movie_1024x436"])
def test_full_stage_full_size(env, name):
    torch, sff, orc = env
    q = scenegen.make_named(name, 2)
    m, got, n = _run_gpu_quad(torch, sff, q, seed=2024)
    ref = orc.run_quad(*q.images(), seed=2024)
    _assert_quad_equal(m, got, n, ref)


def test_filter_and_seeds_on_oracle_fields(env):
    # the filter and the seed emission in isolation, fed the oracle's fields
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 4)
    ref = orc.run_quad(*q.images(), seed=9)
    h, w = q.height, q.width
    p = sff.default_params(region_min=60)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    fwd, fc, inv, ic = t(ref["fwd"]), t(ref["fwd_cost"]), t(ref["inv"]), t(ref["inv_cost"])
    keep = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    cerr = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.consistency_filter(fwd, fc, inv, ic, keep, cerr, ws, p)
    okeep, ocerr = orc.consistency_filter(ref["fwd"], ref["fwd_cost"], ref["inv"], ref["inv_cost"],
                                          _oparams(orc, p))
    torch.cuda.synchronize()
    assert np.array_equal(keep.cpu().numpy(), okeep)
    assert np.array_equal(cerr.cpu().numpy(), ocerr)
    # seeds with too small a capacity: the count is still the total
    cap = sff.seed_capacity(w, h)
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    sff.emit_seeds(fwd, fc, keep, cerr, seeds, 10, count, ws)
    torch.cuda.synchronize()
    osd = orc.emit_seeds(ref["fwd"], ref["fwd_cost"], okeep, ocerr)
    assert int(count.item()) == len(osd)
    assert sff.seeds_to_numpy(seeds.cpu().numpy(), 10).tobytes() == osd[:10].tobytes()
    assert (seeds.cpu().numpy()[200:] == 0).all()


def test_region_filter_random_pieces(env):
    # union-find components vs the oracle's BFS on fields with many small regions
    torch, sff, orc = env
    rng = np.random.default_rng(12)
    h, w = 200, 333
    fwd = rng.integers(-2, 3, (h, w, 4)).astype(np.int16)  # neighbours often within tau_r
    fwd[..., 0] += (rng.integers(0, 4, (h // 10 + 1, w // 10 + 1)) * 5).repeat(10, 0).repeat(10, 1)[:h, :w]
    fc = np.zeros((h, w), np.int32)
    fc[rng.random((h, w)) < 0.05] = 2147483647
    inv = np.zeros_like(fwd)
    ic = np.zeros_like(fc)
    # consistency: feed an inverse that makes ~70 % pass
    for y in range(h):
        for x in range(w):
            u, v, d0, d1 = (int(a) for a in fwd[y, x])
            qx, qy = x + u - d1, y + v
            if 0 <= qx < w and 0 <= qy < h and rng.random() < 0.7:
                inv[qy, qx] = (-(u - d1 + d0), -v, d1, d0)
    p = sff.default_params(region_min=25)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    keep = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    cerr = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.consistency_filter(t(fwd), t(fc), t(inv), t(ic), keep, cerr, ws, p)
    okeep, ocerr = orc.consistency_filter(fwd, fc, inv, ic, _oparams(orc, p))
    torch.cuda.synchronize()
    assert np.array_equal(cerr.cpu().numpy(), ocerr)
    assert np.array_equal(keep.cpu().numpy(), okeep)


def test_run_host_matches_device_path(env):
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 6)
    m = sff.QuadMatcher(q.width, q.height)
    a = m.run_host(*q.images(), seed=77)
    b = m.run_host(*q.images(), seed=77)
    ref = orc.run_quad(*q.images(), seed=77)
    assert a.tobytes() == ref["seeds"].tobytes() == b.tobytes()


def test_no_device_wait_timed_out(env):
    # every bounded device-side wait of the runs above completed
    torch, sff, orc = env
    assert sff.device_timeouts() == 0


def test_every_tuning_gives_identical_fields(env):
    # lanes per pixel and tile shape change the work distribution, never the result
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 7)
    w, h = q.width, q.height
    p = sff.default_params()
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in q.images()]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    ref = None
    # the throughput form at scale 0 (coarse scales derived), then every
    # variant of both forms at all four scales
    space = [sff.make_tuning(*cand) for cand in sff.TUNING_SPACE]
    space += [sff.make_tuning(v[0], v[2], v[3], v[1], [v] * 3, min_ctas=v[4]) for v in sff.VARIANT_SPACE]
    # the schedules: the two fields of the quad alternating tile by tile, and
    # every other launch visiting its tiles last-to-first
    space += [sff.make_tuning(1, 32, 16, 0, None, 0, 1), sff.make_tuning(1, 8, 8, 4, [(1, 4, 8, 8)] * 3, 0, 1),
              sff.make_tuning(1, 32, 8, 0, None, 0, 0, 0, 1), sff.make_tuning(1, 32, 8, 0, None, 0, 1, 0, 15),
              sff.make_tuning(2, 16, 8, 1, [(1, 4, 16, 8)] * 3, 0, 1, 0, 10),
              # programmatic dependent launch of the iterations
              sff.make_tuning(1, 32, 16, 0, [(1, 0, 32, 8, 7), (2, 1, 32, 8), (1, 4, 16, 8)], 0, 1, 0, 9, 0, 1)]
    for t in space:
        cand = t.scale_variants()
        out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
        cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
        sff.match_quad_tuned(*pyrs, w, h, 5, t, out[0], cst[0], out[1], cst[1], ws, p)
        torch.cuda.synchronize()
        got = [a.cpu().numpy() for a in out + cst]
        if ref is None:
            ref = got
            o = orc.run_quad(*q.images(), seed=5)
            assert np.array_equal(got[0], o["fwd"]) and np.array_equal(got[1], o["inv"])
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), cand


@pytest.mark.parametrize("size", [(250, 77), (97, 41)])
def test_latency_form_on_ragged_grids(env, size):
    # the latency form of the iteration kernel (slots 1 and 4) and the
    # register-budgeted throughput form on grids that leave partial tiles at
    # every scale, against the oracle
    torch, sff, orc = env
    w, h = size
    q = scenegen.make_quad("planes", w, h, seed=w + h)
    p = sff.default_params()
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in q.images()]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    o = orc.run_quad(*q.images(), seed=9)
    for (l, c, tx, ty, mb) in [v for v in sff.VARIANT_SPACE if v[1] > 0 or v[4] > 0]:
        t = sff.make_tuning(l, tx, ty, c, [(l, c, tx, ty, mb)] * 3, min_ctas=mb)
        out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
        cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
        sff.match_quad_tuned(*pyrs, w, h, 9, t, out[0], cst[0], out[1], cst[1], ws, p)
        torch.cuda.synchronize()
        assert np.array_equal(out[0].cpu().numpy(), o["fwd"]), (l, c, tx, ty, mb)
        assert np.array_equal(out[1].cpu().numpy(), o["inv"]), (l, c, tx, ty, mb)
        assert np.array_equal(cst[0].cpu().numpy(), o["fwd_cost"]), (l, c, tx, ty, mb)
        assert np.array_equal(cst[1].cpu().numpy(), o["inv_cost"]), (l, c, tx, ty, mb)


@pytest.mark.parametrize("size,iterations", [((250, 77), 12), ((97, 41), 12), ((250, 77), 5), ((97, 41), 1)])
def test_fused_coarse_scales_on_ragged_grids(env, size, iterations):
    # all iterations of each coarse scale in one cooperative launch (every
    # fused variant), with even, odd and single iteration counts (the buffer
    # parity and the no-barrier case), against the oracle
    torch, sff, orc = env
    w, h = size
    q = scenegen.make_quad("planes", w, h, seed=w + h + iterations)
    p = sff.default_params(iterations=iterations)
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in q.images()]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    o = orc.run_quad(*q.images(), seed=13, params=_oparams(orc, p))
    sff.device_status(reset=True)
    for v in sff.FUSED_SPACE + [None]:  # None: the variants derived from the grid sizes
        t = sff.make_tuning(1, 32, 16, 0, None if v is None else [v] * 3, fuse=14)
        out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
        cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
        sff.match_quad_tuned(*pyrs, w, h, 13, t, out[0], cst[0], out[1], cst[1], ws, p)
        torch.cuda.synchronize()
        assert np.array_equal(out[0].cpu().numpy(), o["fwd"]), v
        assert np.array_equal(out[1].cpu().numpy(), o["inv"]), v
        assert np.array_equal(cst[0].cpu().numpy(), o["fwd_cost"]), v
        assert np.array_equal(cst[1].cpu().numpy(), o["inv_cost"]), v
    assert sff.device_status(reset=True) == sff.OK


def test_fused_scales_with_more_tiles_than_resident_ctas(env):
    # 1242x375 driving quad, 8x8 tiles: scale 1 has 2 x 78 x 24 = 3744 tiles,
    # more than the cooperative grid holds, so each CTA loops over tiles;
    # scales 1 and 2 fused, 3 not, one fused scale with a 4-slot variant, and
    # the throughput form fused
    torch, sff, orc = env
    q = scenegen.make_named("driving_1242x375", 3)
    w, h = q.width, q.height
    p = sff.default_params()
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in q.images()]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    o = orc.run_quad(*q.images(), seed=21)
    sff.device_status(reset=True)
    for coarse, fuse in [([(1, 1, 8, 8), (1, 1, 8, 8), (1, 4, 16, 8)], 6), ([(2, 1, 8, 8), (1, 4, 8, 8), (0,) * 5], 2),
                         ([(1, 1, 32, 16), (2, 1, 32, 8), (1, 4, 16, 8)], 14),
                         # throughput form: scale 1 in 2 x 20 x 12 tiles of 32x16, 2 CTAs per SM
                         ([(1, 0, 32, 16), (1, 0, 32, 8, 7), (1, 0, 32, 8)], 14)]:
        t = sff.make_tuning(1, 32, 16, 0, coarse, 0, 1, 0, 1, 0, 1, fuse=fuse)
        out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
        cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
        sff.match_quad_tuned(*pyrs, w, h, 21, t, out[0], cst[0], out[1], cst[1], ws, p)
        torch.cuda.synchronize()
        assert np.array_equal(out[0].cpu().numpy(), o["fwd"]), (coarse, fuse)
        assert np.array_equal(out[1].cpu().numpy(), o["inv"]), (coarse, fuse)
        assert np.array_equal(cst[0].cpu().numpy(), o["fwd_cost"]), (coarse, fuse)
        assert np.array_equal(cst[1].cpu().numpy(), o["inv_cost"]), (coarse, fuse)
    assert sff.device_status(reset=True) == sff.OK


@pytest.mark.parametrize("size", [(250, 77), (97, 41), (8, 8), (1242, 375)])
def test_tma_staged_reference_records(env, size):
    # scale 0 with each CTA's region of reference records staged by one
    # tensor copy (every TMA variant; plain and paired / reversed / dependent
    # launches), on ragged grids, the minimum image (the box larger than the
    # image) and the full driving quad, against the oracle
    torch, sff, orc = env
    w, h = size
    q = (scenegen.make_named("driving_1242x375", 4) if size == (1242, 375)
         else scenegen.make_quad("planes", w, h, seed=w * h % 97))
    p = sff.default_params()
    pyrs = [_gpu_features(torch, sff, im, p)[0] for im in q.images()]
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    o = orc.run_quad(*q.images(), seed=17)
    sff.device_status(reset=True)
    for v in sff.TMA_SPACE:
        for pair, alt, pdl in ((0, 0, 0), (1, 1, 1)):
            t = sff.make_tuning(v[0], v[2], v[3], v[1], None, 0, pair, v[4], alt, 0, pdl, tma=1)
            out = [torch.empty((h, w, 4), dtype=torch.int16, device="cuda") for _ in range(2)]
            cst = [torch.empty((h, w), dtype=torch.int32, device="cuda") for _ in range(2)]
            sff.match_quad_tuned(*pyrs, w, h, 17, t, out[0], cst[0], out[1], cst[1], ws, p)
            torch.cuda.synchronize()
            cfg = (v, pair, alt, pdl)
            assert np.array_equal(out[0].cpu().numpy(), o["fwd"]), cfg
            assert np.array_equal(out[1].cpu().numpy(), o["inv"]), cfg
            assert np.array_equal(cst[0].cpu().numpy(), o["fwd_cost"]), cfg
            assert np.array_equal(cst[1].cpu().numpy(), o["inv_cost"]), cfg
    assert sff.device_status(reset=True) == sff.OK


def test_batch_of_uneven_quads_equals_each_alone(env):
    # quads of different sizes and seeds in shared launches (sff_run_batch):
    # every quad's fields, masks and seeds equal the oracle's run on it alone
    torch, sff, orc = env
    specs = [("planes", 256, 80, 1, 11), ("planes", 96, 40, 2, 12), ("planes", 130, 70, 3, 13),
             ("planes", 64, 48, 4, 14), ("shift", 160, 96, 5, 15)]
    quads = []
    for fam, w, h, sd, ms in specs:
        q = (scenegen.make_shift_quad(w, h, sd, u=-3, v=2, d0=4, d1=6) if fam == "shift"
             else scenegen.make_quad(fam, w, h, sd))
        quads.append((q, ms))
    refs = [orc.run_quad(*q.images(), seed=ms) for q, ms in quads]
    bm = sff.BatchMatcher([(q.width, q.height) for q, _ in quads])
    for k, (q, _) in enumerate(quads):
        bm.load(k, *q.images())
    # sweep schedules of scale 0: all quads in every launch, every quad alone
    # (a budget below any quad), about two quads per group, and each with the
    # two fields of a quad alternating tile by tile
    # (and the features on the tensor cores or in the separable form; the
    # iterations with programmatic dependent launch; scale 0 with TMA-staged
    # reference records; the finer scales' features on the second stream or
    # on the caller's)
    for group_mb, pair, alt, form, pdl, tma, ov in ((0, 0, 0, 0, 0, 0, 1), (1, 0, 0, 0, 0, 0, 1),
                                                    (4, 0, 0, 0, 0, 0, 0), (0, 1, 0, 0, 0, 0, 0),
                                                    (4, 1, 0, 1, 0, 0, 1), (0, 0, 1, 0, 1, 0, 1),
                                                    (4, 1, 1, 1, 1, 0, 0), (0, 1, 1, 0, 1, 1, 1),
                                                    (4, 0, 0, 0, 0, 1, 1), (0, 1, 1, 2, 1, 0, 1),
                                                    (0, 1, 1, 2, 1, 0, 0)):
        bm.tuning = sff.make_tuning(1, 32, 16, 0, None, group_mb, pair, 0, alt, form, pdl, tma=tma, overlap=ov)
        bm.run([ms for _, ms in quads])
        torch.cuda.synchronize()
        for (q, ms), b, ref in zip(quads, bm.quads, refs):
            cfg = (group_mb, pair, alt, form, pdl, tma, ov)
            assert np.array_equal(b.fwd.cpu().numpy(), ref["fwd"]), cfg
            assert np.array_equal(b.inv.cpu().numpy(), ref["inv"]), cfg
            assert np.array_equal(b.fwd_cost.cpu().numpy(), ref["fwd_cost"]), cfg
            assert np.array_equal(b.keep.cpu().numpy(), ref["keep"]), cfg
            assert np.array_equal(b.cerr.cpu().numpy(), ref["cerr"]), cfg
            assert b.seeds_numpy().tobytes() == ref["seeds"].tobytes(), cfg


def test_batch_in_stream_groups_equals_oracle(env):
    # the batch split into groups on concurrent streams (BatchMatcher.streams),
    # run directly and replayed from a CUDA graph: every quad's outputs equal
    # the oracle's run on it alone
    torch, sff, orc = env
    specs = [("planes", 256, 80, 1, 11), ("planes", 96, 40, 2, 12), ("planes", 130, 70, 3, 13),
             ("planes", 64, 48, 4, 14), ("shift", 160, 96, 5, 15)]
    quads = []
    for fam, w, h, sd, ms in specs:
        q = (scenegen.make_shift_quad(w, h, sd, u=-3, v=2, d0=4, d1=6) if fam == "shift"
             else scenegen.make_quad(fam, w, h, sd))
        quads.append((q, ms))
    refs = [orc.run_quad(*q.images(), seed=ms) for q, ms in quads]
    bm = sff.BatchMatcher([(q.width, q.height) for q, _ in quads])
    for k, (q, _) in enumerate(quads):
        bm.load(k, *q.images())
    seeds = [ms for _, ms in quads]
    for ns in (2, 3, 5):
        bm.streams = ns
        for how in ("run", "graph"):
            for b in bm.quads:
                b.fwd.zero_()
                b.seeds.zero_()
            if how == "run":
                bm.run(seeds)
            else:
                g = bm.capture(seeds)
                for b in bm.quads:
                    b.fwd.zero_()
                    b.seeds.zero_()
                g.replay()
            torch.cuda.synchronize()
            for (q, ms), b, ref in zip(quads, bm.quads, refs):
                assert np.array_equal(b.fwd.cpu().numpy(), ref["fwd"]), (ns, how)
                assert np.array_equal(b.inv.cpu().numpy(), ref["inv"]), (ns, how)
                assert np.array_equal(b.keep.cpu().numpy(), ref["keep"]), (ns, how)
                assert b.seeds_numpy().tobytes() == ref["seeds"].tobytes(), (ns, how)


def test_mixed_32_quad_batch_equals_oracle(env):
    # the benchmark's 32-quad batch (8 each of 1242x375 and 1024x436 driving
    # scenes, 640x192 and 512x160 planes scenes, scene seeds 100..131) in
    # shared launches under one CUDA graph: every one of the 32 quads' fields,
    # costs, masks and seeds equals the oracle's run on that quad alone
    torch, sff, orc = env
    import bench
    quads, seeds = bench.make_batch_quads()
    sizes = [(im[0].shape[1], im[0].shape[0]) for im in quads]
    assert sorted(set(sizes)) == [(512, 160), (640, 192), (1024, 436), (1242, 375)]
    bm = sff.BatchMatcher(sizes)
    for k, im in enumerate(quads):
        bm.load(k, *im)
    g = bm.capture(seeds)
    g.replay()
    torch.cuda.synchronize()
    for k, (im, b) in enumerate(zip(quads, bm.quads)):
        ref = orc.run_quad(*im, seed=seeds[k])
        assert np.array_equal(b.fwd.cpu().numpy(), ref["fwd"]), k
        assert np.array_equal(b.inv.cpu().numpy(), ref["inv"]), k
        assert np.array_equal(b.fwd_cost.cpu().numpy(), ref["fwd_cost"]), k
        assert np.array_equal(b.inv_cost.cpu().numpy(), ref["inv_cost"]), k
        assert np.array_equal(b.keep.cpu().numpy(), ref["keep"]), k
        assert np.array_equal(b.cerr.cpu().numpy(), ref["cerr"]), k
        assert b.seeds_numpy().tobytes() == ref["seeds"].tobytes(), k
    assert sff.device_timeouts() == 0


@pytest.mark.parametrize("size", [(64, 48), (256, 80)])
@pytest.mark.parametrize("iterations", [0, 12])
def test_all_ties_initialisation(env, size, iterations):
    # a constant image: every feature is zero, so every temporal K-NN
    # candidate ties at the bound (the tensor-core scan's append buffers fill
    # and compact on the first tile), every epipolar candidate ties and every
    # initial combination costs 0.  Both passes equal the oracle, and without
    # iterations the coarsest grid holds the oracle pin's closed form: the
    # temporal point (0, 0) and the stereo / cross points of lowest x that the
    # sign of d allows
    torch, sff, orc = env
    w, h = size
    img = np.full((h, w, 3), 90, np.uint8)
    p = sff.default_params(iterations=iterations)
    n = 1 << (p.num_scales - 1)
    for mirror, (f, c, of, oc) in enumerate(_match_both(env, [img] * 4, p, seed=3)):
        assert np.array_equal(f, of) and np.array_equal(c, oc), mirror
        if iterations == 0:
            for py in range(0, h, n):
                for px in range(0, w, n):
                    assert tuple(int(v) for v in f[py, px]) == (-px, -py, 0 if mirror else px, 0), (mirror, px, py)
                    assert c[py, px] == 0
    assert sff.device_timeouts() == 0


def test_batch_graph_replay_is_deterministic(env):
    torch, sff, orc = env
    qs = [scenegen.make_quad("planes", 128, 64, s) for s in (21, 22, 23)]
    bm = sff.BatchMatcher([(128, 64)] * 3)
    for k, q in enumerate(qs):
        bm.load(k, *q.images())
    g = bm.capture([1, 2, 3])
    g.replay()
    torch.cuda.synchronize()
    first = [b.seeds_numpy().tobytes() for b in bm.quads]
    g.replay()
    torch.cuda.synchronize()
    assert first == [b.seeds_numpy().tobytes() for b in bm.quads]
    ref = orc.run_quad(*qs[1].images(), seed=2)
    assert first[1] == ref["seeds"].tobytes()
