"""Disparity fill (Sec. 3.1, last paragraph) on the GPU vs the CPU oracle,
through the C ABI: the SGM disparity map and the seeds with disparity-only
entries are integers and must be identical."""
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


def _gpu_sgm(env, left, right, **over):
    torch, sff, _ = env
    h, w, _ = left.shape
    p = sff.default_sgm_params(**over)
    disp = torch.full((h, w), -7, dtype=torch.int16, device="cuda")
    ws = torch.empty(sff.sgm_workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.sgm(torch.as_tensor(left).cuda(), torch.as_tensor(right).cuda(), disp, ws, p)
    torch.cuda.synchronize()
    return disp.cpu().numpy()


@pytest.mark.parametrize("size,D,p1,p2", [((37, 23), 32, 10, 120), ((130, 70), 64, 10, 120), ((300, 9), 32, 3, 40),
                                          ((64, 48), 128, 0, 0), ((97, 41), 256, 15, 193), ((8, 8), 32, 10, 120)])
def test_sgm_random_images(env, size, D, p1, p2):
    w, h = size
    L, R = scenegen.random_images(w, h, seed=w + 7 * h, n=2)
    got = _gpu_sgm(env, L, R, max_disp=D, p1=p1, p2=p2)
    want = env[2].sgm(L, R, env[2].sgm_params(max_disp=D, p1=p1, p2=p2))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name,D", [("planes_256x80", 64), ("driving_1242x375", 128)])
def test_sgm_scenes(env, name, D):
    q = scenegen.make_named(name, 2)
    got = _gpu_sgm(env, q.L0, q.R0, max_disp=D)
    want = env[2].sgm(q.L0, q.R0, env[2].sgm_params(max_disp=D))
    assert np.array_equal(got, want)


def test_sgm_shift_scene_is_exact(env):
    q = scenegen.make_shift_quad(160, 96, 31, u=-6, v=3, d0=11, d1=9)
    got = _gpu_sgm(env, q.L0, q.R0, max_disp=32)
    assert (got[3:-3, 15:-4] == 11).all()


def test_sgm_rejects_bad_parameters(env):
    torch, sff, _ = env
    for over in (dict(max_disp=96), dict(p1=20, p2=10), dict(p2=194)):
        p = sff.default_sgm_params(**over)
        assert sff.sgm_workspace_bytes(64, 48, p) == 0
        with pytest.raises(sff.SffError):
            sff.sgm(torch.zeros((48, 64, 3), dtype=torch.uint8, device="cuda"),
                    torch.zeros((48, 64, 3), dtype=torch.uint8, device="cuda"),
                    torch.empty((48, 64), dtype=torch.int16, device="cuda"),
                    torch.empty(1 << 20, dtype=torch.uint8, device="cuda"), p)


@pytest.mark.parametrize("name,seed", [("planes_256x80", 1), ("planes_256x80", 5)])
def test_seeds_with_disparity_fill(env, name, seed):
    # the oracle's fields and SGM map go to both sides' seed emission
    torch, sff, orc = env
    q = scenegen.make_named(name, seed)
    ref = orc.run_quad(*q.images(), seed=seed)
    disp = orc.sgm(q.L0, q.R0, orc.sgm_params(max_disp=64))
    want = orc.emit_seeds_geo(ref["fwd"], ref["fwd_cost"], ref["keep"], ref["cerr"], disp, tau_c=1)
    assert (want["kind"] == 1).sum() > 0
    h, w = q.height, q.width
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    cap = sff.seed_capacity(w, h)
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h), dtype=torch.uint8, device="cuda")
    sff.emit_seeds_geo(t(ref["fwd"]), t(ref["fwd_cost"]), t(ref["keep"]), t(ref["cerr"]), t(disp), seeds, cap,
                       count, ws)
    torch.cuda.synchronize()
    n = int(count.item())
    assert n == len(want)
    assert sff.seeds_to_numpy(seeds.cpu().numpy(), n).tobytes() == want.tobytes()


def test_whole_stage_with_fill(env):
    # matching stage + SGM + seeds with the fill on the GPU against the oracle's
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 3)
    m = sff.QuadMatcher(q.width, q.height)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    m.run(*dev, seed=3)
    p = sff.default_sgm_params(max_disp=64)
    disp = torch.empty((q.height, q.width), dtype=torch.int16, device="cuda")
    sws = torch.empty(sff.sgm_workspace_bytes(q.width, q.height, p), dtype=torch.uint8, device="cuda")
    sff.sgm(dev[0], dev[1], disp, sws, p)
    cap = sff.seed_capacity(q.width, q.height)
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(sff.workspace_bytes(q.width, q.height), dtype=torch.uint8, device="cuda")
    sff.emit_seeds_geo(m.fwd, m.fwd_cost, m.keep, m.cerr, disp, seeds, cap, count, ws)
    torch.cuda.synchronize()
    ref = orc.run_quad(*q.images(), seed=3)
    odisp = orc.sgm(q.L0, q.R0, orc.sgm_params(max_disp=64))
    want = orc.emit_seeds_geo(ref["fwd"], ref["fwd_cost"], ref["keep"], ref["cerr"], odisp, tau_c=1)
    assert np.array_equal(disp.cpu().numpy(), odisp)
    n = int(count.item())
    assert sff.seeds_to_numpy(seeds.cpu().numpy(), n).tobytes() == want.tobytes()


def test_interpolation_of_seeds_with_the_fill(env):
    # each side interpolates its own seeds with disparity-only entries: those
    # join the plane fits only (d1 = 0 keeps them out of the motion fits)
    torch, sff, orc = env
    q = scenegen.make_named("planes_256x80", 5)
    w, h = q.width, q.height
    m = sff.QuadMatcher(w, h)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    m.run(*dev, seed=5)
    p = sff.default_sgm_params(max_disp=64)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    sws = torch.empty(sff.sgm_workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    sff.sgm(dev[0], dev[1], disp, sws, p)
    cap = sff.seed_capacity(w, h)
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(sff.workspace_bytes(w, h), dtype=torch.uint8, device="cuda")
    sff.emit_seeds_geo(m.fwd, m.fwd_cost, m.keep, m.cerr, disp, seeds, cap, count, ws)
    ip = sff.default_interp_params(w, h, q.focal, q.baseline)
    field = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
    iws = torch.empty(sff.interp_workspace_bytes(w, h, cap), dtype=torch.uint8, device="cuda")
    sff.interpolate(seeds, count, cap, w, h, ip, field, iws)
    torch.cuda.synchronize()
    ref = orc.run_quad(*q.images(), seed=5)
    od = orc.sgm(q.L0, q.R0, orc.sgm_params(max_disp=64))
    os_ = orc.emit_seeds_geo(ref["fwd"], ref["fwd_cost"], ref["keep"], ref["cerr"], od, tau_c=1)
    assert (os_["kind"] == 1).sum() > 0
    want = orc.interpolate(os_, w, h, orc.interp_params(w, h, q.focal, q.baseline))
    assert sff.interp_status(iws, w, h, cap) == 0
    np.testing.assert_allclose(field.cpu().numpy(), want, rtol=1e-5, atol=1e-3)
