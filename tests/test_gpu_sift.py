"""The paper's own matching cost (Eq. 1 with SIFT-PCA features) on the GPU
vs the CPU oracle, through the C ABI.  Both sides follow the same fixed
floating-point order without fused multiply-adds, so phi, the fields and
the float costs (as bit patterns) must be identical."""
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


def _gpu_phi(env, images, S):
    torch, sff, _ = env
    h, w, _ = images[0].shape
    dev = [torch.as_tensor(np.ascontiguousarray(im)).cuda() for im in images]
    phis = [torch.full((S, h, w, 4), float("nan"), dtype=torch.float32, device="cuda") for _ in range(4)]
    ws = torch.empty(sff.sift_workspace_bytes(w, h), dtype=torch.uint8, device="cuda")
    sff.sift_features(dev, phis, ws, sff.default_params(num_scales=S))
    torch.cuda.synchronize()
    return dev, phis


@pytest.mark.parametrize("kind,size,S", [("planes", (256, 80), 4), ("random", (37, 23), 3), ("random", (8, 8), 1),
                                          ("movie", (130, 70), 4)])
def test_phi_bit_exact(env, kind, size, S):
    w, h = size
    if kind == "random":
        images = scenegen.random_images(w, h, seed=w * h, n=4)
    else:
        images = list(scenegen.make_quad(kind, w, h, 3).images())
    _, phis = _gpu_phi(env, images, S)
    want, _, _ = env[2].sift_phi(images, num_scales=S)
    for g, o in zip(phis, want):
        assert np.array_equal(g.cpu().numpy(), o)


def _match_both(env, q, seed, S=4):
    torch, sff, orc = env
    p = sff.default_params(num_scales=S)
    op = orc.default_params(**p.as_dict())
    m = sff.QuadMatcher(q.width, q.height, p)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    m.run(*dev, seed=seed)
    _, phis = _gpu_phi(env, list(q.images()), S)
    L0, R0, L1, R1 = m.pyr
    pL0, pR0, pL1, pR1 = phis
    w, h = q.width, q.height
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    out = []
    for roles, phr, mirror in (((L0, L1, R0, R1), (pL0, pL1, pR0, pR1), 0), ((R1, R0, L1, L0), (pR1, pR0, pL1, pL0), 1)):
        f = torch.empty((h, w, 4), dtype=torch.int16, device="cuda")
        c = torch.empty((h, w), dtype=torch.int32, device="cuda")
        sff.match_views_sift(*roles, *phr, w, h, mirror, seed, f, c, ws, p)
        torch.cuda.synchronize()
        out.append((f.cpu().numpy(), c.cpu().numpy()))
    feats = [orc.features(im, op)[0] for im in q.images()]
    ophi, _, _ = orc.sift_phi(list(q.images()), num_scales=S)
    fL0, fR0, fL1, fR1 = feats
    oL0, oR0, oL1, oR1 = ophi
    want = [orc.match_views_sift(fL0, fL1, fR0, fR1, oL0, oL1, oR0, oR1, w, h, 0, seed, op),
            orc.match_views_sift(fR1, fR0, fL1, fL0, oR1, oR0, oL1, oL0, w, h, 1, seed, op)]
    return out, want


@pytest.mark.parametrize("name,seed", [("planes_256x80", 1), ("planes_256x80", 7)])
def test_fields_with_the_sift_cost_bit_exact(env, name, seed):
    q = scenegen.make_named(name, seed)
    got, want = _match_both(env, q, seed)
    for (gf, gc), (of, oc) in zip(got, want):
        assert np.array_equal(gc, oc)
        assert np.array_equal(gf, of)


def test_sift_cost_on_a_shift_scene(env):
    q = scenegen.make_shift_quad(128, 96, 5, u=-3, v=2, d0=6, d1=4)
    got, want = _match_both(env, q, 11)
    (gf, gc), _ = got[0], None
    assert np.array_equal(gf, want[0][0]) and np.array_equal(gc, want[0][1])
    inner = gf[20:-20, 20:-20].reshape(-1, 4)
    assert (inner == np.array([-3, 2, 6, 4])).all(axis=1).mean() > 0.99


def test_full_size_phi_and_cost_property(env):
    # 1242 x 375: phi of all scales bit-exact; the final state's cost at
    # sampled pixels equals the oracle's cost of the final vector
    torch, sff, orc = env
    q = scenegen.make_named("driving_1242x375", 2)
    images = list(q.images())
    _, phis = _gpu_phi(env, images, 4)
    want, _, _ = orc.sift_phi(images, num_scales=4)
    for g, o in zip(phis, want):
        assert np.array_equal(g.cpu().numpy(), o)
    p = sff.default_params()
    m = sff.QuadMatcher(q.width, q.height, p)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    m.run(*dev, seed=2024)
    L0, R0, L1, R1 = m.pyr
    w, h = q.width, q.height
    ws = torch.empty(sff.workspace_bytes(w, h, p), dtype=torch.uint8, device="cuda")
    f = torch.empty((h, w, 4), dtype=torch.int16, device="cuda")
    c = torch.empty((h, w), dtype=torch.int32, device="cuda")
    sff.match_views_sift(L0, L1, R0, R1, phis[0], phis[2], phis[1], phis[3], w, h, 0, 2024, f, c, ws, p)
    torch.cuda.synchronize()
    field, cost = f.cpu().numpy(), c.cpu().numpy()
    rng = np.random.default_rng(4)
    oL0, oR0, oL1, oR1 = (x[0] for x in want)
    for x, y in zip(rng.integers(0, w, 300), rng.integers(0, h, 300)):
        got = np.array([cost[y, x]], np.int32).view(np.float32)[0]
        assert got == orc.sift_cost(oL0, oL1, oR0, oR1, 1, 0, int(x), int(y), field[y, x])
