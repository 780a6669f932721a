"""Device-side error status through the C ABI (sff_device_status).

A bounded device wait that runs out, and a seed buffer smaller than the
number of seeds, are reported when the caller synchronises; the context stays
usable and the next run is exact.  The waits are made to run out with the
library's failure injection: the thread that issues the temporal K-NN's
tensor-core MMAs stops before one step and issues nothing further
(sff_debug_knn_withhold), so the warps waiting for that step's results give
up after a short limit; or one CTA of a fused iteration launch leaves before
a grid barrier (sff_debug_barrier_withhold), so the others' barrier waits
give up.  Nothing faults: no copy or MMA is left in flight when a CTA exits.
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


def test_withheld_mma_step_times_out_and_is_reported(env):
    torch, sff, orc = env
    # 512 x 160: 1280 coarsest-grid points = 10 candidate tiles, 20 steps, so
    # the bulk-copy thread also waits (for a stage to free up) and gives up
    q = scenegen.make_quad("planes", 512, 160, seed=31)
    m = sff.QuadMatcher(q.width, q.height)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    # the conditions are per device and persist until read: clear what
    # earlier calls of this process raised (a deliberately small seed buffer)
    sff.device_status(reset=True)
    m.run(*dev, seed=5)
    assert sff.device_status(reset=True) == sff.OK
    sff.device_timeouts(reset=True)
    try:
        # step 0: nothing issued at all; step 13: in the second pass, after
        # 13 committed steps that the MMA thread drains
        for step in (0, 13):
            sff.debug_knn_withhold(step, wait_limit_us=20000)
            m.run(*dev, seed=5)
            assert sff.device_status(reset=True) == sff.ERR_TIMEOUT, step
            assert sff.device_timeouts(reset=True) > 0, step
            assert sff.device_drain_timeouts() == 0, step
            # no field holds a vector from a stale candidate list: pixels are
            # empty or hold the (integer) vectors the stage computed
            assert m.fwd.shape == (q.height, q.width, 4)
    finally:
        sff.debug_knn_withhold(-1, 0)
    # the context is usable and the next run is exact and clean
    m.run(*dev, seed=5)
    assert sff.device_status(reset=True) == sff.OK
    assert sff.device_timeouts() == 0
    ref = orc.run_quad(*q.images(), seed=5)
    assert np.array_equal(m.fwd.cpu().numpy(), ref["fwd"])
    assert np.array_equal(m.inv.cpu().numpy(), ref["inv"])
    got = sff.seeds_to_numpy(m.seeds.cpu().numpy(), int(m.count.item()))
    assert got.tobytes() == ref["seeds"].tobytes()


def test_small_seed_buffer_reports_capacity(env):
    torch, sff, orc = env
    q = scenegen.make_quad("planes", 256, 80, seed=32)
    m = sff.QuadMatcher(q.width, q.height)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    sff.device_status(reset=True)
    m.run(*dev, seed=6)
    assert sff.device_status(reset=True) == sff.OK
    full = int(m.count.item())
    assert full > 10
    cap = full // 2
    seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(sff.workspace_bytes(q.width, q.height), dtype=torch.uint8, device="cuda")
    sff.emit_seeds(m.fwd, m.fwd_cost, m.keep, m.cerr, seeds, cap, count, ws)
    assert sff.device_status(reset=True) == sff.ERR_CAPACITY
    assert int(count.item()) == full  # the number needed
    want = sff.seeds_to_numpy(m.seeds.cpu().numpy(), full)[:cap]
    assert sff.seeds_to_numpy(seeds.cpu().numpy(), cap).tobytes() == want.tobytes()
    # an exact fit is no error, and the condition was cleared by the read
    seeds2 = torch.zeros(20 * full, dtype=torch.uint8, device="cuda")
    sff.emit_seeds(m.fwd, m.fwd_cost, m.keep, m.cerr, seeds2, full, count, ws)
    assert sff.device_status(reset=True) == sff.OK
    with pytest.raises(sff.SffError) as e:
        sff.emit_seeds(m.fwd, m.fwd_cost, m.keep, m.cerr, seeds, cap, count, ws)
        sff.check_device_status()
    assert e.value.status == sff.ERR_CAPACITY


def test_withheld_grid_barrier_times_out_and_is_reported(env):
    torch, sff, orc = env
    q = scenegen.make_quad("planes", 512, 160, seed=33)
    # scales 1..3 fused: every launch has 11 barriers
    t = sff.make_tuning(1, 32, 16, 0, [(1, 1, 16, 8), (2, 1, 16, 8), (1, 4, 16, 8)], fuse=14)
    m = sff.QuadMatcher(q.width, q.height, tuning=t)
    dev = [torch.as_tensor(im).cuda() for im in q.images()]
    sff.device_status(reset=True)
    m.run(*dev, seed=7)
    assert sff.device_status(reset=True) == sff.OK
    sff.device_timeouts(reset=True)
    try:
        for barrier in (0, 10):
            sff.debug_barrier_withhold(barrier, wait_limit_us=20000)
            m.run(*dev, seed=7)
            assert sff.device_status(reset=True) == sff.ERR_TIMEOUT, barrier
            assert sff.device_timeouts(reset=True) > 0, barrier
    finally:
        sff.debug_barrier_withhold(-1, 0)
    # the context is usable, the counters were zeroed again before each
    # scale, and the next run is exact and clean
    m.run(*dev, seed=7)
    assert sff.device_status(reset=True) == sff.OK
    assert sff.device_timeouts() == 0
    ref = orc.run_quad(*q.images(), seed=7)
    assert np.array_equal(m.fwd.cpu().numpy(), ref["fwd"])
    assert np.array_equal(m.inv.cpu().numpy(), ref["inv"])
    got = sff.seeds_to_numpy(m.seeds.cpu().numpy(), int(m.count.item()))
    assert got.tobytes() == ref["seeds"].tobytes()
