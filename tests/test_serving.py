"""Serving: continuous batching with resident slots (paper_1710_10096_gb300.serve).

Host-side logic (arrivals, summaries, admission rules with a fake budget) is
tested without a GPU; the GPU tests check that every request's seeds are
identical whether it is matched alone, through the plain per-request server
or in the mix of the continuous-batching server.
"""
import os

import numpy as np
import pytest

import scenegen


def test_poisson_arrivals_shape():
    from paper_1710_10096_gb300.serve import poisson_arrivals
    arr = poisson_arrivals(100.0, 500, 8, 5, seed=3)
    t = np.array([a[0] for a in arr])
    assert len(arr) == 500 and (np.diff(t) > 0).all()
    assert {a[1] for a in arr} <= set(range(8)) and {a[2] for a in arr} <= set(range(5))
    assert abs(500 / t[-1] - 100.0) < 15.0  # rate within sampling error
    assert arr == poisson_arrivals(100.0, 500, 8, 5, seed=3)  # seeded


def test_summary():
    from paper_1710_10096_gb300.serve import Request, summarize
    reqs = []
    for k in range(100):
        r = Request(k, 0, (np.zeros((10, 20, 3), np.uint8),) * 4, 1, t_arrival=0.0)
        r.t_done = (k + 1) / 1000.0
        reqs.append(r)
    s = summarize(reqs, 0.1)
    assert s["requests"] == 100 and s["rejected"] == 0 and abs(s["p50_ms"] - 50.5) < 1e-6 and s["p99_ms"] > 99.0
    assert s["sustained_px_per_s"] == 100 * 200 / 0.1


def test_malformed_requests_are_rejected_at_submission():
    import collections
    import threading

    from paper_1710_10096_gb300.serve import Request, _submit, validate_request
    good = (np.zeros((20, 30, 3), np.uint8),) * 4
    assert validate_request(Request(0, 0, good, 1)) is None
    bad = {
        "three images": good[:3],
        "other size": good[:3] + (np.zeros((20, 31, 3), np.uint8),),
        "float": (np.zeros((20, 30, 3), np.float32),) * 4,
        "grey": (np.zeros((20, 30), np.uint8),) * 4,
        "too small": (np.zeros((7, 30, 3), np.uint8),) * 4,
    }
    for name, ims in bad.items():
        assert validate_request(Request(0, 0, ims, 1)) is not None, name
    # submission: a malformed request is finished at once with its error and
    # never queued, so it can take no slot
    lock, pending, done = threading.Lock(), collections.deque(), []
    _submit(Request(1, 0, good, 1, t_arrival=2.0), lock, pending, done)
    r = Request(2, 0, bad["other size"], 1, t_arrival=3.0)
    _submit(r, lock, pending, done)
    assert [q.rid for q in pending] == [1] and done == [r]
    assert r.error and r.t_done == r.t_arrival


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_10096_gb300 as sff
    sff.build()
    return torch, sff


def _pool():
    return [scenegen.make_quad("planes", 256, 80, 41).images(), scenegen.make_quad("planes", 192, 96, 42).images(),
            scenegen.make_quad("planes", 128, 64, 43).images(), scenegen.make_shift_quad(160, 96, 44, 3, -2, 5, 4).images()]


@pytest.mark.gpu
def test_served_results_equal_alone(gpu):
    torch, sff = gpu
    from paper_1710_10096_gb300.serve import PlainServer, Server, poisson_arrivals, simulate
    pool = _pool()
    alone = []
    for k, imgs in enumerate(pool):
        m = sff.QuadMatcher(imgs[0].shape[1], imgs[0].shape[0])
        alone.append(m.run_host(*imgs, seed=1000 + k).tobytes())
    arrivals = poisson_arrivals(3000.0, 48, 8, len(pool), seed=5)  # fast arrivals: requests mix in batches
    srv = Server(max_batch=8)
    reqs, wall = simulate(srv, arrivals, pool)
    assert srv.batches < len(reqs)  # requests were actually batched together
    for r in reqs:
        assert r.error is None
        assert r.seeds.tobytes() == alone[arrivals[r.rid][2]]
    plain = PlainServer()
    reqs2, _ = simulate(plain, arrivals, pool)
    for r in reqs2:
        assert r.seeds.tobytes() == alone[arrivals[r.rid][2]]


@pytest.mark.gpu
def test_admission_by_memory_budget(gpu):
    torch, sff = gpu
    from paper_1710_10096_gb300.serve import Server, poisson_arrivals, simulate
    pool = _pool()
    srv = Server(max_batch=8)
    one = max(srv._slot_bytes((im[0].shape[1], im[0].shape[0])) for im in pool)
    srv.hbm_budget = int(1.5 * one)  # room for one slot at a time: admissions wait for memory
    reqs, _ = simulate(srv, poisson_arrivals(2000.0, 12, 4, len(pool), seed=9), pool)
    assert all(r.error is None and r.seeds is not None for r in reqs)
    assert srv.bytes_used <= srv.hbm_budget
    # a request larger than the whole budget is rejected, not queued forever
    srv2 = Server(max_batch=4)
    srv2.hbm_budget = 1 << 20
    big = [scenegen.random_images(256, 80, 3)]
    reqs3, _ = simulate(srv2, [(0.0, 0, 0)], [tuple(big[0])])
    assert reqs3[0].error is not None and reqs3[0].seeds is None
