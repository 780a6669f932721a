"""sff_emit_seeds_noalloc: the allocation-free seed emission.

Some callers cannot allocate device memory -- a component that only receives
device pointers from elsewhere and has no allocator, or a latency-critical
loop that must not call cudaMalloc (which may synchronise the device).  For
them the library keeps the seed emission's scratch in a static device array.
These tests call the entry point through the C ABI and check that it returns
exactly what sff_emit_seeds (which takes a caller-allocated workspace)
returns, on two calls in a row with different inputs and sizes, so that the
shared array's leftover contents from the first call cannot leak into the
second.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest


def _lib():
    import paper_1710_10096_gb300 as sff
    sff.build()
    return sff, sff.lib()


def test_noalloc_rejects_oversized_images_without_gpu():
    sff, L = _lib()
    fake = ctypes.c_void_p(0x10000)
    null = ctypes.c_void_p(0)
    # 4096 x 4096 needs 1366 * 1366 blocks > SFF_NOALLOC_MAX_BLOCKS = 2^19
    assert L.sff_emit_seeds_noalloc(fake, fake, fake, fake, 4096, 4096, fake, 10, fake, null) == -1
    assert L.sff_emit_seeds_noalloc(null, fake, fake, fake, 64, 64, fake, 10, fake, null) == -1


def _random_inputs(torch, w, h, seed):
    rng = np.random.default_rng(seed)
    fwd = rng.integers(-300, 300, (h, w, 4)).astype(np.int16)
    cost = rng.integers(0, 50, (h, w)).astype(np.int32)
    keep = (rng.random((h, w)) > 0.45).astype(np.uint8)
    cerr = rng.integers(0, 4, (h, w)).astype(np.uint8)
    return [torch.as_tensor(a).cuda() for a in (fwd, cost, keep, cerr)]


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sff, L = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ctypes.c_void_p
    for (w, h, seed) in [(1242, 375, 1), (256, 80, 2), (1242, 375, 3)]:
        fwd, cost, keep, cerr = _random_inputs(torch, w, h, seed)
        cap = ((w + 2) // 3) * ((h + 2) // 3)
        ws = torch.empty(sff.workspace_bytes(w, h), dtype=torch.uint8, device="cuda")
        ref_seeds = torch.zeros(20 * cap, dtype=torch.uint8, device="cuda")
        new_seeds = torch.full((20 * cap,), 0xAB, dtype=torch.uint8, device="cuda")
        ref_count = torch.zeros(1, dtype=torch.int32, device="cuda")
        new_count = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        args = [p(fwd.data_ptr()), p(cost.data_ptr()), p(keep.data_ptr()), p(cerr.data_ptr()), w, h]
        assert L.sff_emit_seeds(*args, p(ref_seeds.data_ptr()), cap, p(ref_count.data_ptr()),
                                p(ws.data_ptr()), ws.numel(), stream) == 0
        assert L.sff_emit_seeds_noalloc(*args, p(new_seeds.data_ptr()), cap, p(new_count.data_ptr()), stream) == 0
        torch.cuda.synchronize()
        n = int(ref_count.item())
        assert n > 0 and int(new_count.item()) == n
        assert torch.equal(new_seeds[:20 * n], ref_seeds[:20 * n])
