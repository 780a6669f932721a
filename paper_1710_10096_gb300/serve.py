"""Continuous-batching server for the four-view matching stage.

Requests (one stereo quad each) arrive from several camera streams.  The
server keeps per-size slots of device buffers resident (input images,
feature pyramids, fields, masks, seeds, scratch) and admits a request as soon
as a slot of its size is free or can be allocated within the HBM budget.
Admitted requests are matched together by sff_run_batch (shared launches for
all of them); up to `inflight` batches run at once on separate CUDA streams,
so requests that arrive while a batch is on the GPU start in the next batch
without waiting for it to finish, and their work overlaps on the device.

Every request's result is identical to matching its quad alone (same seed):
the batched kernels compute each quad independently.

PlainServer is the per-request reference: one request at a time, in
arrival order, each matched alone.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from . import OK, QuadBuffers, default_params, default_tuning, device_status, lib, run_batch, seeds_to_numpy

__all__ = ["Request", "Server", "PlainServer", "simulate", "poisson_arrivals", "validate_request"]


@dataclasses.dataclass
class Request:
    rid: int
    stream_id: int
    images: tuple  # L0, R0, L1, R1 host uint8 [H, W, 3]
    seed: int
    t_arrival: float = 0.0  # seconds on the server's clock
    t_done: float = 0.0
    seeds: np.ndarray = None  # result (SEED_DTYPE)
    error: str = None  # set when the request was rejected or its batch raised a device-side condition

    @property
    def size(self):
        return self.images[0].shape[1], self.images[0].shape[0]

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def validate_request(req: Request):
    """Why a request cannot be served (None if it can): four uint8 H x W x 3
    host images of one size within the library's limits (8 .. 16384 px)."""
    ims = req.images
    if not isinstance(ims, (tuple, list)) or len(ims) != 4:
        return "a request holds four images (L0, R0, L1, R1)"
    for k, im in enumerate(ims):
        if not isinstance(im, np.ndarray) or im.dtype != np.uint8 or im.ndim != 3 or im.shape[2] != 3:
            return f"image {k}: expected a uint8 numpy array [H, W, 3]"
        if im.shape != ims[0].shape:
            return f"image {k}: shape {im.shape}, image 0 has {ims[0].shape}"
    h, w = ims[0].shape[:2]
    if not (8 <= w <= 16384 and 8 <= h <= 16384):
        return f"size {w}x{h} outside 8..16384"
    return None


def _submit(req: Request, lock, pending, done) -> None:
    """Queues a request, or finishes it at once with its error when it is malformed."""
    err = validate_request(req)
    with lock:
        if err is None:
            pending.append(req)
        else:
            req.error = err
            req.t_done = req.t_arrival
            done.append(req)


class _Slot:
    """Resident device buffers for one quad size plus pinned host staging."""

    def __init__(self, w, h, params, device):
        import torch
        self.buf = QuadBuffers(w, h, params, device)
        self.host_in = torch.empty((4, h, w, 3), dtype=torch.uint8).pin_memory()
        self.host_seeds = torch.empty(20 * self.buf.capacity, dtype=torch.uint8).pin_memory()
        self.host_count = torch.empty(1, dtype=torch.int32).pin_memory()
        self.nbytes = (sum(t.numel() * t.element_size() for t in
                           [self.buf.dev_in, self.buf.workspace, self.buf.fwd, self.buf.inv, self.buf.fwd_cost,
                            self.buf.inv_cost, self.buf.keep, self.buf.cerr, self.buf.seeds]) +
                       sum(p.numel() for p in self.buf.pyr))
        self.req = None


class Server:
    """Continuous batching with resident slots and admission by HBM budget."""

    def __init__(self, params=None, tuning=None, device="cuda", max_batch: int = 32, hbm_budget: int = 24 << 30,
                 inflight: int = 2):
        import torch
        self.params = params or default_params()
        self.tuning = tuning or default_tuning()
        self.device = torch.device(device)
        self.max_batch = max_batch
        free, _total = torch.cuda.mem_get_info(self.device)
        self.hbm_budget = int(min(hbm_budget, max(0, free - (2 << 30))))
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(inflight)]
        self.busy = [None] * inflight  # (event, [slots]) per stream
        self.slots = collections.defaultdict(list)  # size -> [_Slot]
        self.free = collections.defaultdict(list)
        self.bytes_used = 0
        self.pending = collections.deque()  # arrived, not admitted
        self.admitted = collections.deque()  # admitted to a slot, not started
        self.done = []
        self._lock = threading.Lock()
        self.batches = 0
        self._sizes_cache = {}

    def submit(self, req: Request) -> None:
        _submit(req, self._lock, self.pending, self.done)

    def reserve(self, size, count: int) -> int:
        """Pre-allocate up to `count` idle slots of `size` within the budget
        (allocation is slow: it should not happen while requests wait)."""
        made = 0
        with self._lock:
            while len(self.slots[size]) < count:
                need = self._slot_bytes(size)
                if self.bytes_used + need > self.hbm_budget:
                    break
                slot = _Slot(size[0], size[1], self.params, self.device)
                self.bytes_used += need
                self.slots[size].append(slot)
                self.free[size].append(slot)
                made += 1
        return made

    # --- admission: a free slot of the request's size, or a new one within budget
    def _admit(self):
        while self.pending:
            req = self.pending[0]
            size = req.size
            if self.free[size]:
                slot = self.free[size].pop()
            else:
                need = self._slot_bytes(size)
                if need > self.hbm_budget:  # can never fit: reject instead of blocking the queue
                    self.pending.popleft()
                    req.error = f"needs {need} bytes of device memory, budget {self.hbm_budget}"
                    self.done.append(req)
                    continue
                if self.bytes_used + need > self.hbm_budget:
                    if self._evict_free(need):
                        continue
                    break  # head of line waits for memory
                slot = _Slot(size[0], size[1], self.params, self.device)
                self.bytes_used += need
                self.slots[size].append(slot)
            self.pending.popleft()
            slot.req = req
            for k in range(4):
                slot.host_in[k].numpy()[...] = req.images[k]
            self.admitted.append(slot)

    def _evict_free(self, need: int) -> bool:
        """Release idle slots of other sizes until `need` bytes fit."""
        import torch
        freed = False
        for size in list(self.free):
            while self.free[size] and self.bytes_used + need > self.hbm_budget:
                slot = self.free[size].pop()
                self.slots[size].remove(slot)
                self.bytes_used -= self._slot_bytes(size)
                freed = True
        if freed:
            torch.cuda.empty_cache()
        return freed and self.bytes_used + need <= self.hbm_budget

    def _slot_bytes(self, size) -> int:
        if size not in self._sizes_cache:
            from . import pyramid_bytes, quad_workspace_bytes, seed_capacity
            w, h = size
            self._sizes_cache[size] = (4 * pyramid_bytes(w, h, self.params) + quad_workspace_bytes(w, h, self.params)
                                       + w * h * (12 + 12 + 2 + 12) + 20 * seed_capacity(w, h))
        return self._sizes_cache[size]

    # --- launch a batch of admitted requests on a free stream
    def _launch(self, now_fn):
        import torch
        for k, b in enumerate(self.busy):
            if b is not None or not self.admitted:
                continue
            batch = [self.admitted.popleft() for _ in range(min(self.max_batch, len(self.admitted)))]
            s = self.streams[k]
            with torch.cuda.stream(s):
                for slot in batch:
                    slot.buf.dev_in.copy_(slot.host_in, non_blocking=True)
                run_batch([slot.buf.desc(None, slot.req.seed) for slot in batch], self.params, self.tuning, s)
                for slot in batch:
                    slot.host_count.copy_(slot.buf.count, non_blocking=True)
                    slot.host_seeds.copy_(slot.buf.seeds, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
            self.busy[k] = (ev, batch)
            self.batches += 1

    # --- retire finished batches
    def _retire(self, now_fn):
        for k, b in enumerate(self.busy):
            if b is None or not b[0].query():
                continue
            t = now_fn()
            # device-side conditions (a bounded wait that gave up): the
            # condition word is per device, so a condition raised by the
            # other batch in flight fails this one as well
            status = device_status(self.streams[k], reset=True)
            for slot in b[1]:
                n = int(slot.host_count[0])
                slot.req.seeds = seeds_to_numpy(slot.host_seeds[:20 * min(n, slot.buf.capacity)].numpy(), n)
                slot.req.error = None if status == OK else _status_error(status)
                slot.req.t_done = t
                self.done.append(slot.req)
                slot.req = None
                self.free[(slot.buf.width, slot.buf.height)].append(slot)
            self.busy[k] = None

    def step(self, now_fn) -> None:
        with self._lock:
            self._retire(now_fn)
            self._admit()
            self._launch(now_fn)

    def idle(self) -> bool:
        return not self.pending and not self.admitted and all(b is None for b in self.busy)


class PlainServer:
    """Per-request reference: one request at a time in arrival order, matched
    alone (one stage, one CUDA stream, resident buffers per size)."""

    def __init__(self, params=None, tuning=None, device="cuda"):
        import torch
        self.params = params or default_params()
        self.tuning = tuning or default_tuning()
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(device=self.device)
        self.slots = {}
        self.pending = collections.deque()
        self.done = []
        self.cur = None
        self._lock = threading.Lock()
        self.batches = 0

    def submit(self, req: Request) -> None:
        _submit(req, self._lock, self.pending, self.done)

    def step(self, now_fn) -> None:
        import torch
        with self._lock:
            if self.cur is not None:
                ev, slot = self.cur
                if not ev.query():
                    return
                status = device_status(self.stream, reset=True)
                n = int(slot.host_count[0])
                slot.req.seeds = seeds_to_numpy(slot.host_seeds[:20 * min(n, slot.buf.capacity)].numpy(), n)
                slot.req.error = None if status == OK else _status_error(status)
                slot.req.t_done = now_fn()
                self.done.append(slot.req)
                self.cur = None
            if not self.pending:
                return
            req = self.pending.popleft()
            if req.size not in self.slots:
                self.slots[req.size] = _Slot(req.size[0], req.size[1], self.params, self.device)
            slot = self.slots[req.size]
            slot.req = req
            for k in range(4):
                slot.host_in[k].numpy()[...] = req.images[k]
            s = self.stream
            with torch.cuda.stream(s):
                slot.buf.dev_in.copy_(slot.host_in, non_blocking=True)
                run_batch([slot.buf.desc(None, req.seed)], self.params, self.tuning, s)
                slot.host_count.copy_(slot.buf.count, non_blocking=True)
                slot.host_seeds.copy_(slot.buf.seeds, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
            self.cur = (ev, slot)
            self.batches += 1

    def idle(self) -> bool:
        return not self.pending and self.cur is None


def _status_error(status: int) -> str:
    return f"device status: {lib().sff_status_string(status).decode()} ({status})"


def poisson_arrivals(rate: float, n: int, n_streams: int, pool_size: int, seed: int = 7):
    """n requests: exponential gaps at aggregate `rate` per second, each from
    one of n_streams camera streams, each using a quad of the pool."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return [(float(t[i]), int(rng.integers(0, n_streams)), int(rng.integers(0, pool_size))) for i in range(n)]


def simulate(server, arrivals, pool, seed_base: int = 1000, timeout: float = 600.0):
    """Replay arrivals in real time against `server`; returns the finished
    requests and the wall time from the first arrival to the last completion."""
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    reqs = [Request(i, sid, pool[pi], seed_base + pi, t_arrival=ta) for i, (ta, sid, pi) in enumerate(arrivals)]
    nxt = 0
    while True:
        t = now()
        while nxt < len(reqs) and reqs[nxt].t_arrival <= t:
            server.submit(reqs[nxt])
            nxt += 1
        server.step(now)
        if nxt == len(reqs) and server.idle():
            break
        if t > timeout:
            raise TimeoutError("serving simulation did not finish")
        if nxt < len(reqs) and server.idle():
            time.sleep(max(0.0, min(reqs[nxt].t_arrival - now(), 0.001)))
    return reqs, now()


def summarize(reqs, wall: float) -> dict:
    ok = [r for r in reqs if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1e3
    px = sum(r.size[0] * r.size[1] for r in ok)
    return {"requests": len(ok), "rejected": len(reqs) - len(ok), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "sustained_px_per_s": px / wall}
