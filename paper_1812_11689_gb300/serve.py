"""Serving loop: a resident forest answering query sets as they arrive.

Requests (a set of m new points and K) wait in arrival order.  Whenever a
slot (one CUDA stream with its own buffers) is free, the scheduler forms a
batch from the oldest waiting request and the requests behind it with the
same K, up to ``max_batch`` points, and admits it if the device's free memory
(including what the torch caching allocator holds unused) covers the batch's
workspace, queries and outputs with ``reserve`` bytes to spare.  The batch
is copied to the device, answered by rpf_query (Sec. 2, Algorithm 3: route
through every tree, scan the leaves, merge) and copied back, all on the
slot's stream, so batches in different slots overlap on the device while
new requests keep arriving.  A request's latency runs from its arrival to
the moment the host sees its batch's results ready.

Every query is answered independently of the others in its batch (its own
routes, leaves and merge), so a result is the same whether the request is
served alone or in a mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .forest import Forest


@dataclass
class Request:
    rid: int
    Q: np.ndarray          # m x d float32
    K: int
    arrival: float         # seconds on the server clock
    idx: np.ndarray = None
    dist: np.ndarray = None
    done: float = None     # seconds on the server clock
    batch: int = -1

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    event: torch.cuda.Event = None
    reqs: list = field(default_factory=list)
    rows: int = 0
    K: int = 0
    host_q: torch.Tensor = None      # pinned staging, allocated once per slot
    host_idx: torch.Tensor = None
    host_dist: torch.Tensor = None
    keep: list = field(default_factory=list)   # device buffers alive until done
    seq: int = 0                                # launch order


class Server:
    """Continuous-batching query server over one resident forest."""

    def __init__(self, forest: Forest, slots: int = 4, max_batch: int = 8192,
                 reserve: int = 256 << 20, device=None):
        self.forest = forest
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.slots = [_Slot(torch.cuda.Stream(device=self.device)) for _ in range(slots)]
        self.max_batch = int(max_batch)
        self.reserve = int(reserve)
        self.waiting = collections.deque()
        self.finished = []
        self.n_batches = 0
        self.max_inflight = 0
        self.deferred_for_memory = 0
        self.stalled = False  # the oldest batch does not fit even with nothing in flight
        self.deferred_now = False  # the last admission was held back for memory
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ---- admission --------------------------------------------------------------
    def submit(self, req: Request) -> None:
        self.waiting.append(req)

    def _free_bytes(self) -> int:
        free, _ = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return int(free + cached)

    def _need_bytes(self, rows: int, K: int) -> int:
        return (self.forest.workspace_bytes(K, m=rows, all_knn=False)
                + rows * self.forest.d * 4 + rows * K * 8)

    def _form_batch(self):
        head = self.waiting[0]
        batch, rows = [], 0
        for r in self.waiting:
            if r.K != head.K:
                continue
            m = r.Q.shape[0]
            if batch and rows + m > self.max_batch:
                break
            batch.append(r)
            rows += m
        return batch, rows, head.K

    def _pinned(self, slot: _Slot, rows: int, K: int) -> None:
        """Pinned host staging of the slot, grown (rarely) to the batch's size:
        page-locking memory is slow, so it is not done per batch."""
        d = self.forest.d
        if slot.host_q is None or slot.host_q.shape[0] < rows:
            cap = max(rows, self.max_batch)
            slot.host_q = torch.empty((cap, d), dtype=torch.float32).pin_memory()
        if slot.host_idx is None or slot.host_idx.numel() < rows * K:
            cap = max(rows * K, self.max_batch * K)
            slot.host_idx = torch.empty(cap, dtype=torch.int32).pin_memory()
            slot.host_dist = torch.empty(cap, dtype=torch.float32).pin_memory()

    def _launch(self, slot: _Slot, batch, rows: int, K: int) -> None:
        d = self.forest.d
        self._pinned(slot, rows, K)
        Qh = slot.host_q[:rows]
        o = 0
        for r in batch:
            m = r.Q.shape[0]
            Qh[o:o + m].numpy()[...] = r.Q
            o += m
        hidx = slot.host_idx[:rows * K].view(rows, K)
        hdist = slot.host_dist[:rows * K].view(rows, K)
        with torch.cuda.stream(slot.stream):
            Qd = torch.empty((rows, d), dtype=torch.float32, device=self.device)
            idx = torch.empty((rows, K), dtype=torch.int32, device=self.device)
            dist = torch.empty((rows, K), dtype=torch.float32, device=self.device)
            ws = torch.empty(self.forest.workspace_bytes(K, m=rows, all_knn=False),
                             dtype=torch.uint8, device=self.device)
            Qd.copy_(Qh, non_blocking=True)
            self.forest.query(Qd, K, idx=idx, dist=dist, workspace=ws, stream=slot.stream)
            hidx.copy_(idx, non_blocking=True)
            hdist.copy_(dist, non_blocking=True)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.keep = [Qd, idx, dist, ws, hidx, hdist]
        slot.reqs, slot.rows, slot.K = batch, rows, K
        slot.seq = self.n_batches
        for r in batch:
            r.batch = self.n_batches
        self.n_batches += 1
        self.max_inflight = max(self.max_inflight, sum(1 for x in self.slots if x.reqs))

    def _admit(self) -> None:
        for slot in self.slots:
            if not self.waiting:
                return
            if slot.reqs:
                continue
            batch, rows, K = self._form_batch()
            if self._free_bytes() - self._need_bytes(rows, K) < self.reserve:
                self.deferred_for_memory += 1
                self.deferred_now = True
                self.stalled = not any(x.reqs for x in self.slots)
                return
            self.stalled = False
            for r in batch:
                self.waiting.remove(r)
            self._launch(slot, batch, rows, K)

    def _retire(self) -> None:
        for slot in self.slots:
            if not slot.reqs or not slot.event.query():
                continue
            # the batch's device work is done: a bounded wait of it that gave
            # up would be reported here (raises), never silently served
            self.forest.query_status(slot.keep[3], stream=slot.stream)
            t = self.now()
            hidx, hdist = slot.keep[4], slot.keep[5]
            o = 0
            for r in slot.reqs:
                m = r.Q.shape[0]
                r.idx = hidx[o:o + m].numpy().copy()
                r.dist = hdist[o:o + m].numpy().copy()
                r.done = t
                o += m
                self.finished.append(r)
            slot.reqs, slot.keep = [], []

    def step(self) -> None:
        self.deferred_now = False
        self._retire()
        self._admit()

    def busy(self) -> bool:
        return bool(self.waiting) or any(s.reqs for s in self.slots)

    # ---- drivers ----------------------------------------------------------------
    def run(self, requests, arrivals=None):
        """Serve `requests`; arrivals[i] (seconds from start) is when request i
        arrives (None: all at once).  Returns the finished requests."""
        order = list(range(len(requests)))
        if arrivals is not None:
            order.sort(key=lambda i: arrivals[i])
        self.t0 = time.perf_counter()
        k = 0
        while k < len(order) or self.busy():
            t = self.now()
            while k < len(order) and (arrivals is None or arrivals[order[k]] <= t):
                r = requests[order[k]]
                r.arrival = t if arrivals is None else float(arrivals[order[k]])
                self.submit(r)
                k += 1
            self.step()
            if self.stalled:
                raise RuntimeError("a batch needs more free device memory than the device has "
                                   "with nothing in flight; lower max_batch or reserve")
            nxt = (float(arrivals[order[k]]) - self.now()
                   if k < len(order) and arrivals is not None else None)
            self._idle(nxt)
        return self.finished

    def _idle(self, nxt) -> None:
        """Block until something can change instead of polling: with every
        slot busy, or requests held back for memory, wait on the oldest batch's
        event; with a free slot and nothing waiting, sleep until the next
        arrival (in steps of at most 100 us while batches are in flight)."""
        inflight = [s for s in self.slots if s.reqs]
        if not inflight:
            if nxt is not None and nxt > 0:
                time.sleep(nxt)
            return
        if self.waiting and (len(inflight) < len(self.slots)) and not self.deferred_now:
            return  # admissible work is waiting: step again at once
        if len(inflight) == len(self.slots) or self.waiting or nxt is None:
            min(inflight, key=lambda s: s.seq).event.synchronize()
        elif nxt > 0:
            time.sleep(min(nxt, 1e-4))


def latency_summary(reqs) -> dict:
    lat = np.array([r.latency for r in reqs], np.float64) * 1e3
    rows = sum(r.Q.shape[0] for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "queries": int(rows),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "queries_per_s": round(rows / span, 1) if span > 0 else None}
