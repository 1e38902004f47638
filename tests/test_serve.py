"""Serving loop: continuous batching over a resident forest.

GPU: every request's result is the same served alone (one rpf_query call)
and served in a mix (batched with other requests, several batches in flight
on different streams).  CPU: the scheduler's batch formation and its
admission by free device memory, with the device calls replaced by fakes.
"""
import numpy as np
import pytest

from paper_1812_11689_gb300 import synth


class _FakeForest:
    d = 8

    def workspace_bytes(self, K, m=0, all_knn=True):
        return 1000 * m * K


def _server(free_bytes, slots=2, max_batch=100, reserve=0):
    from paper_1812_11689_gb300 import serve
    s = serve.Server.__new__(serve.Server)
    s.forest = _FakeForest()
    s.slots = [serve._Slot(stream=None) for _ in range(slots)]
    s.max_batch, s.reserve = max_batch, reserve
    import collections
    s.waiting = collections.deque()
    s.finished, s.n_batches, s.max_inflight, s.deferred_for_memory = [], 0, 0, 0
    s.stalled = False
    s.deferred_now = False
    s.launched = []
    s._free_bytes = lambda: free_bytes

    def fake_launch(slot, batch, rows, K):
        slot.reqs, slot.rows, slot.K = batch, rows, K
        s.launched.append(([r.rid for r in batch], rows, K))
        s.n_batches += 1
    s._launch = fake_launch
    return s


def _req(rid, m, K):
    from paper_1812_11689_gb300 import serve
    return serve.Request(rid, np.zeros((m, 8), np.float32), K, 0.0)


def test_batches_take_same_k_requests_in_arrival_order_up_to_max_batch():
    s = _server(free_bytes=1 << 40, slots=2, max_batch=100)
    for rid, (m, K) in enumerate([(30, 10), (50, 50), (40, 10), (40, 10), (20, 50)]):
        s.submit(_req(rid, m, K))
    s._admit()
    # slot 0: K=10 requests 0 and 2 (70 rows; request 3 would exceed 100)
    # slot 1: the oldest waiting is now request 1 (K=50), joined by request 4
    assert s.launched == [([0, 2], 70, 10), ([1, 4], 70, 50)]
    assert [r.rid for r in s.waiting] == [3]


def test_admission_waits_for_free_device_memory():
    need = 1000 * 30 * 10 + 30 * 8 * 4 + 30 * 10 * 8
    s = _server(free_bytes=need - 1, slots=2)
    s.submit(_req(0, 30, 10))
    s._admit()
    assert s.launched == [] and s.deferred_for_memory == 1 and len(s.waiting) == 1
    assert s.stalled  # nothing in flight could free memory
    s._free_bytes = lambda: need
    s._admit()
    assert s.launched == [([0], 30, 10)] and not s.waiting


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch
    from paper_1812_11689_gb300 import forest, serve
    X = synth.make("mix50_d96", n=30000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=8, leaf_max=128, n_try=5, seed=4)
    sizes = synth.request_sizes(40, seed=3, max_size=600)
    reqs = [serve.Request(i, synth.queries("mix50_d96", int(m), stream=200 + i),
                          10 if i % 2 == 0 else 50, 0.0) for i, m in enumerate(sizes)]
    alone = []
    for r in reqs:
        i, d = f.query(torch.from_numpy(r.Q).cuda(), r.K)
        alone.append((i.cpu().numpy(), d.cpu().numpy()))
    srv = serve.Server(f, slots=3, max_batch=1500)
    arrivals = synth.poisson_arrivals(len(reqs), rate_per_s=4000.0, seed=5)
    out = srv.run(reqs, arrivals)
    assert len(out) == len(reqs)
    for r in reqs:
        ai, ad = alone[r.rid]
        assert np.array_equal(r.idx, ai) and np.array_equal(r.dist, ad), r.rid
        assert r.latency >= 0.0
    assert srv.n_batches < len(reqs)   # requests were batched together
    assert srv.max_inflight >= 2       # and batches overlapped on the device
    f.close()
