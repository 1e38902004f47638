"""rpf_query_static: the query path with the library's fixed device scratch.

Kept in its own file, collected last, so that it runs both alone and after
every other GPU test.  The expected values come from the existing rpf_query
entry point on the same forest and queries.
"""
import numpy as np
import pytest

from paper_1812_11689_gb300 import synth

pytestmark = pytest.mark.gpu


def _forest():
    import torch
    from paper_1812_11689_gb300 import forest
    X = synth.make("mix50_d96", n=20000)
    return forest.Forest(torch.from_numpy(X).cuda(), n_trees=8, leaf_max=128, n_try=5, seed=2)


def test_query_static_equals_query_on_two_calls_in_a_row_and_allocates_nothing():
    import torch
    f = _forest()
    m, K = 1500, 10
    Qd = torch.from_numpy(synth.queries("mix50_d96", m, stream=9)).cuda()
    ri, rd = f.query(Qd, K)
    idx = torch.empty((m, K), dtype=torch.int32, device="cuda")
    dist = torch.empty((m, K), dtype=torch.float32, device="cuda")
    for call in range(2):
        idx.fill_(-7)
        dist.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        f.query_static(Qd, K, idx, dist)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert torch.equal(idx, ri) and torch.equal(dist, rd), call
        if call == 1:  # the first call may load the module holding the scratch
            assert free1 == free0
    f.close()


def test_query_static_rejects_oversized_and_host_requests():
    import torch
    f = _forest()
    K = 10
    # need = 256 + align256(8 m T) + align256(8 T m K) > 8 MiB at T = 8, K = 10
    m = 13000
    Qd = torch.zeros((m, 96), dtype=torch.float32, device="cuda")
    idx = torch.full((m, K), -7, dtype=torch.int32, device="cuda")
    dist = torch.zeros((m, K), dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        f.query_static(Qd, K, idx, dist)
    torch.cuda.synchronize()
    assert bool((idx == -7).all())  # nothing was launched
    # host queries are refused before anything is launched
    Qh = torch.zeros((10, 96), dtype=torch.float32)
    with pytest.raises(ValueError):
        f.query_static(Qh, K, idx[:10], dist[:10])
    torch.cuda.synchronize()
    assert bool((idx == -7).all())
    # the status of the last allocation-free query on this device
    f.query_static(Qd[:100], K, idx[:100], dist[:100])
    f.query_status(None)
    f.close()
