"""CUDA-graph capture of the search paths.  With a caller workspace and
device outputs, rpf_query only enqueues kernels and a memset (no allocation,
no synchronisation), so a serving loop can replay one graph per batch shape;
the replays give the lists of an uncaptured call, for new query values too.
rpf_all_knn_async enqueues the all-kNN launches the same way."""
import numpy as np
import pytest

from paper_1812_11689_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,scan", [(0, None), (1, "bf16"), (1, "fp32")])
def test_query_graph_replays_match_uncaptured_calls(form, scan):
    import torch
    from paper_1812_11689_gb300 import forest
    torch.cuda.set_device(0)
    X = synth.make("aniso20_d64", n=20000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=6, leaf_max=128, n_try=5, form=form)
    if form == 1:
        f.set_query_scan(scan)
    m, K = 512, 10
    Qd = torch.from_numpy(synth.queries("aniso20_d64", m, stream=21)).cuda()
    idx = torch.empty((m, K), dtype=torch.int32, device="cuda")
    dist = torch.empty((m, K), dtype=torch.float32, device="cuda")
    ws = torch.empty(f.workspace_bytes(K, m=m, all_knn=False), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up outside the capture
        f.query(Qd, K, idx=idx, dist=dist, workspace=ws, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        f.query(Qd, K, idx=idx, dist=dist, workspace=ws, stream=s)
    for stream in (21, 22):
        Qn = torch.from_numpy(synth.queries("aniso20_d64", m, stream=stream)).cuda()
        ri, rd = f.query(Qn, K)
        Qd.copy_(Qn)
        idx.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(idx, ri) and torch.equal(dist, rd), stream
        f.query_status(ws)
    f.close()


@pytest.mark.parametrize("form", [0, 1])
def test_all_knn_graph_replays_match_the_synchronous_call(form):
    """rpf_all_knn_async only enqueues (persistent tile launch per group of
    trees, then the merge), so it records into a CUDA graph; every replay
    rewrites the lists of the synchronous call and reports its outcome in
    the workspace's first word."""
    import torch
    from paper_1812_11689_gb300 import forest
    torch.cuda.set_device(0)
    X = synth.make("aniso20_d64", n=20000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=6, leaf_max=128, n_try=5, form=form)
    K = 10
    ri, rd = f.all_knn(K)
    idx = torch.empty((f.n, K), dtype=torch.int32, device="cuda")
    dist = torch.empty((f.n, K), dtype=torch.float32, device="cuda")
    ws = torch.empty(f.workspace_bytes(K), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up outside the capture
        f.all_knn_async(K, idx, dist, ws, stream=s)
    f.query_status(ws, stream=s)
    assert torch.equal(idx, ri) and torch.equal(dist, rd)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        f.all_knn_async(K, idx, dist, ws, stream=s)
    for _ in range(2):
        idx.fill_(-7)
        dist.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(idx, ri) and torch.equal(dist, rd)
        f.query_status(ws)
    f.close()


def test_all_knn_async_checks_its_buffers_before_launching():
    import torch
    from paper_1812_11689_gb300 import forest
    torch.cuda.set_device(0)
    X = synth.make("aniso20_d64", n=3000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=2, leaf_max=64, n_try=3)
    K = 5
    ws = torch.empty(f.workspace_bytes(K), dtype=torch.uint8, device="cuda")
    idx = torch.full((f.n, K), -7, dtype=torch.int32, device="cuda")
    dist = torch.zeros((f.n, K), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        f.all_knn_async(K, idx[:10], dist, ws)            # wrong shape
    with pytest.raises(ValueError):
        f.all_knn_async(K, idx.cpu(), dist, ws)           # host output
    with pytest.raises(ValueError):
        f.all_knn_async(K, idx, dist, ws[:100])           # small workspace
    torch.cuda.synchronize()
    assert bool((idx == -7).all())  # nothing was launched
    f.close()
