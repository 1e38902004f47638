"""The query path is capturable in a CUDA graph: with a caller workspace and
device outputs, rpf_query only enqueues kernels and a memset (no allocation,
no synchronisation), so a serving loop can replay one graph per batch shape.
The replays give the lists of an uncaptured call, for new query values too."""
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
