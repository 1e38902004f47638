"""Failure detection without a GPU fault.

CPU: the checks of caller buffers run before anything is launched; the
allocation-failure hook is exported and turns an allocation into RPF_ENOMEM.
GPU: a bounded device wait on a barrier that nothing completes gives up with
RPF_ETIMEOUT and the context stays usable; an injected allocation failure at
every allocation of a build, an all-kNN and a query returns RPF_ENOMEM and
the next call succeeds with the oracle's answer.
"""
import ctypes

import numpy as np
import pytest

from paper_1812_11689_gb300 import synth

RPF_ENOMEM, RPF_ETIMEOUT = -2, -4


def test_query_static_arguments_are_checked_before_any_launch():
    torch = pytest.importorskip("torch")
    from paper_1812_11689_gb300 import forest
    dev = torch.device("cpu")
    Q = torch.zeros((7, 10), dtype=torch.float32)
    good_i = torch.zeros((7, 5), dtype=torch.int32)
    good_d = torch.zeros((7, 5), dtype=torch.float32)
    bad = [
        (torch.zeros((7, 9), dtype=torch.float32), good_i, good_d),    # Q columns != d
        (Q.double(), good_i, good_d),                                    # Q dtype
        (Q, torch.zeros((6, 5), dtype=torch.int32), good_d),             # idx rows
        (Q, torch.zeros((7, 4), dtype=torch.int32), good_d),             # idx columns
        (Q, good_i.long(), good_d),                                      # idx dtype
        (Q, good_i, torch.zeros((7, 5), dtype=torch.float64)),           # dist dtype
        (Q, torch.zeros((5, 7), dtype=torch.int32).t(), good_d),         # not contiguous
        (Q, good_i, torch.zeros((7, 6), dtype=torch.float32)),           # dist shape
    ]
    for q, i, d in bad:
        with pytest.raises(ValueError):
            forest._check_query_static(10, q, 5, i, d, dev)
    # right shapes and dtypes, but host tensors for a forest on a CUDA device
    with pytest.raises(ValueError):
        forest._check_query_static(10, Q, 5, good_i, good_d, torch.device("cuda", 0))
    assert forest._check_query_static(10, Q, 5, good_i, good_d, None) == 7  # shapes only


def test_query_outputs_are_checked():
    from paper_1812_11689_gb300 import forest
    forest._check_out("idx", np.zeros((3, 4), np.int32), (3, 4), np.int32)
    for a in (np.zeros((3, 5), np.int32), np.zeros((3, 4), np.int64),
              np.zeros((4, 3), np.int32).T):
        with pytest.raises(ValueError):
            forest._check_out("idx", a, (3, 4), np.int32)


def test_alloc_failure_hook_is_exported_and_returns_enomem():
    from paper_1812_11689_gb300 import _lib, build
    build.build()
    L = _lib.lib()
    p = _lib.rpf_params(2, 50, 5, 0, 0, 0, 0)
    buf = (ctypes.c_float * 20)()
    out = ctypes.c_void_p()
    L.rpf_debug_fail_alloc(0)
    assert L.rpf_build(buf, 10, 2, ctypes.byref(p), None, ctypes.byref(out)) == RPF_ENOMEM
    assert not out.value
    L.rpf_debug_fail_alloc(-1)


# ---------------------------------------------------------------------------
@pytest.mark.gpu
def test_bounded_wait_gives_up_and_the_context_stays_usable():
    import torch
    import oracle
    from paper_1812_11689_gb300 import forest
    torch.cuda.set_device(0)
    for limit in (1_000_000, 50_000_000):  # 1 ms, 50 ms
        assert forest.wait_selftest(limit) == RPF_ETIMEOUT
    X = synth.make("mix5_d10", n=2000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=4, leaf_max=50, n_try=5,
                      form=forest.FORM_CHOSEN)
    i, d = f.all_knn(5)
    o = oracle.Forest(X, 4, 50, 5)
    oi, od = o.all_knn(5)
    assert np.array_equal(i.cpu().numpy(), oi) and np.array_equal(d.cpu().numpy(), od)
    f.close()


@pytest.mark.gpu
def test_every_allocation_failure_returns_enomem_then_service_resumes():
    import torch
    import oracle
    from paper_1812_11689_gb300 import forest
    from paper_1812_11689_gb300._lib import RpfError
    torch.cuda.set_device(0)
    X = synth.make("aniso20_d64", n=9000)
    Xd = torch.from_numpy(X).cuda()
    kw = dict(n_trees=3, leaf_max=128, n_try=5, form=forest.FORM_CHOSEN)
    failures = 0
    for k in range(400):
        forest.debug_fail_alloc(k)
        try:
            f = forest.Forest(Xd, **kw)
        except RpfError as e:
            assert e.code == RPF_ENOMEM, (k, e.code)
            failures += 1
            continue
        forest.debug_fail_alloc(-1)
        f.close()
        break
    else:
        pytest.fail("more than 400 allocations in one build")
    assert failures >= 10  # every table and scratch buffer of the build was hit
    torch.cuda.synchronize()
    f = forest.Forest(Xd, **kw)
    for k in range(3):  # the all-kNN workspace and the host-output staging
        forest.debug_fail_alloc(k)
        try:
            f.all_knn(10, idx=np.empty((9000, 10), np.int32), dist=np.empty((9000, 10), np.float32))
        except RpfError as e:
            assert e.code == RPF_ENOMEM
    forest.debug_fail_alloc(0)
    with pytest.raises(RpfError) as ei:
        f.query(Xd[:100], 10)
    assert ei.value.code == RPF_ENOMEM
    forest.debug_fail_alloc(-1)
    gi, gd = f.all_knn(10)
    o = oracle.Forest(X, 3, 128, 5)
    rows = np.arange(0, 9000, 7, dtype=np.int32)
    oi, od = o.all_knn_rows(rows, 10)
    assert np.array_equal(gi.cpu().numpy()[rows], oi)
    assert np.array_equal(gd.cpu().numpy()[rows], od)
    qi, qd = f.query(Xd[:100], 10)
    ri, rd = o.query(X[:100], 10)
    assert np.array_equal(qi.cpu().numpy(), ri) and np.array_equal(qd.cpu().numpy(), rd)
    f.close()


@pytest.mark.gpu
def test_query_status_reports_a_clean_asynchronous_query():
    import torch
    from paper_1812_11689_gb300 import forest
    torch.cuda.set_device(0)
    X = synth.make("mix5_d10", n=2000)
    f = forest.Forest(torch.from_numpy(X).cuda(), n_trees=4, leaf_max=50, n_try=5)
    Q = torch.from_numpy(X[:64]).cuda()
    ws = torch.empty(f.workspace_bytes(5, m=64, all_knn=False), dtype=torch.uint8, device="cuda")
    idx = torch.empty((64, 5), dtype=torch.int32, device="cuda")
    dist = torch.empty((64, 5), dtype=torch.float32, device="cuda")
    f.query(Q, 5, idx=idx, dist=dist, workspace=ws)
    f.query_status(ws)
    ri, rd = f.query(X[:64], 5)  # host buffers: synchronous, status checked inside
    assert np.array_equal(idx.cpu().numpy(), ri) and np.array_equal(dist.cpu().numpy(), rd)
    with pytest.raises(ValueError):
        f.query_static(Q, 5, idx[:, :4].contiguous(), dist)
    with pytest.raises(ValueError):
        f.query(Q, 5, idx=idx[:10], dist=dist)
    f.close()
