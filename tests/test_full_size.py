"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark times (chosen leaf form, certified FP32 growth with FP64 fallback).

The oracle grows its trees with one tree per host core.  Because every draw
is keyed by the tree index, the first T' trees of a GPU forest are exactly
the oracle's T'-tree forest, so the large forests are checked on their first
trees where the oracle would take minutes for all of them:

* anisotropic mixture, 200,000 x 64, leaf bound 128: all 96 trees (the
  benchmark's operating point) and every all-kNN list at T = 96 and T = 40;
* heavy-tailed, 500,000 x 32, leaf bound 64: the 128-tree forest's first 32
  trees (more than 90 level-synchronous levels) and all-kNN over them on a
  20,000-point sample;
* points near a 16-dimensional subspace, 1,000,000 x 128, leaf bound 256:
  the 64-tree forest's first 8 trees and all-kNN over them on a sample;
* the 2,000,000 x 96 mixture behind the serving workload: an 8-tree forest
  and 2,000 new queries at K = 10 and 50.
"""
import numpy as np
import pytest

import oracle
from paper_1812_11689_gb300 import synth
from _parity import check_knn, compare_trees

pytestmark = pytest.mark.gpu


def _gpu(X, T, L, ntry=5, seed=0):
    import torch
    from paper_1812_11689_gb300 import build, forest
    build.build()
    return forest.Forest(torch.from_numpy(X).cuda(), n_trees=T, leaf_max=L, n_try=ntry,
                         seed=seed, form=forest.FORM_CHOSEN)


def _sample(n, size, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size, replace=False)).astype(np.int32)


def test_anisotropic_200k_every_tree_and_every_list():
    w = synth.WORKLOADS["aniso20_d64"]
    X = synth.make("aniso20_d64")
    T = 96
    g = _gpu(X, T, w.leaf_max)
    o = oracle.Forest(X, T, w.leaf_max, w.n_try)
    compare_trees(g, o, T)
    gi, gd = g.all_knn(w.k)
    oi, od = o.all_knn(w.k)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)
    del o
    # the configured T = 40: the first 40 trees of the same forest
    o40 = oracle.Forest(X, w.n_trees, w.leaf_max, w.n_try)
    gi, gd = g.all_knn(w.k, n_trees=w.n_trees)
    oi, od = o40.all_knn(w.k)
    assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    assert g.counters()["bf16_fallback_rows"] >= 0
    g.close()


def test_heavy_tailed_500k_deep_level_synchronous_phase():
    w = synth.WORKLOADS["student3_d32"]
    X = synth.make("student3_d32")
    g = _gpu(X, w.n_trees, w.leaf_max)
    Tc = 32
    o = oracle.Forest(X, Tc, w.leaf_max, w.n_try)
    compare_trees(g, o, Tc)
    assert g.counters()["phase_a_levels"] > 90
    rows = _sample(w.n, 20000, 1)
    gi, gd = g.all_knn(w.k, n_trees=Tc)
    oi, od = o.all_knn_rows(rows, w.k)
    check_knn(gi.cpu().numpy()[rows], gd.cpu().numpy()[rows], oi, od, X, rows)
    g.close()


def test_subspace_1m_d128_first_trees_and_sampled_lists():
    w = synth.WORKLOADS["subspace16_d128"]
    X = synth.make("subspace16_d128")
    g = _gpu(X, w.n_trees, w.leaf_max)
    Tc = 8
    o = oracle.Forest(X, Tc, w.leaf_max, w.n_try)
    compare_trees(g, o, Tc)
    rows = _sample(w.n, 20000, 2)
    gi, gd = g.all_knn(w.k, n_trees=Tc)
    oi, od = o.all_knn_rows(rows, w.k)
    check_knn(gi.cpu().numpy()[rows], gd.cpu().numpy()[rows], oi, od, X, rows)
    g.close()


def test_mixture_2m_d96_trees_and_queries():
    import torch
    w = synth.WORKLOADS["mix50_d96"]
    X = synth.make("mix50_d96")
    T = 8
    g = _gpu(X, T, w.leaf_max)
    o = oracle.Forest(X, T, w.leaf_max, w.n_try)
    compare_trees(g, o, T)
    Q = synth.queries("mix50_d96", 2000, stream=77)
    for K in w.extra["k_set"]:
        qi, qd = g.query(torch.from_numpy(Q).cuda(), K)
        ri, rd = o.query(Q, K)
        assert np.array_equal(qi.cpu().numpy(), ri) and np.array_equal(qd.cpu().numpy(), rd), K
    g.close()
