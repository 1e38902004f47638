"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact: candidate directions, every tree's permutation and leaf table, the
split records (chosen try, split point, rank-split flag) keyed by node key,
and the neighbour indices; distances bit-exact against the oracle's FP32 key
and within 1e-5 relative of FP64 (the tolerance the method's FP32 distance
key guarantees: (d + 3) 2^-24 < 1e-5 for d <= 128).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1812_11689_gb300 import synth
from _parity import REL_TOL_FP64, check_knn, compare_trees  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1812_11689_gb300 import build
    build.build()


def F(*a, **k):
    from paper_1812_11689_gb300 import forest
    return forest.Forest(*a, **k)


def gpu_forest(X, T, L, ntry, seed=0, growth=0, form=0):
    return F(torch.from_numpy(np.ascontiguousarray(X)).cuda(), n_trees=T, leaf_max=L,
             n_try=ntry, seed=seed, growth=growth, form=form)


@pytest.mark.parametrize("d", [1, 2, 10, 64, 127])
def test_directions_bit_exact(d):
    from paper_1812_11689_gb300 import forest
    rng = np.random.default_rng(d)
    keys = np.concatenate([[1], rng.integers(0, 2 ** 63, 300, dtype=np.int64).astype(np.uint64)])
    for t, j in ((0, 0), (7, 3)):
        g = forest.directions(11, t, keys, j, d)
        o = np.stack([oracle.direction(11, t, int(k), j, d) for k in keys])
        assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


@pytest.mark.parametrize("growth", [1, 2])
def test_trees_bit_exact_mix5(growth):
    X = synth.make("mix5_d10")
    g = gpu_forest(X, 10, 50, 5, growth=growth)
    o = oracle.Forest(X, 10, 50, 5, seed=0)
    compare_trees(g, o, 10)


@pytest.mark.parametrize("name,n,L,ntry", [("aniso20_d64", 20000, 128, 5),
                                           ("student3_d32", 20000, 64, 5),
                                           ("subspace16_d128", 8000, 256, 3),
                                           ("mix50_d96", 9000, 128, 1),
                                           ("student3_d32", 6000, 64, 10),
                                           ("aniso20_d64", 6000, 128, 20)])
def test_trees_bit_exact_workload_shapes(name, n, L, ntry):
    X = synth.make(name, n=n)
    o = oracle.Forest(X, 4, L, ntry, seed=5)
    for growth in (1, 2):
        g = gpu_forest(X, 4, L, ntry, seed=5, growth=growth)
        compare_trees(g, o, 4)


def test_trees_bit_exact_level_synchronous_odd_dimension():
    # d = 10 (not a multiple of 4): the level-synchronous projections take
    # the per-thread path instead of the staged row tiles
    X = synth.make("mix5_d10", n=12000)
    o = oracle.Forest(X, 3, 50, 5, seed=3)
    for growth in (1, 2):
        compare_trees(gpu_forest(X, 3, 50, 5, seed=3, growth=growth), o, 3)


def test_growth_modes_agree_and_certification_skips_fp64():
    X = synth.make("aniso20_d64", n=30000)
    a = gpu_forest(X, 6, 128, 5, growth=1)
    b = gpu_forest(X, 6, 128, 5, growth=2)
    for t in range(6):
        assert np.array_equal(a.perm(t), b.perm(t))
    ia, ib = a.info(), b.info()
    assert ia["n_nodes"] == ib["n_nodes"]
    # FP64 fallback only for a minority of nodes under certification, but
    # some (their tries in contention recomputed in FP64) -- and every split
    # record equal to the all-FP64 growth's
    assert 0 < ib["n_exact_nodes"] < 0.25 * (ib["n_nodes"] - ib["n_leaves"])
    assert ia["n_exact_nodes"] == ia["n_nodes"] - ia["n_leaves"]
    na, nb = a.nodes(), b.nodes()
    ka = np.lexsort((na["key"], na["tree"]))
    kb = np.lexsort((nb["key"], nb["tree"]))
    for f in ("tree", "key", "left", "jstar"):
        assert np.array_equal(na[f][ka] >= 0 if f == "left" else na[f][ka],
                              nb[f][kb] >= 0 if f == "left" else nb[f][kb]), f
    assert np.array_equal(na["flag"][ka] & 1, nb["flag"][kb] & 1)
    assert np.array_equal(na["c"][ka].view(np.uint64), nb["c"][kb].view(np.uint64))


@pytest.mark.parametrize("form", [0, 1])
def test_all_knn_bit_exact_mix5(form):
    X = synth.make("mix5_d10")
    g = gpu_forest(X, 10, 50, 5, form=form)
    gi, gd = g.all_knn(5)
    o = oracle.Forest(X, 10, 50, 5, seed=0)
    oi, od = o.all_knn(5)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)


@pytest.mark.parametrize("form", [0, 1])
def test_all_knn_bit_exact_aniso_subsample(form):
    X = synth.make("aniso20_d64", n=20000)
    g = gpu_forest(X, 8, 128, 5, form=form)
    gi, gd = g.all_knn(10)
    o = oracle.Forest(X, 8, 128, 5, seed=0)
    oi, od = o.all_knn(10)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)


@pytest.mark.parametrize("K", [1, 7, 16, 20, 33, 128])
def test_all_knn_k_range_and_grouped_workspace(K):
    X = synth.make("subspace16_d128", n=3000)
    g = gpu_forest(X, 5, 200, 3)
    o = oracle.Forest(X, 5, 200, 3, seed=0)
    oi, od = o.all_knn(K)
    gi, gd = g.all_knn(K)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)
    # a workspace with room for two trees at a time gives the same lists
    ws_b = (2 * 3000 * K * 8 + 255) // 256 * 256 + (3000 * K * 8 + 255) // 256 * 256
    ws = torch.empty(ws_b, dtype=torch.uint8, device="cuda")
    hi, hd = g.all_knn(K, workspace=ws)
    assert torch.equal(hi, gi) and torch.equal(hd, gd)


def test_host_buffers_match_device_buffers():
    X = synth.make("mix5_d10", n=1500)
    g = F(X, n_trees=6, leaf_max=40, n_try=3, seed=2)  # host input
    hi = np.empty((1500, 6), np.int32)
    hd = np.empty((1500, 6), np.float32)
    g.all_knn(6, idx=hi, dist=hd)
    di, dd = g.all_knn(6)
    assert np.array_equal(hi, di.cpu().numpy()) and np.array_equal(hd, dd.cpu().numpy())
    o = oracle.Forest(X, 6, 40, 3, seed=2)
    oi, od = o.all_knn(6)
    assert np.array_equal(hi, oi)


def test_query_matches_oracle_and_routes_build_points():
    X = synth.make("aniso20_d64", n=12000)
    Q = synth.queries("aniso20_d64", 700)
    g = gpu_forest(X, 6, 128, 5)
    o = oracle.Forest(X, 6, 128, 5, seed=0)
    for K in (1, 10, 50):
        qi, qd = g.query(torch.from_numpy(Q).cuda(), K)
        oi, od = o.query(Q, K)
        assert np.array_equal(qi.cpu().numpy(), oi) and np.array_equal(qd.cpu().numpy(), od)
    # host queries, host outputs
    hi, hd = g.query(Q[:100], 10)
    oi, od = o.query(Q[:100], 10)
    assert np.array_equal(hi, oi) and np.array_equal(hd, od)
    # a data point routed through the forest lands in its own leaves: its
    # query answer is its all-kNN answer with itself at distance 0 in front
    ai, ad = g.all_knn(9)
    qi, qd = g.query(torch.from_numpy(X[:500]).cuda(), 10)
    qi, qd, ai = qi.cpu().numpy(), qd.cpu().numpy(), ai.cpu().numpy()
    dup = {tuple(r) for r in X[:500]}
    for i in range(500):
        if qd[i, 1] == 0.0:  # an exact duplicate of point i exists; order by index
            continue
        assert qi[i, 0] == i and qd[i, 0] == 0.0
        assert np.array_equal(qi[i, 1:], ai[i])
    assert len(dup) > 0
    # empty query set
    ei, ed = g.query(torch.empty((0, 64), device="cuda"), 5)
    assert ei.shape == (0, 5)


def test_single_leaf_forest_is_exact_knn():
    X = synth.make("mix5_d10", n=700)
    g = gpu_forest(X, 2, 700, 5)
    gi, gd = g.all_knn(7)
    bi, bd, _ = oracle.brute_knn(X, 7)
    assert np.array_equal(gi.cpu().numpy(), bi) and np.array_equal(gd.cpu().numpy(), bd)


def test_degenerate_inputs():
    # all points identical: every split is a rank split
    X = np.ones((600, 5), np.float32)
    for growth in (1, 2):
        g = gpu_forest(X, 3, 16, 3, growth=growth)
        o = oracle.Forest(X, 3, 16, 3, seed=0)
        compare_trees(g, o, 3)
        gi, gd = g.all_knn(3)
        oi, od = o.all_knn(3)
        assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    # duplicates and a constant column
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3000, 6)).astype(np.float32)
    X[:, 2] = 7.0
    X[100:400] = X[0]
    g = gpu_forest(X, 4, 20, 4)
    o = oracle.Forest(X, 4, 20, 4, seed=0)
    compare_trees(g, o, 4)
    gi, gd = g.all_knn(5)
    oi, od = o.all_knn(5)
    assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    # d = 1
    X = rng.standard_normal((5000, 1)).astype(np.float32)
    g = gpu_forest(X, 3, 30, 2)
    o = oracle.Forest(X, 3, 30, 2, seed=0)
    compare_trees(g, o, 3)


@pytest.mark.parametrize("n,K", [(1, 1), (2, 3), (5, 8)])
def test_tiny_inputs_pad(n, K):
    X = synth.make("mix5_d10", n=max(n, 1))[:n]
    g = gpu_forest(X, 3, 1, 2)
    gi, gd = g.all_knn(K)
    o = oracle.Forest(X, 3, 1, 2, seed=0)
    oi, od = o.all_knn(K)
    assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    assert np.all(gi.cpu().numpy()[:, n - 1:] == -1)


def test_ragged_large_node_multi_chunk():
    # one tree whose root spans many 4096-position chunks with a ragged tail
    X = synth.make("student3_d32", n=4096 * 5 + 77)
    o = oracle.Forest(X, 2, 1000, 7, seed=3)
    for growth in (1, 2):
        g = gpu_forest(X, 2, 1000, 7, seed=3, growth=growth)
        compare_trees(g, o, 2)


def test_brute_knn_matches_oracle_brute_force():
    from paper_1812_11689_gb300 import forest
    X = synth.make("aniso20_d64", n=6000)
    rows = np.arange(0, 6000, 7, dtype=np.int32)
    gi, gd = forest.brute_knn(torch.from_numpy(X).cuda(), torch.from_numpy(X[rows]).cuda(), 10,
                              self_idx=torch.from_numpy(rows).cuda())
    oi, od, _ = oracle.brute_knn(X, 10, rows=rows)
    assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    Q = synth.queries("aniso20_d64", 50)
    hi, hd = forest.brute_knn(X, Q, 3)  # host buffers, no exclusion
    oi, od, _ = oracle.brute_knn(X, 3, Q=Q)
    assert np.array_equal(hi, oi) and np.array_equal(hd, od)


def test_trace_counts_and_times_launches():
    from paper_1812_11689_gb300 import forest
    X = synth.make("mix5_d10", n=3000)
    forest.Trace.read()
    forest.Trace.enable(True)
    l0 = forest.Trace.launch_count()
    f = gpu_forest(X, 4, 50, 3)
    f.all_knn(5)
    l1 = forest.Trace.launch_count()
    forest.Trace.enable(False)
    tr = forest.Trace.read()
    assert l1 - l0 == sum(v["launches"] for v in tr.values())
    assert tr["k_leaf_plain"]["launches"] >= 1 and tr["k_merge"]["launches"] >= 1
    assert all(v["ms"] >= 0.0 for v in tr.values())


@pytest.mark.parametrize("K", [1, 7, 10, 16, 20])
def test_chosen_form_equals_plain_and_oracle(K):
    X = synth.make("aniso20_d64", n=12000)
    o = oracle.Forest(X, 4, 128, 5, seed=3)
    oi, od = o.all_knn(K)
    p = gpu_forest(X, 4, 128, 5, seed=3, form=0)
    c = gpu_forest(X, 4, 128, 5, seed=3, form=1)
    pi, pd = p.all_knn(K)
    ci, cd = c.all_knn(K)
    assert torch.equal(pi, ci) and torch.equal(pd, cd)
    check_knn(ci.cpu().numpy(), cd.cpu().numpy(), oi, od, X)


@pytest.mark.parametrize("shape", ["simplex_d256", "cross_polytope_d64"])
def test_chosen_form_certificate_fallback_is_exact(shape):
    # near-equidistant points: all pairwise squared distances agree to ~1e-6
    # relative, below what the split-BF16 Gram resolves, so the certificate
    # fails and rows are rescanned exactly -- the lists must still equal the
    # oracle's.  d = 256 runs the Gram in two 128-coordinate chunks.
    rng = np.random.default_rng(0)
    if shape == "simplex_d256":
        n = d = 256
        X = 10.0 * np.eye(n, d)
        T, L, ntry = 3, 64, 3
    else:
        d = 64
        X = np.concatenate([10.0 * np.eye(d), -10.0 * np.eye(d)])
        T, L, ntry = 3, 128, 3
    X = (X + 1e-5 * rng.standard_normal(X.shape)).astype(np.float32)
    o = oracle.Forest(X, T, L, ntry, seed=1)
    oi, od = o.all_knn(10)
    c = gpu_forest(X, T, L, ntry, seed=1, form=1)
    ci, cd = c.all_knn(10)
    assert np.array_equal(ci.cpu().numpy(), oi) and np.array_equal(cd.cpu().numpy(), od)
    assert c.counters()["bf16_fallback_rows"] > 0


def test_chosen_form_margin_wider_than_the_kept_keys():
    # groups of 16 near-equidistant points (regular simplices, edge ~1.4, far
    # apart): a row's 15 group-mates all lie within the certified margin, more
    # than the K + 2 keys the selection keeps, so the row collects its margin
    # columns in a second pass; the lists must equal the oracle's
    rng = np.random.default_rng(4)
    d, g, ng = 64, 16, 150
    centres = 50.0 * rng.standard_normal((ng, d))
    X = np.concatenate([c + np.eye(g, d) for c in centres])
    X = (X + 1e-6 * rng.standard_normal(X.shape)).astype(np.float32)
    o = oracle.Forest(X, 3, 100, 5, seed=2)
    oi, od = o.all_knn(10)
    c = gpu_forest(X, 3, 100, 5, seed=2, form=1)
    ci, cd = c.all_knn(10)
    assert np.array_equal(ci.cpu().numpy(), oi) and np.array_equal(cd.cpu().numpy(), od)


@pytest.mark.parametrize("form", [0, 1])
def test_all_knn_over_tree_prefixes_equals_the_smaller_forests(form):
    # nested ensembles: the first T' trees of a forest are the T'-tree forest
    X = synth.make("student3_d32", n=15000)
    g = gpu_forest(X, 8, 64, 5, seed=6, form=form)
    for Tp in (1, 3, 8):
        gi, gd = g.all_knn(10, n_trees=Tp)
        oi, od = oracle.Forest(X, Tp, 64, 5, seed=6).all_knn(10)
        check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)
    with pytest.raises(RuntimeError):
        g.all_knn(10, n_trees=9)


@pytest.mark.parametrize("name,n,d_ok", [("subspace16_d128", 9000, 128), ("aniso20_d64", 9000, 64)])
def test_chosen_form_leaves_up_to_256_points(name, n, d_ok):
    # leaf bound 256: 256-row tiles, two M = 128 tensor-core blocks against all
    # rows; d = 128 also runs the Gram in two 64-coordinate chunks
    X = synth.make(name, n=n)
    assert X.shape[1] == d_ok
    o = oracle.Forest(X, 3, 256, 3, seed=8)
    oi, od = o.all_knn(20)
    c = gpu_forest(X, 3, 256, 3, seed=8, form=1)
    p = gpu_forest(X, 3, 256, 3, seed=8, form=0)
    ci, cd = c.all_knn(20)
    pi, pd = p.all_knn(20)
    assert torch.equal(ci, pi) and torch.equal(cd, pd)
    check_knn(ci.cpu().numpy(), cd.cpu().numpy(), oi, od, X)


@pytest.mark.parametrize("case", ["identical", "duplicates", "huge", "tiny", "small", "few"])
def test_chosen_form_degenerate_and_extreme_scales(case):
    # d = 8 so that the tensor-core form runs; leaves of all-equal points
    # (spread 0) and coordinates near 3e18 or 1e-25 fall outside the range
    # the certificate covers and are scanned exactly; 1e-10 stays inside it
    rng = np.random.default_rng(11)
    n, d = 3000, 8
    if case == "identical":
        X = np.full((600, d), 2.5, np.float32)
    elif case == "duplicates":
        X = rng.standard_normal((n, d)).astype(np.float32)
        X[200:900] = X[5]
    elif case == "huge":
        X = (3e18 * rng.standard_normal((n, d))).astype(np.float32)
    elif case == "tiny":
        X = (1e-25 * rng.standard_normal((n, d))).astype(np.float32)
    elif case == "small":
        X = (1e-10 * rng.standard_normal((n, d))).astype(np.float32)
    else:
        X = rng.standard_normal((40, d)).astype(np.float32)
    o = oracle.Forest(X, 3, 64, 3, seed=2)
    oi, od = o.all_knn(10)
    c = gpu_forest(X, 3, 64, 3, seed=2, form=1)
    ci, cd = c.all_knn(10)
    assert np.array_equal(ci.cpu().numpy(), oi) and np.array_equal(cd.cpu().numpy(), od)


def _median_forest(X, T, L, ntry, seed=0, growth=0, form=0):
    from paper_1812_11689_gb300 import forest
    return F(torch.from_numpy(np.ascontiguousarray(X)).cuda(), n_trees=T, leaf_max=L, n_try=ntry,
             seed=seed, growth=growth, form=form, split_rule=forest.SPLIT_MEDIAN)


@pytest.mark.parametrize("name,n,L,ntry", [("mix5_d10", 2000, 50, 5),
                                           ("aniso20_d64", 30000, 128, 5),
                                           ("student3_d32", 20000, 64, 3)])
def test_median_rule_trees_and_all_knn_bit_exact(name, n, L, ntry):
    # the level-synchronous phase (nodes > 4096 points) and the CTA subtrees
    # both select the median by radix passes; both growth modes
    X = synth.make(name, n=n)
    o = oracle.Forest(X, 4, L, ntry, seed=7, split_rule=1)
    for growth in (1, 2):
        g = _median_forest(X, 4, L, ntry, seed=7, growth=growth)
        compare_trees(g, o, 4)
    oi, od = o.all_knn(10)
    for form in (0, 1):
        g = _median_forest(X, 4, L, ntry, seed=7, form=form)
        gi, gd = g.all_knn(10)
        check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)


def test_median_rule_ties_and_queries():
    # integer coordinates on a line and a duplicate block: ties at the median
    # are split by point index; queries route on the median value
    rng = np.random.default_rng(9)
    X1 = rng.integers(0, 40, size=(12000, 1)).astype(np.float32)
    o = oracle.Forest(X1, 3, 30, 2, seed=2, split_rule=1)
    compare_trees(_median_forest(X1, 3, 30, 2, seed=2), o, 3)
    X = synth.make("mix50_d96", n=9000)
    X[100:700] = X[3]
    o = oracle.Forest(X, 3, 64, 3, seed=4, split_rule=1)
    g = _median_forest(X, 3, 64, 3, seed=4)
    compare_trees(g, o, 3)
    Q = synth.queries("mix50_d96", 300, stream=31)
    qi, qd = g.query(torch.from_numpy(Q).cuda(), 10)
    oi, od = o.query(Q, 10)
    assert np.array_equal(qi.cpu().numpy(), oi) and np.array_equal(qd.cpu().numpy(), od)


def test_median_rule_mixed_band_sizes_in_one_level():
    # 3000 copies of one off-centre point among 9000 others: depending on the
    # tree's direction the root median falls inside the copies (a band far
    # above 256 points, radix passes) or outside them (a small band, settled
    # directly), so one level of the level-synchronous phase mixes both
    X = synth.make("mix50_d96", n=12000)
    X[9000:] = X[17]
    o = oracle.Forest(X, 6, 64, 3, seed=21, split_rule=1)
    compare_trees(_median_forest(X, 6, 64, 3, seed=21), o, 6)


@pytest.mark.parametrize("form,split_rule", [(0, 0), (1, 0), (1, 1)])
def test_add_trees_equals_the_larger_build(form, split_rule):
    # 3 trees, then 2 and 1 more: the forest a 6-tree build grows
    from paper_1812_11689_gb300 import forest
    X = synth.make("aniso20_d64", n=15000)
    kw = dict(leaf_max=128, n_try=5, seed=12, form=form, split_rule=split_rule)
    Xd = torch.from_numpy(X).cuda()
    g = forest.Forest(Xd, n_trees=3, **kw)
    g.add_trees(2)
    g.add_trees(1)
    assert g.info()["n_trees"] == 6
    o = oracle.Forest(X, 6, 128, 5, seed=12, split_rule=split_rule)
    compare_trees(g, o, 6)
    oi, od = o.all_knn(10)
    gi, gd = g.all_knn(10)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)
    Q = synth.queries("aniso20_d64", 200, stream=41)
    qi, qd = g.query(torch.from_numpy(Q).cuda(), 10)
    ri, rd = o.query(Q, 10)
    assert np.array_equal(qi.cpu().numpy(), ri) and np.array_equal(qd.cpu().numpy(), rd)
    with pytest.raises(RuntimeError):
        g.add_trees(0)


def test_autotune_picks_a_configuration_and_keeps_the_lists():
    X = synth.make("aniso20_d64", n=20000)
    c = gpu_forest(X, 4, 128, 5, seed=3, form=1)
    ci0, cd0 = c.all_knn(10)
    Qd = torch.from_numpy(synth.queries("aniso20_d64", 400, stream=8)).cuda()
    qi0, qd0 = c.query(Qd, 10)
    ch = c.autotune(10)
    assert ch["gram_chunk"] in (16, 32, 48, 64) and 1 <= ch["ctas_per_sm"] <= 4
    assert ch["tile_rows"] in (128, 256)
    assert ch["query_scan"] in ("bf16", "fp32")
    qi1, qd1 = c.query(Qd, 10)  # whichever scan was kept: the same lists
    assert torch.equal(qi0, qi1) and torch.equal(qd0, qd1)
    ci1, cd1 = c.all_knn(10)
    assert torch.equal(ci0, ci1) and torch.equal(cd0, cd1)
    # a new forest of the same shape takes the tuned tile rows
    c2 = gpu_forest(X, 4, 128, 5, seed=3, form=1)
    ci2, cd2 = c2.all_knn(10)
    assert torch.equal(ci0, ci2) and torch.equal(cd0, cd2)
    p = gpu_forest(X, 4, 128, 5, seed=3, form=0)
    pi0, pd0 = p.all_knn(10)
    ph = p.autotune(10)
    assert ph["gram_chunk"] == 0 and ph["tile_region"] % 32 == 0 and ph["tile_region"] >= 32
    assert p.counters()["tile_region"] == ph["tile_region"]
    pi1, pd1 = p.all_knn(10)
    assert torch.equal(pi0, pi1) and torch.equal(pd0, pd1) and torch.equal(pi0, ci0)


@pytest.mark.parametrize("d", [3, 10, 13, 30])
def test_chosen_form_runs_the_tensor_path_at_any_dimension(d):
    # rows of d % 4 != 0 floats are not 16-byte multiples: the tile kernel
    # loads them with the warps instead of bulk copies; lists stay bit-exact
    rng = np.random.default_rng(d)
    X = (rng.standard_normal((6000, d)) * rng.uniform(0.5, 2.0, d)).astype(np.float32)
    X[:40] = X[40:80]  # duplicates: equal keys across rows
    g = gpu_forest(X, 4, 100, 3, form=1)
    gi, gd = g.all_knn(8)
    o = oracle.Forest(X, 4, 100, 3, seed=0)
    oi, od = o.all_knn(8)
    check_knn(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, X)
    c = g.counters()
    assert c["chosen_form_plain_groups"] == 0  # the tensor path ran
    # K above the tensor path's 32: the plain form runs, and is counted
    gi, gd = g.all_knn(40)
    oi, od = o.all_knn(40)
    assert np.array_equal(gi.cpu().numpy(), oi) and np.array_equal(gd.cpu().numpy(), od)
    assert g.counters()["chosen_form_plain_groups"] >= 1


@pytest.mark.parametrize("name,n,L,Ks", [("mix50_d96", 20000, 128, (1, 10, 32, 50)),
                                         ("aniso20_d64", 12000, 128, (10, 20)),
                                         ("mix5_d10", 3000, 50, (5, 12))])
def test_chosen_form_queries_bf16_scan_bit_exact(name, n, L, Ks):
    # the chosen form's query scan reads BF16 rows and re-ranks a certified
    # shortlist exactly: the lists equal the plain form's and the oracle's
    X = synth.make(name, n=n)
    Q = synth.queries(name, 600, stream=31)
    c = gpu_forest(X, 5, L, 5, form=1)
    p = gpu_forest(X, 5, L, 5, form=0)
    o = oracle.Forest(X, 5, L, 5, seed=0)
    Qd = torch.from_numpy(Q).cuda()
    for K in Ks:
        pi, pd = p.query(Qd, K)
        oi, od = o.query(Q, K)
        assert np.array_equal(pi.cpu().numpy(), oi) and np.array_equal(pd.cpu().numpy(), od), K
        # each scan of the chosen form, whatever an earlier autotune picked
        for mode in ("bf16", "fp32", None):
            c.set_query_scan(mode)
            ci, cd = c.query(Qd, K)
            assert torch.equal(ci, pi) and torch.equal(cd, pd), (K, mode)


def test_chosen_form_queries_long_shortlist_falls_back_exactly():
    # points on a thin shell around the origin, queried at the origin: every
    # leaf point is within the certified margin of the K-th, so each leaf is
    # rescanned exactly (counted) and the lists stay bit-exact
    rng = np.random.default_rng(5)
    g = rng.standard_normal((4000, 64))
    X = (g / np.linalg.norm(g, axis=1, keepdims=True) * (1.0 + 1e-4 * rng.random((4000, 1))))
    X = X.astype(np.float32)
    Q = np.zeros((50, 64), np.float32)
    Q[1:] = 1e-3 * rng.standard_normal((49, 64)).astype(np.float32)
    c = gpu_forest(X, 3, 128, 3, form=1)
    c.set_query_scan("bf16")
    o = oracle.Forest(X, 3, 128, 3, seed=0)
    before = c.counters()["bf16_fallback_rows"]
    ci, cd = c.query(torch.from_numpy(Q).cuda(), 10)
    oi, od = o.query(Q, 10)
    assert np.array_equal(ci.cpu().numpy(), oi) and np.array_equal(cd.cpu().numpy(), od)
    assert c.counters()["bf16_fallback_rows"] > before


def test_set_form_switches_a_built_forest_and_keeps_the_lists():
    X = synth.make("aniso20_d64", n=9000)
    Q = torch.from_numpy(synth.queries("aniso20_d64", 300, stream=4)).cuda()
    f = gpu_forest(X, 4, 128, 5, form=0)
    pi, pd = f.all_knn(10)
    qi, qd = f.query(Q, 10)
    f.set_form(1)  # builds the tile packing and the BF16 copy
    ci, cd = f.all_knn(10)
    ri, rd = f.query(Q, 10)
    assert torch.equal(pi, ci) and torch.equal(pd, cd)
    assert torch.equal(qi, ri) and torch.equal(qd, rd)
    assert f.counters()["chosen_form_plain_groups"] == 0
    f.set_form(0)
    ai, ad = f.all_knn(10)
    assert torch.equal(pi, ai) and torch.equal(pd, ad)


def test_gather_probe_rate_is_positive_and_checks_its_arguments():
    from paper_1812_11689_gb300 import _lib, forest
    X = torch.from_numpy(synth.make("aniso20_d64", n=50000)).cuda()
    assert forest.gather_rate(X, rows=1 << 18, reps=2) > 0
    with pytest.raises(ValueError):
        forest.gather_rate(X.cpu())
    out = torch.zeros(1, device="cuda")
    L = _lib.lib()
    assert L.rpf_gather_probe(X.data_ptr(), X.shape[0], 6, 1, 0, out.data_ptr(), None) == -1
    assert out.item() == 0.0
