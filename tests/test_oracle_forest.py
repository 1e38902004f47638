"""Pins of the oracle's rpTree growth (Algorithms 1-2) and ensemble search
(Algorithm 3) against invariants, special cases and brute force.

* every tree partitions all n points exactly once, no leaf exceeds the bound
  and every split node exceeds it (Algorithm 1, leaf rule);
* every split sends p < c left and p >= c right, with c in (a, b], and the
  chosen direction has the largest projected dispersion (Algorithm 2) --
  recomputed here with NumPy, independently of the oracle's arithmetic;
* d = 1 trees cut the sorted line into intervals;
* T = 1 with a leaf bound >= n is exact kNN, bit for bit;
* the kNN lists equal a Python union-of-leaves search (Algorithm 3), are sound
  (each neighbour shares a leaf with the point) and per-tree top-K truncation
  loses nothing;
* nested ensembles: adding trees never raises any point's miss count nor its
  K-th neighbour distance, and d_hat_K >= d_K (Sec. 5.1);
* brute force agrees with a NumPy FP64 argsort away from near-ties.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_11689_gb300 import synth


@pytest.fixture(scope="module")
def cfg1():
    X = synth.make("mix5_d10")
    return X, oracle.Forest(X, 10, 50, 5, seed=0)


def _check_tree(F, t, X):
    n = F.n
    perm = F.perm(t)
    assert np.array_equal(np.sort(perm), np.arange(n))
    nd = F.nodes(t)
    begins, lens = F.leaves(t)
    # leaves tile [0, n)
    assert begins[0] == 0 and np.all(begins[1:] == begins[:-1] + lens[:-1])
    assert begins[-1] + lens[-1] == n
    assert lens.min() >= 1 and lens.max() <= F.L
    # stable partitions from the ascending root: every leaf stays ascending
    for b, m in zip(begins, lens):
        assert np.all(np.diff(perm[b:b + m]) > 0)
    internal = np.where(nd["leaf"] == 0)[0]
    assert np.all(nd["len"][internal] > F.L)
    for i in internal:
        b, m = nd["begin"][i], nd["len"][i]
        li, ri = nd["left"][i], nd["right"][i]
        assert nd["begin"][li] == b and nd["begin"][ri] == b + nd["len"][li]
        assert nd["len"][li] + nd["len"][ri] == m and nd["len"][li] >= 1 and nd["len"][ri] >= 1
        assert nd["key"][li] == np.uint64(oracle.child_key(int(nd["key"][i]), 0))
        assert nd["key"][ri] == np.uint64(oracle.child_key(int(nd["key"][i]), 1))
        L_mem, R_mem = perm[b:b + nd["len"][li]], perm[b + nd["len"][li]:b + m]
        if nd["flag"][i]:
            continue
        r = F.node_dir(t, i)
        c, a, bb = nd["c"][i], nd["a"][i], nd["b"][i]
        pl = X[L_mem].astype(np.float64) @ r
        pr = X[R_mem].astype(np.float64) @ r
        scale = np.abs(X[np.concatenate([L_mem, R_mem])].astype(np.float64)).sum(1).max()
        tol = 4 * X.shape[1] * 2.0 ** -53 * scale
        assert np.all(pl < c + tol) and np.all(pr >= c - tol)
        assert a < c <= bb
        allp = np.concatenate([pl, pr])
        assert abs(allp.min() - a) <= tol and abs(allp.max() - bb) <= tol
        # c = a + u (b - a), u from the split word of the accepted attempt
        u = oracle.u53(oracle.word(F.seed, 2, t, int(nd["key"][i]), int(nd["attempt"][i]), 0))
        assert abs(c - (a + u * (bb - a))) <= 4 * 2.0 ** -53 * max(abs(a), abs(bb))
        # Algorithm 2: the chosen try has the largest dispersion of the nTry
        mem = np.concatenate([L_mem, R_mem])
        Vs = []
        for j in range(F.n_try):
            rj = oracle.direction(F.seed, t, int(nd["key"][i]), j, X.shape[1])
            p = X[mem].astype(np.float64) @ rj
            Vs.append(np.sum((p - p.mean()) ** 2))
        Vs = np.array(Vs)
        js = int(nd["jstar"][i])
        assert np.array_equal(rj if js == F.n_try - 1 else oracle.direction(
            F.seed, t, int(nd["key"][i]), js, X.shape[1]), r)
        top = np.sort(Vs)[::-1]
        if F.n_try > 1 and top[0] - top[1] > 1e-9 * top[0]:
            assert js == int(np.argmax(Vs))
    return nd


def test_trees_partition_and_split_rules(cfg1):
    X, F = cfg1
    for t in range(F.T):
        _check_tree(F, t, X)


def test_heavy_tailed_and_anisotropic_trees():
    for name, n, L in (("student3_d32", 3000, 64), ("aniso20_d64", 3000, 128)):
        X = synth.make(name, n=n)
        F = oracle.Forest(X, 3, L, 5, seed=11)
        for t in range(F.T):
            _check_tree(F, t, X)


def test_single_try_tree_is_basic_rptree():
    X = synth.make("mix5_d10", n=1500)
    F = oracle.Forest(X, 2, 20, 1, seed=3)
    for t in range(F.T):
        nd = _check_tree(F, t, X)
        assert set(nd["jstar"][nd["leaf"] == 0]) <= {0}


def test_d1_leaves_are_intervals_of_the_sorted_line():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((1000, 1)).astype(np.float32)
    F = oracle.Forest(X, 4, 30, 3, seed=5)
    for t in range(F.T):
        perm = F.perm(t)
        begins, lens = F.leaves(t)
        spans = sorted((X[perm[b:b + m], 0].min(), X[perm[b:b + m], 0].max())
                       for b, m in zip(begins, lens))
        for (lo0, hi0), (lo1, hi1) in zip(spans[:-1], spans[1:]):
            assert hi0 < lo1


def test_degenerate_data_duplicates_and_constant_columns():
    X = np.ones((300, 5), np.float32)
    F = oracle.Forest(X, 2, 16, 3, seed=0)
    for t in range(F.T):
        nd = _check_tree(F, t, X)
        assert np.all(nd["flag"][nd["leaf"] == 0] == 1)
    idx, dist = F.all_knn(3)
    assert np.all(dist == 0.0) and np.all(idx >= 0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((400, 6)).astype(np.float32)
    X[:, 2] = 7.0
    X[100:200] = X[0]
    F = oracle.Forest(X, 3, 10, 4, seed=2)
    for t in range(F.T):
        _check_tree(F, t, X)


def test_nested_ensemble_prefix_trees_identical():
    X = synth.make("mix5_d10", n=800)
    F3 = oracle.Forest(X, 3, 25, 3, seed=9)
    F6 = oracle.Forest(X, 6, 25, 3, seed=9)
    for t in range(3):
        assert np.array_equal(F3.perm(t), F6.perm(t))
    assert not np.array_equal(F6.perm(3), F6.perm(4))


def test_one_tree_with_leaf_bound_ge_n_is_exact_knn():
    X = synth.make("mix5_d10", n=700)
    F = oracle.Forest(X, 1, 700, 5, seed=0)
    assert F.nodes(0)["leaf"].tolist() == [1]
    idx, dist = F.all_knn(7)
    bi, bd, _ = oracle.brute_knn(X, 7)
    assert np.array_equal(idx, bi) and np.array_equal(dist, bd)


def _python_union_knn(F, X, K, exclude_self=True):
    n = F.n
    leaf_of = []
    for t in range(F.T):
        perm = F.perm(t)
        lo = np.empty(n, np.int64)
        for b, m in zip(*F.leaves(t)):
            lo[perm[b:b + m]] = b
        leaf_of.append((perm, lo, dict(zip(*F.leaves(t)))))
    out_i = np.full((n, K), -1, np.int32)
    out_d = np.full((n, K), np.inf, np.float32)
    for i in range(n):
        cand = set()
        for perm, lo, lens in leaf_of:
            b = lo[i]
            cand.update(int(v) for v in perm[b:b + lens[b]])
        cand.discard(i)
        ranked = sorted((float(oracle.d32(X[i], X[j])), j) for j in cand)[:K]
        for k, (dv, j) in enumerate(ranked):
            out_i[i, k] = j
            out_d[i, k] = np.sqrt(np.float32(dv))
    return out_i, out_d


def test_all_knn_equals_union_of_leaves_definition():
    X = synth.make("mix5_d10", n=600)
    F = oracle.Forest(X, 4, 20, 3, seed=4)
    idx, dist = F.all_knn(5)
    pi, pd = _python_union_knn(F, X, 5)
    assert np.array_equal(idx, pi) and np.array_equal(dist, pd)


def test_all_knn_rows_equals_all_knn_and_the_union_definition(cfg1):
    # orc_all_knn_rows answers chosen rows of Algorithm 3 with Q = U (the
    # sampled form used at large n): on the 2,000-point workload, every row in
    # a shuffled order with repeats matches orc_all_knn element by element,
    # for several K, and a sample matches the Python union-of-leaves search
    X, F = cfg1
    rng = np.random.default_rng(7)
    rows = np.concatenate([rng.permutation(F.n), rng.integers(0, F.n, 300)]).astype(np.int32)
    for K in (1, 5, 17):
        idx, dist = F.all_knn(K)
        ri, rd = F.all_knn_rows(rows, K)
        assert np.array_equal(ri, idx[rows]) and np.array_equal(rd.view(np.uint32),
                                                                 dist[rows].view(np.uint32))
    Xs = synth.make("mix5_d10", n=600)
    Fs = oracle.Forest(Xs, 4, 20, 3, seed=4)
    pi, pd = _python_union_knn(Fs, Xs, 5)
    sub = np.array([0, 3, 599, 250, 3], np.int32)
    ri, rd = Fs.all_knn_rows(sub, 5)
    assert np.array_equal(ri, pi[sub]) and np.array_equal(rd, pd[sub])


def test_per_tree_truncation_is_exact_and_sound(cfg1):
    X, F = cfg1
    K = 5
    idx, dist = F.all_knn(K)
    n = F.n
    # per-tree top-K lists, then merge: must equal the union search
    per_tree = []
    member_sets = []
    for t in range(F.T):
        perm = F.perm(t)
        best = {}
        sets = np.empty(n, np.int64)
        for b, m in zip(*F.leaves(t)):
            mem = perm[b:b + m]
            sets[mem] = b
            for i in mem:
                c = sorted((float(oracle.d32(X[i], X[j])), int(j)) for j in mem if j != i)[:K]
                best[int(i)] = c
        per_tree.append(best)
        member_sets.append(sets)
    for i in range(0, n, 7):
        merged = sorted(set(c for t in range(F.T) for c in per_tree[t][i]))[:K]
        assert [j for _, j in merged] == [int(v) for v in idx[i] if v >= 0]
        # soundness: each neighbour shares a leaf with i in some tree
        for j in idx[i]:
            assert any(member_sets[t][j] == member_sets[t][i] for t in range(F.T))


def test_nested_ensemble_misses_never_increase_and_dhat_ge_d():
    X = synth.make("mix5_d10", n=1500)
    K = 5
    ti, td, _ = oracle.brute_knn(X, K)
    F = oracle.Forest(X, 16, 30, 3, seed=1)
    prev_miss, prev_dk, prev_rate = None, None, None
    for T in (1, 2, 4, 8, 16):
        sub = oracle.Forest(X, T, 30, 3, seed=1)
        idx, dist = sub.all_knn(K)
        miss = np.array([len(set(ti[i]) - set(idx[i])) for i in range(len(X))])
        dk = dist[:, -1]
        assert np.all(dk >= td[:, -1])
        if prev_miss is not None:
            assert np.all(miss <= prev_miss) and np.all(dk <= prev_dk)
        rate = oracle.missing_rate(idx, ti)
        assert rate == miss.sum() / (len(X) * K)
        if prev_rate is not None:
            assert rate <= prev_rate
        assert oracle.knn_distance_discrepancy(dist, td) >= 0.0
        prev_miss, prev_dk, prev_rate = miss, dk, rate
    assert prev_rate < 0.02
    del F


def test_brute_force_against_numpy_fp64():
    X = synth.make("aniso20_d64", n=700)
    K = 10
    bi, bd, b64 = oracle.brute_knn(X, K)
    X64 = X.astype(np.float64)
    G = ((X64[:, None, :] - X64[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(G, np.inf)
    order = np.argsort(G, axis=1, kind="stable")[:, :K]
    ref = np.sqrt(np.take_along_axis(G, order, 1))
    assert np.allclose(b64, ref, rtol=1e-12, atol=0)
    rel = np.abs(bd.astype(np.float64) - b64) / b64
    assert rel.max() <= (64 + 3) * 2.0 ** -24
    # index sets agree wherever the K-th and (K+1)-th FP64 distances are apart
    Gs = np.sort(G, axis=1)
    gap = (Gs[:, K] - Gs[:, K - 1]) > 1e-5 * Gs[:, K]
    for i in np.where(gap)[0]:
        assert set(bi[i]) == set(order[i])


def test_underfilled_lists_are_padded():
    X = synth.make("mix5_d10", n=4)
    F = oracle.Forest(X, 2, 2, 2, seed=0)
    idx, dist = F.all_knn(5)
    assert np.all(idx[:, 3:] == -1) and np.all(np.isinf(dist[:, 3:]))
    bi, bd, _ = oracle.brute_knn(X, 5)
    assert np.all(bi[:, 3] == -1) and np.all(bi[:, :3] >= 0)


def test_query_routes_points_to_their_build_leaf_and_matches_union():
    X = synth.make("mix5_d10", n=900)
    F = oracle.Forest(X, 5, 30, 3, seed=6)
    for t in range(F.T):
        nd = F.nodes(t)
        if np.any(nd["flag"] == 1):
            continue
        perm = F.perm(t)
        for i in range(0, 900, 13):
            leaf = F.route(t, X[i])
            b, m = nd["begin"][leaf], nd["len"][leaf]
            assert nd["leaf"][leaf] == 1 and i in set(perm[b:b + m])
    Q = synth.queries("mix5_d10", 50)
    qi, qd = F.query(Q, 6)
    for r in range(50):
        cand = set()
        for t in range(F.T):
            nd = F.nodes(t)
            leaf = F.route(t, Q[r])
            cand.update(int(v) for v in F.perm(t)[nd["begin"][leaf]:nd["begin"][leaf] + nd["len"][leaf]])
        ranked = sorted((float(oracle.d32(Q[r], X[j])), j) for j in cand)[:6]
        assert [j for _, j in ranked] == qi[r].tolist()


def test_metric_definitions_on_hand_examples():
    true_i = np.array([[1, 2, 3], [0, 2, 3]])
    found = np.array([[1, 3, 9], [0, 2, 3]])
    assert oracle.missing_rate(found, true_i) == pytest.approx(1 / 6)
    found_pad = np.array([[1, -1, -1], [3, 2, 0]])
    assert oracle.missing_rate(found_pad, true_i) == pytest.approx(2 / 6)
    td = np.array([[1.0, 2.0, 4.0], [1.0, 1.0, 2.0]])
    fd = np.array([[1.0, 2.0, 5.0], [1.0, 1.0, 2.0]])
    assert oracle.knn_distance_discrepancy(fd, td) == pytest.approx((3.5 - 3.0) / 3.0)
    assert oracle.knn_distance_discrepancy(td, td) == 0.0


def _median_checks(F, X, exact_line=False):
    depth_bound = 0
    while -(-F.n // 2 ** depth_bound) > F.L:  # ceil(n / 2^k) > L
        depth_bound += 1
    for t in range(F.T):
        perm = F.perm(t)
        assert np.array_equal(np.sort(perm), np.arange(F.n))
        nd = F.nodes(t)
        assert nd["depth"][nd["leaf"] == 1].max() <= depth_bound
        for i in np.where(nd["leaf"] == 0)[0]:
            b, m = nd["begin"][i], nd["len"][i]
            nl = nd["len"][nd["left"][i]]
            assert nl == m // 2  # halving, rank splits included
            if nd["flag"][i]:
                continue
            r = F.node_dir(t, i)
            mem = perm[b:b + m]
            p = X[mem].astype(np.float64) @ r
            c = nd["c"][i]
            if exact_line:  # d = 1: the products are exact, so is the order
                order = np.lexsort((mem, p))
                assert set(mem[order[:nl]]) == set(mem[:nl])
                assert c == p[order[nl]]
            else:
                tol = 4 * X.shape[1] * 2.0 ** -53 * np.abs(X[mem]).astype(np.float64).sum(1).max()
                assert p[:nl].max() <= c + tol and p[nl:].min() >= c - tol
                assert abs(p[nl:].min() - c) <= tol  # c is the first right point's


def test_median_rule_halves_every_split_at_the_median():
    X = synth.make("aniso20_d64", n=3000)
    F = oracle.Forest(X, 3, 40, 4, seed=1, split_rule=1)
    _median_checks(F, X)
    # the uniform rule on the same data is generally deeper than the halving bound
    assert oracle.Forest(X, 3, 40, 4, seed=1).nodes(0)["depth"].max() >= \
        F.nodes(0)["depth"].max()


def test_median_rule_on_a_line_with_many_ties():
    rng = np.random.default_rng(5)
    X = rng.integers(0, 40, size=(2000, 1)).astype(np.float32)
    F = oracle.Forest(X, 3, 30, 2, seed=2, split_rule=1)
    _median_checks(F, X, exact_line=True)


def test_median_rule_identical_points_take_rank_splits():
    X = np.full((500, 3), 1.5, np.float32)
    F = oracle.Forest(X, 2, 20, 3, seed=0, split_rule=1)
    for t in range(2):
        nd = F.nodes(t)
        assert np.all(nd["flag"][nd["leaf"] == 0] == 1)
    _median_checks(F, X)
