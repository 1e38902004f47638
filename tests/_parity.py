"""Shared checks of the GPU parity tests (GPU forest against the oracle).

The tolerance: distances are reported as sqrtf of the canonical FP32 squared
distance, whose relative error against FP64 is at most (d + 3) 2^-24, below
1e-5 for every d <= 164.
"""
import numpy as np

REL_TOL_FP64 = 1e-5


def compare_trees(g, o, T):
    """Trees 0..T-1 of the GPU forest g (which may hold more: nested
    ensembles) against the oracle forest o: permutations, leaf tables and the
    split records (chosen try, rank-split flag, split point bits) keyed by
    (tree, node key)."""
    nodes = g.nodes()
    for t in range(T):
        assert np.array_equal(g.perm(t), o.perm(t)), "perm of tree %d differs" % t
    tr, b, ln = g.leaves()
    for t in range(T):
        ob, ol = o.leaves(t)
        sel = tr == t
        order = np.argsort(b[sel])
        assert np.array_equal(b[sel][order], ob) and np.array_equal(ln[sel][order], ol)
    # split records keyed by (tree, node key)
    gi = {}
    for i in range(len(nodes["key"])):
        if nodes["left"][i] >= 0 and nodes["tree"][i] < T:
            gi[(int(nodes["tree"][i]), int(nodes["key"][i]))] = (
                int(nodes["jstar"][i]), int(nodes["flag"][i]) & 1, nodes["c"][i])
    count = 0
    for t in range(T):
        on = o.nodes(t)
        for i in np.where(on["leaf"] == 0)[0]:
            js, fl, c = gi[(t, int(on["key"][i]))]
            assert js == int(on["jstar"][i]) and fl == int(on["flag"][i])
            if not fl:
                assert np.float64(c).view(np.uint64) == np.float64(on["c"][i]).view(np.uint64)
            count += 1
    assert count == len(gi)


def check_knn(gi, gd, oi, od, X, rows=None):
    """Indices and distances bit-exact against the oracle; distances within
    REL_TOL_FP64 of the FP64 Euclidean distance (rows: the data rows the
    lists belong to, all rows if None)."""
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd, od)
    # distances vs FP64 (non-padded slots)
    rows = np.arange(len(gi)) if rows is None else rows
    ok = gi >= 0
    xi = X[np.repeat(rows, gi.shape[1])[ok.ravel()]].astype(np.float64)
    xj = X[gi[ok]].astype(np.float64)
    d64 = np.sqrt(((xi - xj) ** 2).sum(1))
    rel = np.abs(gd[ok].astype(np.float64) - d64) / np.maximum(d64, 1e-30)
    assert rel.max() <= REL_TOL_FP64
