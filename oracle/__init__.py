"""rpForests CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow C restatement of random projection forests kNN search (Yan et al.,
arXiv 1812.11689): rpTree growth (Sec. 2, Algorithm 1), direction choice
(Algorithm 2), ensemble kNN search (Algorithm 3), exact brute-force kNN and the
Sec. 5.1 metrics (missing rate, kNN-distance discrepancy).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1812_11689_gb300`` and never imports
it; the CUDA library never imports this package.

Parity notes: every function here is pinned by tests in ``tests/test_oracle_*``
to something outside itself (published SplitMix64 outputs, libm accuracy,
closed forms, brute force, invariants of Algorithms 1-3).  The absolute missing
rates the paper plots (Figs. 2-3) are not available, so those values are
"parity unpinned"; only their trends are checked.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librpf_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-math-errno", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/ (idempotent)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u64 = ctypes.c_uint64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_mix64.restype = _u64
            L.orc_mix64.argtypes = [_u64]
            L.orc_word.restype = _u64
            L.orc_word.argtypes = [_u64] * 6
            L.orc_child_key.restype = _u64
            L.orc_child_key.argtypes = [_u64, ctypes.c_int]
            L.orc_u53.restype = ctypes.c_double
            L.orc_u53.argtypes = [_u64]
            L.orc_lnf.restype = ctypes.c_float
            L.orc_lnf.argtypes = [ctypes.c_float]
            L.orc_sincos2pif.restype = None
            L.orc_sincos2pif.argtypes = [ctypes.c_float, _f32p, _f32p]
            L.orc_direction.restype = None
            L.orc_direction.argtypes = [_u64, _u64, _u64, _u64, ctypes.c_int, _f64p]
            L.orc_proj.restype = ctypes.c_double
            L.orc_proj.argtypes = [_f32p, _f64p, ctypes.c_int]
            L.orc_csum.restype = ctypes.c_double
            L.orc_csum.argtypes = [_f64p, ctypes.c_int64]
            L.orc_d32.restype = ctypes.c_float
            L.orc_d32.argtypes = [_f32p, _f32p, ctypes.c_int]
            L.orc_build.restype = ctypes.c_void_p
            L.orc_build.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, _u64, ctypes.c_int32,
                                    ctypes.c_int32]
            L.orc_build_range.restype = ctypes.c_void_p
            L.orc_build_range.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _u64,
                                          ctypes.c_int32, ctypes.c_int32]
            L.orc_all_knn_keys.restype = None
            L.orc_all_knn_keys.argtypes = [ctypes.c_void_p, _f32p, _i32p, ctypes.c_int64,
                                           ctypes.c_int32, _i32p, _f32p, ctypes.c_int32]
            L.orc_free.restype = None
            L.orc_free.argtypes = [ctypes.c_void_p]
            L.orc_n_nodes.restype = ctypes.c_int64
            L.orc_n_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            L.orc_get_perm.restype = None
            L.orc_get_perm.argtypes = [ctypes.c_void_p, ctypes.c_int32, _i32p]
            L.orc_get_nodes.restype = None
            L.orc_get_nodes.argtypes = [ctypes.c_void_p, ctypes.c_int32, _i64p, _f64p]
            L.orc_get_node_dir.restype = None
            L.orc_get_node_dir.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, _f64p]
            L.orc_all_knn.restype = None
            L.orc_all_knn.argtypes = [ctypes.c_void_p, _f32p, ctypes.c_int32, _i32p, _f32p,
                                      ctypes.c_int32]
            L.orc_all_knn_rows.restype = None
            L.orc_all_knn_rows.argtypes = [ctypes.c_void_p, _f32p, _i32p, ctypes.c_int64,
                                           ctypes.c_int32, _i32p, _f32p, ctypes.c_int32]
            L.orc_route.restype = ctypes.c_int64
            L.orc_route.argtypes = [ctypes.c_void_p, ctypes.c_int32, _f32p]
            L.orc_query.restype = None
            L.orc_query.argtypes = [ctypes.c_void_p, _f32p, _f32p, ctypes.c_int64,
                                    ctypes.c_int32, _i32p, _f32p, ctypes.c_int32]
            L.orc_brute_knn.restype = None
            L.orc_brute_knn.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _f32p,
                                        ctypes.c_int64, _i32p, ctypes.c_int32, _i32p, _f32p,
                                        _f64p, ctypes.c_int32]
            L.orc_have_openmp.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------
# scalar building blocks (exposed for the pins)
# --------------------------------------------------------------------------
def mix64(z: int) -> int:
    return int(lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def word(seed, tag, t, key, j, c) -> int:
    return int(lib().orc_word(seed, tag, t, key, j, c))


def child_key(key: int, side: int) -> int:
    return int(lib().orc_child_key(key, side))


def u53(w: int) -> float:
    return float(lib().orc_u53(w))


def lnf(u: float) -> np.float32:
    return np.float32(lib().orc_lnf(np.float32(u)))


def sincos2pif(u: float):
    c, s = ctypes.c_float(), ctypes.c_float()
    lib().orc_sincos2pif(np.float32(u), ctypes.byref(c), ctypes.byref(s))
    return np.float32(c.value), np.float32(s.value)


def direction(seed: int, t: int, key: int, j: int, d: int) -> np.ndarray:
    r = np.empty(d, np.float64)
    lib().orc_direction(seed, t, key, j, d, _p(r, _f64p))
    return r


def proj(x: np.ndarray, r: np.ndarray) -> float:
    x = np.ascontiguousarray(x, np.float32)
    r = np.ascontiguousarray(r, np.float64)
    return float(lib().orc_proj(_p(x, _f32p), _p(r, _f64p), x.size))


def csum(v: np.ndarray) -> float:
    v = np.ascontiguousarray(v, np.float64)
    return float(lib().orc_csum(_p(v, _f64p), v.size))


def d32(x: np.ndarray, y: np.ndarray) -> np.float32:
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    return np.float32(lib().orc_d32(_p(x, _f32p), _p(y, _f32p), x.size))


# --------------------------------------------------------------------------
# forest
# --------------------------------------------------------------------------
NODE_FIELDS = ("key", "begin", "len", "depth", "leaf", "jstar", "flag", "attempt",
               "left", "right")


class Forest:
    """T rpTrees grown on X (Algorithm 3, first loop).

    split_rule 0: c drawn uniformly on [a, b] (Algorithm 1); 1: the median of
    the projections (Sec. 2's other usual split point), ties by point index.
    """

    def __init__(self, X: np.ndarray, n_trees: int, leaf_max: int, n_try: int,
                 seed: int = 0, threads: int | None = None, split_rule: int = 0,
                 tree_first: int = 0):
        """tree_first: global index of the first tree grown; the forest then
        holds trees tree_first .. tree_first + n_trees - 1 of the ensemble."""
        self.X = np.ascontiguousarray(X, np.float32)
        self.n, self.d = self.X.shape
        self.T, self.L, self.n_try, self.seed = n_trees, leaf_max, n_try, seed
        self.split_rule = split_rule
        self.tree_first = tree_first
        self.threads = threads or default_threads()
        h = lib().orc_build_range(_p(self.X, _f32p), self.n, self.d, tree_first, n_trees,
                                  leaf_max, n_try, seed, self.threads, split_rule)
        if not h:
            raise ValueError("orc_build rejected its arguments")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def perm(self, t: int) -> np.ndarray:
        out = np.empty(self.n, np.int32)
        lib().orc_get_perm(self._h, t, _p(out, _i32p))
        return out

    def nodes(self, t: int) -> dict:
        nn = lib().orc_n_nodes(self._h, t)
        I = np.empty((nn, 10), np.int64)
        D = np.empty((nn, 3), np.float64)
        lib().orc_get_nodes(self._h, t, _p(I, _i64p), _p(D, _f64p))
        out = {f: I[:, i] for i, f in enumerate(NODE_FIELDS)}
        out["key"] = I[:, 0].view(np.uint64)
        out["c"], out["a"], out["b"] = D[:, 0], D[:, 1], D[:, 2]
        return out

    def node_dir(self, t: int, i: int) -> np.ndarray:
        r = np.empty(self.d, np.float64)
        lib().orc_get_node_dir(self._h, t, i, _p(r, _f64p))
        return r

    def leaves(self, t: int):
        """(begin, len) of every leaf of tree t, sorted by begin."""
        nd = self.nodes(t)
        m = nd["leaf"] == 1
        order = np.argsort(nd["begin"][m], kind="stable")
        return nd["begin"][m][order], nd["len"][m][order]

    def all_knn(self, K: int):
        idx = np.empty((self.n, K), np.int32)
        dist = np.empty((self.n, K), np.float32)
        lib().orc_all_knn(self._h, _p(self.X, _f32p), K, _p(idx, _i32p), _p(dist, _f32p),
                          self.threads)
        return idx, dist

    def all_knn_rows(self, rows, K: int):
        rows = np.ascontiguousarray(rows, np.int32)
        idx = np.empty((rows.size, K), np.int32)
        dist = np.empty((rows.size, K), np.float32)
        lib().orc_all_knn_rows(self._h, _p(self.X, _f32p), _p(rows, _i32p), rows.size, K,
                               _p(idx, _i32p), _p(dist, _f32p), self.threads)
        return idx, dist

    def all_knn_keys(self, K: int, rows=None):
        """Per-point lists over this forest's trees with the squared key d32
        (FP32) instead of the distance: (idx int32, d32 float32), rows of all
        points unless `rows` is given."""
        rows = (np.arange(self.n, dtype=np.int32) if rows is None
                else np.ascontiguousarray(rows, np.int32))
        idx = np.empty((rows.size, K), np.int32)
        d32 = np.empty((rows.size, K), np.float32)
        lib().orc_all_knn_keys(self._h, _p(self.X, _f32p), _p(rows, _i32p), rows.size, K,
                               _p(idx, _i32p), _p(d32, _f32p), self.threads)
        return idx, d32

    def route(self, t: int, q: np.ndarray) -> int:
        q = np.ascontiguousarray(q, np.float32)
        return int(lib().orc_route(self._h, t, _p(q, _f32p)))

    def query(self, Q: np.ndarray, K: int):
        Q = np.ascontiguousarray(Q, np.float32)
        m = Q.shape[0]
        idx = np.empty((m, K), np.int32)
        dist = np.empty((m, K), np.float32)
        lib().orc_query(self._h, _p(self.X, _f32p), _p(Q, _f32p), m, K, _p(idx, _i32p),
                        _p(dist, _f32p), self.threads)
        return idx, dist


def brute_knn(X: np.ndarray, K: int, rows=None, Q=None, threads: int | None = None):
    """Exact kNN under the (d32, idx) order.

    rows: indices of data points to answer (self excluded); Q: new points
    (nothing excluded).  Returns (idx int32, dist float32, dist64 float64).
    """
    X = np.ascontiguousarray(X, np.float32)
    n, d = X.shape
    if Q is None:
        rows = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, np.int32)
        Qa = np.ascontiguousarray(X[rows])
        selfp = _p(rows, _i32p)
    else:
        Qa = np.ascontiguousarray(Q, np.float32)
        rows = None
        selfp = None
    nr = Qa.shape[0]
    idx = np.empty((nr, K), np.int32)
    dist = np.empty((nr, K), np.float32)
    d64 = np.empty((nr, K), np.float64)
    lib().orc_brute_knn(_p(X, _f32p), n, d, _p(Qa, _f32p), nr, selfp, K, _p(idx, _i32p),
                        _p(dist, _f32p), _p(d64, _f64p), threads or default_threads())
    return idx, dist, d64


def merge_key_lists(idx_lists, d32_lists, K: int):
    """The K nearest of the union of several candidate lists per point
    (Algorithm 3's N_q = union of leaves, taken over groups of trees): for
    each point, the distinct (d32, index) pairs of all lists in ascending
    order, the first K, padded with (-1, +inf); distances are sqrtf(d32).
    idx_lists / d32_lists: G arrays of shape (n, K')."""
    n = idx_lists[0].shape[0]
    idx = np.full((n, K), -1, np.int32)
    dist = np.full((n, K), np.inf, np.float32)
    for i in range(n):
        pairs = set()
        for il, dl in zip(idx_lists, d32_lists):
            for j, v in zip(il[i], dl[i]):
                if j >= 0:
                    pairs.add((float(v), int(j)))
        best = sorted(pairs)[:K]
        for k, (v, j) in enumerate(best):
            idx[i, k] = j
            dist[i, k] = np.sqrt(np.float32(v))
    return idx, dist


# --------------------------------------------------------------------------
# Sec. 5.1 metrics
# --------------------------------------------------------------------------
def missing_rate(found_idx: np.ndarray, true_idx: np.ndarray) -> float:
    """m_bar_k = (1/(nk)) sum_i m(i), m(i) = |trueK(i) minus found(i)| (Sec. 5.1).

    Padding entries (-1) in the true lists are not neighbours and are not
    counted; padding in the found lists never matches, so it counts as a miss.
    """
    found_idx = np.asarray(found_idx)
    true_idx = np.asarray(true_idx)
    n, K = true_idx.shape
    miss = 0
    for i in range(n):
        t = set(int(v) for v in true_idx[i] if v >= 0)
        f = set(int(v) for v in found_idx[i] if v >= 0)
        miss += len(t - f)
    return miss / float(n * K)


def knn_distance_discrepancy(found_dist: np.ndarray, true_dist: np.ndarray) -> float:
    """Relative gap of the average k-th NN distance (Sec. 5.1, d_bar_k):

    (mean_i dhat_K(i) - mean_i d_K(i)) / mean_i d_K(i), over points whose true
    and found lists are both full.  It is >= 0 because dhat_K(i) >= d_K(i).
    """
    fk = np.asarray(found_dist)[:, -1].astype(np.float64)
    tk = np.asarray(true_dist)[:, -1].astype(np.float64)
    ok = np.isfinite(fk) & np.isfinite(tk)
    if not ok.any():
        return 0.0
    mt = tk[ok].mean()
    if mt == 0.0:
        return 0.0
    return float((fk[ok].mean() - mt) / mt)
