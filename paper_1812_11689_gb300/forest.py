"""Python face of the rpForests CUDA library: the same calls as the C ABI.

``Forest(X, ...)`` -> rpf_build, ``.all_knn(K)`` -> rpf_all_knn,
``.query(Q, K)`` -> rpf_query, ``.close()`` -> rpf_free.  Tensors are passed
by pointer; torch supplies device memory and streams only.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, rpf_params

FORM_PLAIN, FORM_CHOSEN = 0, 1
GROWTH_DEFAULT, GROWTH_FP64, GROWTH_CERTIFIED = 0, 1, 2
SPLIT_UNIFORM, SPLIT_MEDIAN = 0, 1


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int:
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError("expected a torch.Tensor or numpy.ndarray")


def _as_points(X):
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X, np.float32)
        if X.ndim != 2:
            raise ValueError("points must be a 2-D array")
        return X
    if not isinstance(X, torch.Tensor) or X.dim() != 2:
        raise ValueError("points must be a 2-D tensor")
    if X.dtype != torch.float32:
        X = X.float()
    return X.contiguous()


def _check_buffer(name, t, shape, dtype, device=None):
    """Checks of a caller buffer before any launch: type, dtype, contiguity,
    shape, then (for the allocation-free path) that it lives on `device`."""
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch.Tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must have dtype %s, not %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, not %s" % (name, tuple(shape), tuple(t.shape)))
    if device is not None and (not t.is_cuda or t.device != device):
        raise ValueError("%s must be a CUDA tensor on %s" % (name, device))


def _check_out(name, t, shape, dtype):
    """An output buffer of rpf_query: a contiguous tensor or array of the
    right dtype and shape (device or host)."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.dtype(dtype) or not t.flags.c_contiguous or t.shape != tuple(shape):
            raise ValueError("%s must be a contiguous %s array of shape %s"
                             % (name, np.dtype(dtype), tuple(shape)))
        return
    _check_buffer(name, t, shape, {np.int32: torch.int32, np.float32: torch.float32}[dtype])


def _check_query_static(d, Q, K, idx, dist, device):
    """Arguments of rpf_query_static: Q (m x d float32), idx (m x K int32) and
    dist (m x K float32), contiguous CUDA tensors on the forest's device."""
    if not isinstance(Q, torch.Tensor) or Q.dim() != 2:
        raise ValueError("Q must be a 2-D torch.Tensor")
    m = int(Q.shape[0])
    _check_buffer("Q", Q, (m, d), torch.float32, device)
    _check_buffer("idx", idx, (m, K), torch.int32, device)
    _check_buffer("dist", dist, (m, K), torch.float32, device)
    return m


class Forest:
    """T random projection trees over X (n x d, float32; device or host)."""

    def __init__(self, X, n_trees: int = 10, leaf_max: int = 50, n_try: int = 5,
                 form: int = FORM_PLAIN, growth: int = GROWTH_DEFAULT, seed: int = 0,
                 stream=None, split_rule: int = SPLIT_UNIFORM, tree_first: int = 0):
        """tree_first > 0 grows trees tree_first .. tree_first + n_trees - 1
        of the ensemble (rpf_build_shard)."""
        X = _as_points(X)
        self.n, self.d = int(X.shape[0]), int(X.shape[1])
        self.device = X.device if isinstance(X, torch.Tensor) and X.is_cuda else \
            torch.device("cuda", torch.cuda.current_device())
        self.params = rpf_params(n_trees, leaf_max, n_try, split_rule, form, growth, seed)
        h = ctypes.c_void_p()
        self.tree_first = int(tree_first)
        if self.tree_first:
            check(_lib.lib().rpf_build_shard(_ptr(X), self.n, self.d, ctypes.byref(self.params),
                                             self.tree_first, _stream_handle(stream),
                                             ctypes.byref(h)), "rpf_build_shard")
        else:
            check(_lib.lib().rpf_build(_ptr(X), self.n, self.d, ctypes.byref(self.params),
                                       _stream_handle(stream), ctypes.byref(h)), "rpf_build")
        self._h = h

    # ---- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().rpf_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    # ---- search -------------------------------------------------------------
    def workspace_bytes(self, K: int, m: int = 0, all_knn: bool = True) -> int:
        return int(_lib.lib().rpf_workspace_bytes(self._h, m, K, 1 if all_knn else 0))

    def all_knn(self, K: int, idx=None, dist=None, workspace=None, stream=None, n_trees=None):
        """rpf_all_knn; with n_trees, rpf_all_knn_trees over the first n_trees trees."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if idx is None:
            idx = torch.empty((self.n, K), dtype=torch.int32, device=dev)
        if dist is None:
            dist = torch.empty((self.n, K), dtype=torch.float32, device=dev)
        ws, wsb = (0, 0) if workspace is None else (_ptr(workspace), workspace.numel()
                                                     * workspace.element_size())
        if n_trees is None:
            check(_lib.lib().rpf_all_knn(self._h, K, _ptr(idx), _ptr(dist), ws or None, wsb,
                                         _stream_handle(stream)), "rpf_all_knn")
        else:
            check(_lib.lib().rpf_all_knn_trees(self._h, int(n_trees), K, _ptr(idx), _ptr(dist),
                                               ws or None, wsb, _stream_handle(stream)),
                  "rpf_all_knn_trees")
        return idx, dist

    def all_knn_async(self, K: int, idx, dist, workspace, stream=None):
        """rpf_all_knn_async: the lists of all_knn, only enqueued (nothing
        allocated, no synchronisation), so the call can be recorded into a
        CUDA graph.  idx (n x K int32), dist (n x K float32) and workspace
        (at least workspace_bytes(K) bytes) are caller-owned contiguous CUDA
        tensors, checked here before anything is launched;
        query_status(workspace) reports the outcome once the work is done."""
        _check_buffer("idx", idx, (self.n, K), torch.int32, self.device)
        _check_buffer("dist", dist, (self.n, K), torch.float32, self.device)
        if (not isinstance(workspace, torch.Tensor) or not workspace.is_cuda
                or not workspace.is_contiguous()):
            raise ValueError("workspace must be a contiguous CUDA tensor")
        wsb = workspace.numel() * workspace.element_size()
        if wsb < self.workspace_bytes(K):
            raise ValueError("workspace needs %d bytes, not %d" % (self.workspace_bytes(K), wsb))
        check(_lib.lib().rpf_all_knn_async(self._h, K, _ptr(idx), _ptr(dist), _ptr(workspace),
                                           wsb, _stream_handle(stream)), "rpf_all_knn_async")
        return idx, dist

    def all_knn_keys(self, K: int, keys=None, workspace=None, stream=None):
        """rpf_all_knn_keys: (n, K, 2) int32 pairs (d32 bits, index) per point."""
        if keys is None:
            keys = torch.empty((self.n, K, 2), dtype=torch.int32, device=self.device)
        else:
            _check_out("keys", keys, (self.n, K, 2), np.int32)
        ws, wsb = (0, 0) if workspace is None else (_ptr(workspace), workspace.numel()
                                                     * workspace.element_size())
        check(_lib.lib().rpf_all_knn_keys(self._h, K, _ptr(keys), ws or None, wsb,
                                          _stream_handle(stream)), "rpf_all_knn_keys")
        return keys

    def autotune(self, K: int, stream=None) -> dict:
        """rpf_autotune: time the leaf tiles' configurations on this forest
        (plain: tile region; chosen: tile rows, Gram chunk, CTAs per SM) and
        keep the fastest for forests of this shape."""
        chosen = (ctypes.c_int32 * 5)()
        check(_lib.lib().rpf_autotune(self._h, K, _stream_handle(stream), chosen),
              "rpf_autotune")
        return {"gram_chunk": chosen[0], "ctas_per_sm": chosen[1], "tile_rows": chosen[2],
                "tile_region": chosen[3],
                "query_scan": {1: "bf16", 0: "fp32", -1: None}[chosen[4]]}

    def set_form(self, form: int, stream=None) -> None:
        """rpf_set_form: switch between the plain and the chosen form."""
        check(_lib.lib().rpf_set_form(self._h, int(form), _stream_handle(stream)), "rpf_set_form")
        self.params.form = int(form)

    def set_query_scan(self, mode) -> None:
        """rpf_set_query_scan: the chosen form's query leaf scan; None = the
        autotuner's pick, "fp32" or "bf16"."""
        code = {None: -1, "fp32": 0, "bf16": 1}[mode]
        check(_lib.lib().rpf_set_query_scan(self._h, code), "rpf_set_query_scan")

    def add_trees(self, n_new: int, stream=None) -> None:
        """rpf_add_trees: grow n_new more trees (the same forest that a build
        with n_trees + n_new trees gives)."""
        check(_lib.lib().rpf_add_trees(self._h, int(n_new), _stream_handle(stream)),
              "rpf_add_trees")
        self.params.n_trees += int(n_new)

    def query(self, Q, K: int, idx=None, dist=None, workspace=None, stream=None):
        """rpf_query.  With a workspace and device outputs the call only
        enqueues the work; query_status(workspace) reports its outcome."""
        Q = _as_points(Q)
        m = int(Q.shape[0])
        if Q.shape[1] != self.d:
            raise ValueError("Q must have %d columns, not %d" % (self.d, Q.shape[1]))
        if idx is not None:
            _check_out("idx", idx, (m, K), np.int32)
        if dist is not None:
            _check_out("dist", dist, (m, K), np.float32)
        if workspace is not None and (not isinstance(workspace, torch.Tensor) or not
                                      workspace.is_cuda or not workspace.is_contiguous()):
            raise ValueError("workspace must be a contiguous CUDA tensor")
        on_dev = isinstance(Q, torch.Tensor) and Q.is_cuda
        if idx is None:
            idx = (torch.empty((m, K), dtype=torch.int32, device=Q.device) if on_dev
                   else np.empty((m, K), np.int32))
        if dist is None:
            dist = (torch.empty((m, K), dtype=torch.float32, device=Q.device) if on_dev
                    else np.empty((m, K), np.float32))
        ws, wsb = (0, 0) if workspace is None else (_ptr(workspace), workspace.numel()
                                                     * workspace.element_size())
        check(_lib.lib().rpf_query(self._h, _ptr(Q) if m else None, m, K,
                                   _ptr(idx) if m else None, _ptr(dist) if m else None,
                                   ws or None, wsb, _stream_handle(stream)), "rpf_query")
        return idx, dist

    def query_status(self, workspace=None, stream=None) -> None:
        """rpf_query_status: waits for the stream and raises if a bounded
        device wait of the last query or all_knn_async on `workspace` (None:
        the last query_static on this device) gave up."""
        check(_lib.lib().rpf_query_status(None if workspace is None else _ptr(workspace),
                                          _stream_handle(stream)), "rpf_query_status")

    def query_static(self, Q, K: int, idx, dist, stream=None):
        """rpf_query_static: the query with the library's fixed device scratch.

        Q, idx and dist are caller-owned contiguous CUDA tensors on the
        forest's device (checked here, before anything is launched); nothing
        is allocated.  Calls that may overlap in time share the scratch and
        must be serialised (one stream)."""
        m = _check_query_static(self.d, Q, K, idx, dist, self.device)
        check(_lib.lib().rpf_query_static(self._h, _ptr(Q) if m else None, m, K,
                                          _ptr(idx) if m else None, _ptr(dist) if m else None,
                                          _stream_handle(stream)), "rpf_query_static")
        return idx, dist

    # ---- inspection ------------------------------------------------------------
    def info(self) -> dict:
        n, d, T, nn, nl, md, ne = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(),
                                   ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(),
                                   ctypes.c_int64())
        check(_lib.lib().rpf_forest_info(self._h, *(ctypes.byref(v) for v in
                                                    (n, d, T, nn, nl, md, ne))), "info")
        return {"n": n.value, "d": d.value, "n_trees": T.value, "n_nodes": nn.value,
                "n_leaves": nl.value, "max_depth": md.value, "n_exact_nodes": ne.value}

    def counters(self) -> dict:
        out = np.zeros(5, np.int64)
        check(_lib.lib().rpf_forest_counters(self._h, out.ctypes.data, 5), "counters")
        return {"exact_nodes": int(out[0]), "bf16_fallback_rows": int(out[1]),
                "phase_a_levels": int(out[2]), "tile_region": int(out[3]),
                "chosen_form_plain_groups": int(out[4])}

    def perm(self, t: int) -> np.ndarray:
        out = np.empty(self.n, np.int32)
        check(_lib.lib().rpf_forest_perm(self._h, t, out.ctypes.data), "perm")
        return out

    def leaves(self):
        nl = self.info()["n_leaves"]
        tr, b, ln = (np.empty(nl, np.int32) for _ in range(3))
        check(_lib.lib().rpf_forest_leaves(self._h, tr.ctypes.data, b.ctypes.data,
                                           ln.ctypes.data), "leaves")
        return tr, b, ln

    def nodes(self) -> dict:
        nn = self.info()["n_nodes"]
        key = np.empty(nn, np.uint64)
        i32 = {k: np.empty(nn, np.int32) for k in ("tree", "begin", "len", "left", "right",
                                                    "jstar", "flag")}
        c = np.empty(nn, np.float64)
        check(_lib.lib().rpf_forest_nodes(self._h, key.ctypes.data, *(i32[k].ctypes.data for k in
                                          ("tree", "begin", "len", "left", "right", "jstar",
                                           "flag")), c.ctypes.data), "nodes")
        out = {"key": key, "c": c}
        out.update(i32)
        return out


def directions(seed: int, t: int, keys, j: int, d: int, stream=None) -> np.ndarray:
    """Candidate directions of Algorithm 2 for (tree t, node keys, try j), on the GPU."""
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.empty((keys.size, d), np.float64)
    check(_lib.lib().rpf_directions(seed, t, keys.ctypes.data, keys.size, j, d, out.ctypes.data,
                                    _stream_handle(stream)), "rpf_directions")
    return out


def brute_knn(X, Q, K: int, self_idx=None, stream=None):
    """Exact kNN of the rows of Q among X on the GPU (d32 key, index ties)."""
    X = _as_points(X)
    Q = _as_points(Q)
    m = int(Q.shape[0])
    on_dev = isinstance(Q, torch.Tensor) and Q.is_cuda
    if on_dev:
        idx = torch.empty((m, K), dtype=torch.int32, device=Q.device)
        dist = torch.empty((m, K), dtype=torch.float32, device=Q.device)
    else:
        idx, dist = np.empty((m, K), np.int32), np.empty((m, K), np.float32)
    sp = None
    if self_idx is not None:
        if isinstance(self_idx, np.ndarray):
            self_idx = np.ascontiguousarray(self_idx, np.int32)
        else:
            self_idx = self_idx.to(torch.int32).contiguous()
        sp = _ptr(self_idx)
    check(_lib.lib().rpf_brute_knn(_ptr(X), int(X.shape[0]), int(X.shape[1]),
                                   _ptr(Q) if m else None, m, sp, K,
                                   _ptr(idx) if m else None, _ptr(dist) if m else None,
                                   _stream_handle(stream)), "rpf_brute_knn")
    return idx, dist


def gather_rate(X, rows: int = 1 << 24, reps: int = 10, seed: int = 1) -> float:
    """rpf_gather_probe timed with CUDA events on the current stream: GB/s of
    random whole rows of the device matrix X (n x d FP32)."""
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32
            and X.is_contiguous() and X.dim() == 2):
        raise ValueError("X must be a contiguous 2-D float32 CUDA tensor")
    out = torch.zeros(1, dtype=torch.float32, device=X.device)
    s = torch.cuda.current_stream(X.device)
    L = _lib.lib()
    n, d = int(X.shape[0]), int(X.shape[1])
    for r in range(2):  # warm-up
        check(L.rpf_gather_probe(_ptr(X), n, d, rows, seed + r, _ptr(out), s.cuda_stream),
              "rpf_gather_probe")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for r in range(reps):
        check(L.rpf_gather_probe(_ptr(X), n, d, rows, seed + 2 + r, _ptr(out), s.cuda_stream),
              "rpf_gather_probe")
    e1.record(s)
    e1.synchronize()
    return rows * d * 4 / (e0.elapsed_time(e1) * 1e-3 / reps) / 1e9


def merge_keys(lists, K: int, idx=None, dist=None, stream=None):
    """rpf_merge_keys: lists (G, n, K, 2) int32 (d32 bits, index) -> final
    (idx, dist) of the n points (the union over the G groups of trees)."""
    if lists.dim() != 4 or lists.shape[2] != K or lists.shape[3] != 2:
        raise ValueError("lists must have shape (G, n, K, 2)")
    lists = lists.contiguous()
    G, n = int(lists.shape[0]), int(lists.shape[1])
    dev = lists.device
    if idx is None:
        idx = torch.empty((n, K), dtype=torch.int32, device=dev)
    if dist is None:
        dist = torch.empty((n, K), dtype=torch.float32, device=dev)
    _check_out("idx", idx, (n, K), np.int32)
    _check_out("dist", dist, (n, K), np.float32)
    check(_lib.lib().rpf_merge_keys(n, K, G, _ptr(lists) if n else None, _ptr(idx) if n else None,
                                    _ptr(dist) if n else None, _stream_handle(stream)),
          "rpf_merge_keys")
    return idx, dist


def set_wait_limit(limit_ns: int = 0) -> None:
    """rpf_set_wait_limit: time limit of every bounded device wait (0: 2 s)."""
    _lib.lib().rpf_set_wait_limit(int(limit_ns))


def wait_selftest(limit_ns: int, stream=None) -> int:
    """rpf_wait_selftest: return code of one bounded wait that nothing completes."""
    return int(_lib.lib().rpf_wait_selftest(int(limit_ns), _stream_handle(stream)))


def debug_fail_alloc(after: int) -> None:
    """rpf_debug_fail_alloc: the allocation after `after` more succeed fails (-1: off)."""
    _lib.lib().rpf_debug_fail_alloc(int(after))


class Trace:
    """Per-kernel CUDA-event timing of the library's launches (rpf_trace_*)."""

    @staticmethod
    def enable(on: bool = True):
        _lib.lib().rpf_trace_enable(1 if on else 0)

    @staticmethod
    def launch_count() -> int:
        return int(_lib.lib().rpf_launch_count())

    @staticmethod
    def read() -> dict:
        cap = 256
        names = ctypes.create_string_buffer(48 * cap)
        launches = np.zeros(cap, np.int64)
        ms = np.zeros(cap, np.float64)
        k = ctypes.c_int32()
        check(_lib.lib().rpf_trace_read(cap, names, launches.ctypes.data, ms.ctypes.data,
                                        ctypes.byref(k)), "rpf_trace_read")
        out = {}
        for i in range(min(k.value, cap)):
            nm = names.raw[48 * i:48 * i + 48].split(b"\0", 1)[0].decode()
            if launches[i]:
                out[nm] = {"launches": int(launches[i]), "ms": float(ms[i])}
        return out
