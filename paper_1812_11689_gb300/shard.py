"""Tree-sharded all-kNN over several processes, one GPU each.

The trees of Algorithm 3 are independent (Sec. 2; the paper grows them on
separate cores, Sec. 5.3), so a forest of T trees splits by tree.  Rank r of
G grows trees [r T / G, (r + 1) T / G) over all n points (rpf_build_shard:
every draw is keyed by the global tree index, so these are the trees one
process would grow at those indexes) and computes, for every point, its K
nearest in the union of its leaves over those trees, as (d32, index) pairs
(rpf_all_knn_keys).  One exchange follows.  Rank q owns the points
[q n / G, (q + 1) n / G); an all-to-all sends every rank the lists of the
points it owns from every rank, and merging those G lists per point
(rpf_merge_keys) gives exactly the single forest's answer: a point in the K
nearest of the whole union is in the K nearest of every group's union that
contains it.  The pairs carry the FP32 squared distance itself, so the merge
orders exactly as the single forest does.

`run_sharded` holds the host steps with the two compute steps passed in;
`sharded_all_knn` supplies the CUDA library's.  On GPUs the exchange is one
NCCL all-to-all of n K 8 bytes per rank.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

EMPTY_D32_BITS = 0x7F800000  # +inf: an empty slot of a list


def tree_range(T: int, world: int, rank: int):
    """Trees [lo, hi) of rank `rank` in a balanced split of T trees."""
    base, extra = divmod(T, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def point_ranges(n: int, world: int):
    """Points [lo, hi) owned by each rank."""
    return [(q * n // world, (q + 1) * n // world) for q in range(world)]


def empty_keys(n: int, K: int, device) -> torch.Tensor:
    keys = torch.empty((n, K, 2), dtype=torch.int32, device=device)
    keys[..., 0] = EMPTY_D32_BITS
    keys[..., 1] = -1
    return keys


def exchange(keys: torch.Tensor, world: int, rank: int, group=None) -> torch.Tensor:
    """All-to-all of the (n, K, 2) lists: returns (world, n_r, K, 2), the
    lists of this rank's points from every rank, in rank order."""
    n, K = int(keys.shape[0]), int(keys.shape[1])
    rng = point_ranges(n, world)
    lo, hi = rng[rank]
    inp = keys.reshape(n, 2 * K).contiguous()
    out = torch.empty((world * (hi - lo), 2 * K), dtype=keys.dtype, device=keys.device)
    dist.all_to_all_single(out, inp, output_split_sizes=[hi - lo] * world,
                           input_split_sizes=[h - l for l, h in rng], group=group)
    return out.view(world, hi - lo, K, 2)


def run_sharded(n: int, K: int, T: int, local_keys, merge, device, group=None):
    """Host steps of the sharded all-kNN on this rank.

    local_keys(tree_first, n_trees) -> (n, K, 2) int32 lists of those trees;
    merge(lists (G, n_r, K, 2)) -> (idx, dist) of this rank's points.
    Returns (lo, hi, idx, dist)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    t0, t1 = tree_range(T, world, rank)
    keys = local_keys(t0, t1 - t0) if t1 > t0 else empty_keys(n, K, device)
    recv = exchange(keys, world, rank, group)
    lo, hi = point_ranges(n, world)[rank]
    idx, dist_ = merge(recv)
    return lo, hi, idx, dist_


def sharded_all_knn(X: torch.Tensor, K: int, n_trees: int, leaf_max: int, n_try: int = 5,
                    form: int = 1, seed: int = 0, split_rule: int = 0, group=None):
    """All-kNN of a forest of n_trees trees split by tree over the ranks of
    `group` (one GPU each, X resident on every rank).  Returns this rank's
    (lo, hi, idx, dist): the lists of points lo .. hi - 1."""
    from . import forest

    n = int(X.shape[0])

    def local_keys(t0, nt):
        f = forest.Forest(X, n_trees=nt, leaf_max=leaf_max, n_try=n_try, form=form, seed=seed,
                          split_rule=split_rule, tree_first=t0)
        try:
            return f.all_knn_keys(K)
        finally:
            f.close()

    def merge(lists):
        return forest.merge_keys(lists, K)

    return run_sharded(n, K, n_trees, local_keys, merge, X.device, group)


def keys_from_lists(idx: np.ndarray, d32: np.ndarray) -> torch.Tensor:
    """(n, K, 2) int32 pairs from an index list and an FP32 squared-distance
    list (the rpf_all_knn_keys layout)."""
    return torch.from_numpy(np.stack([np.ascontiguousarray(d32, np.float32).view(np.int32),
                                      np.ascontiguousarray(idx, np.int32)], axis=-1))
