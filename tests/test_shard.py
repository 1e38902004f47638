"""Tree-sharded all-kNN: a forest split by tree over G ranks, one exchange
of per-point (d32, index) lists by point ownership, and a merge per point,
equals the single forest's all-kNN bit for bit.

CPU: gloo ranks (world size 2 and 3), the lists of every rank's trees from
the oracle grown on that tree range, merged by the oracle's union of lists
-- the exchange and ownership logic of the product module under test.
GPU: the CUDA path on one device, ranks simulated in turn (rpf_build_shard,
rpf_all_knn_keys, rpf_merge_keys), against rpf_all_knn of the whole forest.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1812_11689_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_tree_and_point_ranges_cover_everything_once():
    from paper_1812_11689_gb300 import shard
    for T in (1, 2, 5, 40, 96):
        for world in (1, 2, 3, 8):
            got = [shard.tree_range(T, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == T
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1
    for n in (1, 7, 2000):
        for world in (1, 2, 3):
            pr = shard.point_ranges(n, world)
            assert pr[0][0] == 0 and pr[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(pr, pr[1:]))


def _rank_main(rank, world, port, T, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1812_11689_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = synth.make("mix5_d10")
    K = 5

    def local_keys(t0, nt):
        f = oracle.Forest(X, nt, 50, 5, seed=0, threads=1, tree_first=t0)
        i, d32 = f.all_knn_keys(K)
        return shard.keys_from_lists(i, d32)

    def merge(lists):
        L = lists.numpy()
        idx_l = [L[g, :, :, 1] for g in range(L.shape[0])]
        d32_l = [L[g, :, :, 0].view(np.float32) for g in range(L.shape[0])]
        return oracle.merge_key_lists(idx_l, d32_l, K)

    lo, hi, idx, dist_ = shard.run_sharded(X.shape[0], K, T, local_keys, merge,
                                           torch.device("cpu"))
    q.put((rank, lo, hi, idx, dist_))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,T", [(2, 10), (3, 5), (2, 1)])
def test_sharded_lists_equal_the_single_forest_on_gloo_ranks(world, T):
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, T, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    X = synth.make("mix5_d10")
    oi, od = oracle.Forest(X, T, 50, 5, seed=0).all_knn(5)
    seen = np.zeros(X.shape[0], bool)
    for rank, lo, hi, idx, dist_ in got:
        assert np.array_equal(idx, oi[lo:hi]) and np.array_equal(dist_, od[lo:hi]), rank
        seen[lo:hi] = True
    assert seen.all()


def test_oracle_tree_ranges_are_the_forest_trees_and_lists_merge_to_it():
    # the oracle restatement the gloo test leans on: trees grown from index
    # t0 are the whole forest's trees t0.., and merging the groups' squared-
    # key lists gives the whole forest's lists
    import oracle
    X = synth.make("mix5_d10", n=900)
    F = oracle.Forest(X, 7, 30, 3, seed=2)
    parts = [oracle.Forest(X, 3, 30, 3, seed=2), oracle.Forest(X, 4, 30, 3, seed=2, tree_first=3)]
    for t in range(7):
        src, tt = (parts[0], t) if t < 3 else (parts[1], t - 3)
        assert np.array_equal(F.perm(t), src.perm(tt))
    i, d = F.all_knn(6)
    lists = [p.all_knn_keys(6) for p in parts]
    mi, md = oracle.merge_key_lists([l[0] for l in lists], [l[1] for l in lists], 6)
    assert np.array_equal(mi, i) and np.array_equal(md, d)
    ki, kd = F.all_knn_keys(6)
    assert np.array_equal(ki, i) and np.array_equal(np.sqrt(kd), d)


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1])
def test_shards_on_one_gpu_merge_to_the_single_forest(form):
    import torch
    import oracle
    from paper_1812_11689_gb300 import forest, shard
    from _parity import compare_trees
    X = synth.make("aniso20_d64", n=20000)
    Xd = torch.from_numpy(X).cuda()
    T, K, G = 10, 10, 3
    full = forest.Forest(Xd, n_trees=T, leaf_max=128, n_try=5, form=form)
    fi, fd = full.all_knn(K)
    keys = []
    for r in range(G):
        t0, t1 = shard.tree_range(T, G, r)
        f = forest.Forest(Xd, n_trees=t1 - t0, leaf_max=128, n_try=5, form=form, tree_first=t0)
        if r == 1:  # the shard's trees are the oracle's trees t0 .. t1 - 1
            compare_trees(f, oracle.Forest(X, t1 - t0, 128, 5, tree_first=t0), t1 - t0)
        keys.append(f.all_knn_keys(K))
        f.close()
    for q, (lo, hi) in enumerate(shard.point_ranges(X.shape[0], G)):
        lists = torch.stack([k[lo:hi] for k in keys])
        mi, md = forest.merge_keys(lists, K)
        assert torch.equal(mi, fi[lo:hi]) and torch.equal(md, fd[lo:hi]), q
    # the keys of the whole forest are its lists before the square root
    kk = full.all_knn_keys(K)
    assert torch.equal(kk[..., 1], fi)
    d32 = np.ascontiguousarray(kk[..., 0].cpu().numpy()).view(np.float32)
    assert np.array_equal(np.sqrt(d32), fd.cpu().numpy())
    full.close()
