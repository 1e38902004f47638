"""Host-side pieces of the benchmark that need no GPU: the per-point missing
counts (Sec. 5.1) against the oracle's definition, and the oracle step that
both the CPU baseline and the reference arm time."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_missing_counts_follow_the_missing_rate_definition():
    import bench
    import oracle
    rng = np.random.default_rng(0)
    true = rng.integers(0, 50, size=(200, 6)).astype(np.int32)
    for i in range(200):  # distinct true neighbours per row, some padded
        true[i] = rng.permutation(50)[:6]
    true[:10, 4:] = -1
    found = true.copy()
    flip = rng.random(found.shape) < 0.3
    found[flip] = rng.integers(50, 100, size=flip.sum())
    found[5, :] = -1
    m = bench.missing_counts(found, true)
    assert m.shape == (200,)
    assert m.sum() / true.size == oracle.missing_rate(found, true)
    assert m[5] == (true[5] >= 0).sum()


def test_oracle_step_times_every_tree_and_scales_the_answers_only():
    import bench
    from paper_1812_11689_gb300 import synth
    w = synth.WORKLOADS["mix5_d10"]
    X = synth.make("mix5_d10")
    full = bench.oracle_step(X, w, 4, 2, rows_fraction=1.0)
    part = bench.oracle_step(X, w, 4, 2, rows_fraction=0.25)
    for r in (full, part):
        assert r["kind"] == "oracle" and r["cores"] == 2 and r["n_trees"] == 4
        assert r["value"] > 0
        # value = n / (growth + scaled answering); the seconds are rounded to 1 ms
        assert abs(X.shape[0] / r["value"] - r["full_workload_seconds"]) <= 6e-4
    assert "all 4 trees" in part["sample"] and "500 sampled points" in part["sample"]
    st = bench.oracle_single_thread(X, w, 4, trees=2, rows=200)
    assert st["cores"] == 1 and st["value"] > 0
