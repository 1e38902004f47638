#!/usr/bin/env python
"""All-kNN throughput of the GB300 rpForests library (one JSON line).

A step is one pass of the whole hot path over one synthetic data set: grow T
random projection trees (rpf_build) and answer all-kNN for every point
(rpf_all_knn).  value = points answered per second (n / step time), inputs
resident in HBM, L2 flushed between steps.  e2e = the same through the C ABI
with host buffers (pinned X in, pinned idx/dist out, copies inside the timed
region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the plain C restatement of the paper's
algorithms) on the host cores, on a bounded sample of the same workload, and
scales it to the full workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="aniso20_d64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large batched workload (1M points, d = 128, T = 64)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the ensemble sweep (128 nested trees, heavy-tailed data)")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving measurement (resident 2M-point forest)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-step", action="store_true",
                    help="one warm-up step and one step of the chosen form at the operating "
                         "point, nothing else (the command the ncu summaries under profiles/ "
                         "are taken from)")
    ap.add_argument("--profile-trees", type=int, default=0,
                    help="tree count of --profile-step (default: the operating point)")
    return ap.parse_args()


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            j = json.load(open(p))
            for k in ("bf16_tflops", "bf16_TFLOPs"):
                if k in j:
                    return float(j[k]), "measured"
        except Exception:
            pass
    return BF16_TFLOPS


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            j = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_bandwidth_gbs"):
                if k in j:
                    return float(j[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline of the GPU arm and every step of --impl reference)
# ---------------------------------------------------------------------------
ORACLE_ROWS_FRACTION = 0.25   # share of the points whose all-kNN lists one step answers


def oracle_step(X, w, n_trees, threads, rows_fraction=ORACLE_ROWS_FRACTION, seed=0):
    """One timed pass of the oracle over the workload: all n_trees trees grown
    on all n points (one tree per thread, the paper's multicore scheme), then
    the all-kNN lists of a seeded sample of the points over those trees.  The
    trees are not sampled; the answering time is scaled by n / rows (every
    point's answer is independent work, spread over the threads dynamically).
    Returns the throughput of the whole job (build + all n answers)."""
    import oracle
    oracle.build()
    n = X.shape[0]
    nr = n if rows_fraction >= 1.0 else max(1, int(n * rows_fraction))
    rows = np.sort(np.random.default_rng(seed).choice(n, size=nr, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    F = oracle.Forest(X, n_trees, w.leaf_max, w.n_try, seed=seed, threads=threads)
    t_grow = time.perf_counter() - t0
    t0 = time.perf_counter()
    if nr == n:
        F.all_knn(w.k)
    else:
        F.all_knn_rows(rows, w.k)
    t_rows = time.perf_counter() - t0
    del F
    t_full = t_grow + t_rows * (n / nr)
    sample = ("all %d trees grown on all %d points with %d threads; all-kNN answered for %d "
              "sampled points (%.0f %%) over those trees, the answering time scaled by n / rows"
              % (n_trees, n, threads, nr, 100.0 * nr / n))
    return {"value": n / t_full, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": sample, "n_trees": n_trees, "step_seconds": round(t_grow + t_rows, 3),
            "grow_seconds": round(t_grow, 3), "answer_seconds": round(t_rows, 3),
            "full_workload_seconds": round(t_full, 3)}


def oracle_single_thread(X, w, n_trees, seed=0, trees=2, rows=2000):
    """The oracle on one thread, on a stated sample: `trees` trees grown on all
    points and the all-kNN lists of `rows` sampled points over them, scaled by
    trees (growth and answering both grow linearly with the tree count) and
    by rows."""
    import oracle
    oracle.build()
    n = X.shape[0]
    r = np.sort(np.random.default_rng(seed).choice(n, size=rows, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    F = oracle.Forest(X, trees, w.leaf_max, w.n_try, seed=seed, threads=1)
    t_grow = time.perf_counter() - t0
    t0 = time.perf_counter()
    F.all_knn_rows(r, w.k)
    t_rows = time.perf_counter() - t0
    t_full = (t_grow + t_rows * (n / rows)) * (n_trees / trees)
    return {"value": n / t_full, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": "%d trees grown on all %d points and all-kNN for %d sampled points over "
                      "them, one thread; scaled by trees (to %d) and by n / rows"
                      % (trees, n, rows, n_trees),
            "sample_seconds": round(t_grow + t_rows, 3)}


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


SUBTREE_MAX = 4096          # nodes of at most this many points grow CTA-locally
TC_BIG_MIN = 12             # leaves of at least this many points take the tensor path


def small_subtree_max(L, median):
    """Largest subtree the library grows with one warp per CTA (k_subtree_w):
    above the leaf bound, at most 1024 points, 1024 under the median rule."""
    m = 1024 if median else (max(512, 2 * L) + 15) // 16 * 16
    return 0 if (m > 1024 or m <= L) else m
T_GRID = (40, 48, 56, 64, 72, 80, 88, 96, 104, 112, 120, 128)  # nested ensembles swept
FP32_LANES = 152 * 128      # FP32 lanes of a GB300 (152 SMs x 128)
BF16_TFLOPS = (1900.0, "fallback (dense BF16, one earlier GB300 measurement)")
SM_MAX_GHZ = 2.07


def replica_value(total_ms, n, steps, world, device):
    """Whole-job throughput of `world` independent replicas (weak scaling):
    each rank answered n points per step; the job's time is the slowest
    rank's (max over ranks).  Returns (ms per step, points per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / steps
    return ms_step, world * n / (ms_step * 1e-3)


def discrepancy_full(found_d, true_d):
    """kNN-distance discrepancy of Sec. 5.1 at k = K: relative gap of the mean
    K-th distance found to the mean true K-th distance, over the points whose
    found and true lists are both full; also returns how many were not."""
    fk = found_d[:, -1].astype(np.float64)
    tk = true_d[:, -1].astype(np.float64)
    ok = np.isfinite(fk) & np.isfinite(tk)
    if not ok.any():
        return None, int((~ok).sum())
    mt = tk[ok].mean()
    return round(float((fk[ok].mean() - mt) / mt), 6), int((~ok).sum())


def work_model(fo, w, n):
    """Algorithmic bytes (and FLOPs) per step of each main kernel.

    Growth: every point of an internal node is projected once per level; its
    X row (4d B) is the minimum read.  Phase A (nodes > 4096 points) also
    reads perm and the point norm and writes nTry FP32 projections; phase B
    reads perm and writes the final permutation once per subtree (the
    four-warp kernel writes back the segments it hands to the one-warp one).  Leaf
    tiles: every point's row once per tree plus its perm entry and its
    per-tree top-K list (8K B); FLOPs 2 d m^2 per leaf of m points.  Merge:
    T per-tree lists in, the final list out.
    """
    nd = fo.nodes()
    ln = nd["len"].astype(np.int64)
    internal = nd["left"] >= 0
    A = internal & (ln > SUBTREE_MAX)
    B = internal & (ln <= SUBTREE_MAX)
    Sw = small_subtree_max(w.leaf_max, fo.params.split_rule == 1)
    Bw = B & (ln <= Sw)  # grown by the one-warp kernel
    Bb = B & ~Bw
    # subtree roots: the perm segment is read once and written once (final
    # permutation, or handed over to the one-warp kernel)
    par = np.full(len(ln), SUBTREE_MAX + 1, np.int64)
    for side in ("left", "right"):
        ch = nd[side][internal]
        ok = ch >= 0
        par[ch[ok]] = ln[internal][ok]
    handed = Bw & (par > Sw) & (par <= SUBTREE_MAX)
    rb = 8 * int(ln[Bb & (par > SUBTREE_MAX)].sum()) + 4 * int(ln[handed].sum())
    rw = 8 * int(ln[Bw & (par > Sw)].sum())
    pl_a, pl_b = int(ln[A].sum()), int(ln[B].sum())
    pl_bb, pl_bw = int(ln[Bb].sum()), int(ln[Bw].sum())
    leaf_len = ln[~internal]
    d, T, K, nt = w.d, fo.info()["n_trees"], w.k, w.n_try
    return {
        "k_subtree": {"bytes": pl_bb * (4 * d + 4) + rb},
        "k_subtree_w": {"bytes": pl_bw * (4 * d + 4) + rw},
        "k_proj_a": {"bytes": pl_a * (4 * d + 4 + 4 + 4 * nt), "units": pl_a},
        "k_side_count": {"bytes": pl_a * (4 + 4 + 1)},
        "k_scatter": {"bytes": pl_a * (1 + 4 + 4)},
        "k_leaf_plain": {"bytes": n * T * (4 * d + 4 + 8 * K),
                         "flops": 2 * d * int((leaf_len ** 2).sum())},
        "k_leaf_tc": {"bytes": n * T * (4 * d + 4 + 8 * K),
                      "flops": 2 * d * int((leaf_len ** 2).sum()),
                      "tensor_flops": 3 * 2 * ((d + 15) // 16 * 16)
                      * int((leaf_len[(leaf_len >= TC_BIG_MIN) & (leaf_len > K + 1)] ** 2).sum())},
        "k_merge": {"bytes": n * (T * 8 * K + 8 * K)},
        "_point_levels": {"phase_a": pl_a, "phase_b": pl_b, "phase_b_one_warp": pl_bw,
                          "leaf_m2_per_point_per_tree": float((leaf_len ** 2).sum()) / (n * T)},
    }


def traffic_record(kernel, workload, units_per_launch=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of the kernel (the summary states the source digest).
    A summary of one launch of a kernel whose launches differ in size states
    the units (point-levels) of the captured launch; its bytes are scaled to
    units_per_launch."""
    import hashlib
    import re
    p = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", txt)
    src = re.search(r"source_sha256:\s*([0-9a-f]+)\s+files:\s*(.+)", txt)
    if not m or not src:
        return None
    h = hashlib.sha256()
    for f in src.group(2).split():
        f = os.path.join(ROOT, f)
        if not os.path.exists(f):
            return None
        h.update(open(f, "rb").read())
    if h.hexdigest() != src.group(1):
        return None
    u = re.search(r"captured_units:\s*([0-9]+)", txt)
    if u and units_per_launch:
        return int(int(m.group(1)) * units_per_launch / int(u.group(1)))
    return int(m.group(1))


GROWTH_KERNELS = ("k_proj_a", "k_subtree", "k_subtree_w")


def rooflines(trace, work, hbm_peak, peak_kind, steps, workload, gather_peak=None):
    """Per-kernel roofline fractions; the kernel with the largest share first."""
    tot = sum(v["ms"] for v in trace.values()) or 1.0
    fp32_peak = 2 * FP32_LANES * SM_MAX_GHZ * 1e9 / 1e12  # TFLOP/s, FMA = 2
    out = []
    for k, t in sorted(trace.items(), key=lambda kv: -kv[1]["ms"]):
        if k not in work or t["launches"] == 0:
            continue
        ms_launch = t["ms"] / t["launches"]
        per_launch = work[k]["bytes"] * steps / t["launches"]
        ach = per_launch / (ms_launch * 1e-3) / 1e9
        r = {"kernel": k, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
             "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
             "peak_source": peak_kind,
             "traffic": traffic_record(k, workload, work[k].get("units", 0) * steps / t["launches"]),
             "algorithmic_bytes_per_launch": int(per_launch),
             "ms_per_launch": round(ms_launch, 5), "launches_per_step": t["launches"] // steps,
             "share": round(t["ms"] / tot, 4)}
        if gather_peak and k in GROWTH_KERNELS:
            # the growth kernels read X from L2: their own ceiling is the
            # rate of random whole-row reads (rpf_gather_probe, this run)
            r["l2_row_gather"] = {"achieved": round(ach, 1), "peak": gather_peak, "unit": "GB/s",
                                  "frac": round(ach / gather_peak, 4),
                                  "peak_source": "rpf_gather_probe on the workload's matrix, "
                                                 "timed in this run"}
        if "tensor_flops" in work[k]:
            tf = work[k]["tensor_flops"] * steps / t["launches"] / (ms_launch * 1e-3) / 1e12
            bp, bsrc = bf16_peak()
            r["tensor_bf16"] = {"achieved": round(tf, 2), "peak": bp,
                                "unit": "TFLOP/s", "frac": round(tf / bp, 5),
                                "peak_source": bsrc,
                                "flops": "3 BF16 products (split hi/lo) x 2 d16 m^2 per "
                                         "leaf of at least 12 points and more than K + 1"}
        if "flops" in work[k]:
            fl = work[k]["flops"] * steps / t["launches"] / (ms_launch * 1e-3) / 1e12
            r["fp32_alu"] = {"achieved": round(fl, 2), "peak": round(fp32_peak, 1),
                             "unit": "TFLOP/s", "frac": round(fl / fp32_peak, 4),
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
        out.append(r)
    return out


def missing_counts(found, true):
    """m(i) = |trueK(i) minus found(i)| for every row (Sec. 5.1), as index
    sets; -1 pads of the true lists are not neighbours, -1 pads of the found
    lists match nothing."""
    hit = (true[:, :, None] == found[:, None, :]).any(-1)
    return ((~hit) & (true >= 0)).sum(1)


def nested_sweep(forest_mod, Xd, w, rule, bi, bd, form, seed):
    """One forest of max(T_GRID) trees under split rule `rule`; all-kNN over
    its first T trees (the T-tree forest: nested ensembles) for every T of
    the grid, with the missing rate and distance discrepancy over all n
    points against exact brute force.  Returns the sweep and the smallest T
    whose missing rate is at most 1 %."""
    f = forest_mod.Forest(Xd, n_trees=max(T_GRID), leaf_max=w.leaf_max, n_try=w.n_try,
                          seed=seed, form=form, split_rule=rule)
    sweep, t_op = [], None
    for T in T_GRID:
        i, d = f.all_knn(w.k, n_trees=T)
        m = float(missing_counts(i.cpu().numpy(), bi).sum()) / bi.size
        sweep.append({"n_trees": T, "missing_rate": round(m, 6),
                      "knn_distance_discrepancy": discrepancy_full(d.cpu().numpy(), bd)[0]})
        if t_op is None and m <= 0.01:
            t_op = T
    f.close()
    return sweep, t_op


def run_gb300(args, rank, world, local_rank):
    import torch
    from paper_1812_11689_gb300 import forest, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.WORKLOADS[args.workload]
    X = synth.make(args.workload, seed=args.seed + rank)
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    chosen, plain = forest.FORM_CHOSEN, forest.FORM_PLAIN

    # ground truth over all n points: exact brute force (d32 order, self excluded)
    allrows = torch.arange(n, dtype=torch.int32, device=dev)
    bi, bd = forest.brute_knn(Xd, Xd, w.k, self_idx=allrows)
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()

    # the metric's operating point: the smallest nested T whose all-kNN lists
    # miss at most 1 % of the true neighbours, under Algorithm 1's uniform
    # split point (exact over all n points)
    sweep_u, t_op = nested_sweep(forest, Xd, w, forest.SPLIT_UNIFORM, bi, bd, chosen, args.seed)
    stated = w.extra.get("n_trees_le_1pct")
    verified = t_op is not None and t_op == stated
    if t_op is None:
        t_op = max(T_GRID)
    if world > 1:  # every replica times the same T: the largest any rank needs
        t = torch.tensor([t_op], dtype=torch.int64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_op = int(t.item())
    kw = dict(n_trees=t_op, leaf_max=w.leaf_max, n_try=w.n_try, seed=args.seed)
    ws = {}

    def step(form, kwt=None):
        f = forest.Forest(Xd, form=form, **(kwt or kw))
        if (form, f.params.n_trees) not in ws:
            ws[(form, f.params.n_trees)] = torch.empty(f.workspace_bytes(w.k), dtype=torch.uint8,
                                                       device=dev)
        out = f.all_knn(w.k, workspace=ws[(form, f.params.n_trees)])
        return f, out

    def timed(form, K, kwt=None):
        kwt = kwt or kw
        wst = ws[(form, kwt["n_trees"])]
        times, b_ms, a_ms = [], [], []
        for _ in range(K):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            f = forest.Forest(Xd, form=form, **kwt)
            e1.record(stream)
            f.all_knn(w.k, workspace=wst)
            e2.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e2))
            b_ms.append(e0.elapsed_time(e1))
            a_ms.append(e1.elapsed_time(e2))
            f.close()
        return times, b_ms, a_ms

    tuned = None
    for _ in range(args.warmup):
        for form in (chosen, plain):
            f, _ = step(form)
            if form == chosen and tuned is None:  # once: later forests reuse the choice
                tuned = f.autotune(w.k)
            f.close()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    l0 = forest.Trace.launch_count()
    times, b_ms, a_ms = timed(chosen, args.steps)
    l1 = forest.Trace.launch_count()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    # per-kernel CUDA-event times: the same steps again, traced (event pairs
    # around every launch), outside the timed region above
    forest.Trace.read()
    forest.Trace.enable(True)
    timed(chosen, args.steps)
    forest.Trace.enable(False)
    trace = forest.Trace.read()
    ms_step, value = replica_value(sum(times), n, args.steps, world, dev)

    # plain FP32 form at the same T
    p_times, p_b, p_a = timed(plain, args.steps)
    forest.Trace.read()
    forest.Trace.enable(True)
    timed(plain, args.steps)
    forest.Trace.enable(False)
    trace_p = forest.Trace.read()
    p_ms = sum(p_times) / len(p_times)

    # end to end through the C ABI with host buffers
    Xh = torch.from_numpy(X).pin_memory()
    ih = torch.empty((n, w.k), dtype=torch.int32).pin_memory()
    dh = torch.empty((n, w.k), dtype=torch.float32).pin_memory()
    e2e_t = []
    for it in range(args.steps + 1):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = forest.Forest(Xh, form=chosen, **kw)
        f.all_knn(w.k, idx=ih, dist=dh, workspace=ws[(chosen, t_op)])
        torch.cuda.synchronize()
        if it:
            e2e_t.append(time.perf_counter() - t0)
        f.close()
    e2e_s = sum(e2e_t) / len(e2e_t)

    # accuracy at the operating point: chosen == plain bit for bit; missing
    # rate and discrepancy over all n points
    fc, (ci, cd) = step(chosen)
    fp, (pi, pd) = step(plain)
    same = bool(torch.equal(ci, pi) and torch.equal(cd, pd))
    ci_h, cd_h = ci.cpu().numpy(), cd.cpu().numpy()
    miss = float(missing_counts(ci_h, bi).sum()) / bi.size
    disc, short = discrepancy_full(cd_h, bd)
    rel = None
    ok = ci_h >= 0
    if ok.any():  # reported distances against FP64 on a sample of rows
        r = np.random.default_rng(1).choice(n, 2000, replace=False)
        ii, dd, oo = ci_h[r], cd_h[r], ok[r]
        xi = X[np.repeat(r, w.k).reshape(-1, w.k)[oo]].astype(np.float64)
        xj = X[ii[oo]].astype(np.float64)
        d64 = np.sqrt(((xi - xj) ** 2).sum(1))
        rel = float((np.abs(dd[oo].astype(np.float64) - d64) / np.maximum(d64, 1e-30)).max())
    info = fc.info()

    # the configured T (fewer trees, higher missing rate), timed the same way
    kw_c = dict(kw, n_trees=w.n_trees)
    for form in (chosen, plain):
        f, _ = step(form, kw_c)
        f.close()
    c_t, c_b, c_a = timed(chosen, args.steps, kw_c)
    cp_t, _, _ = timed(plain, args.steps, kw_c)
    at_cfg = {"n_trees": w.n_trees,
              "missing_rate": next(x["missing_rate"] for x in sweep_u if x["n_trees"] == w.n_trees),
              "value": round(world * n / (sum(c_t) / len(c_t) * 1e-3), 1),
              "ms_per_step": round(sum(c_t) / len(c_t), 3),
              "stage_ms": {"build": round(sum(c_b) / len(c_b), 3),
                           "all_knn": round(sum(c_a) / len(c_a), 3)},
              "plain_value": round(world * n / (sum(cp_t) / len(cp_t) * 1e-3), 1)}

    # the median split rule (the paper's other usual split point) at its own
    # operating point
    med = None
    if not args.no_sweep:
        sweep_m, t_m = nested_sweep(forest, Xd, w, forest.SPLIT_MEDIAN, bi, bd, chosen, args.seed)
        med = {"sweep": sweep_m, "n_trees": t_m}
        if t_m is not None:
            kw_m = dict(kw, n_trees=t_m, split_rule=forest.SPLIT_MEDIAN)
            for form in (chosen, plain):
                f, _ = step(form, kw_m)
                f.close()
            m_t, m_b, m_a = timed(chosen, args.steps, kw_m)
            mp_t, _, _ = timed(plain, args.steps, kw_m)
            med.update({"value": round(world * n / (sum(m_t) / len(m_t) * 1e-3), 1),
                        "ms_per_step": round(sum(m_t) / len(m_t), 3),
                        "stage_ms": {"build": round(sum(m_b) / len(m_b), 3),
                                     "all_knn": round(sum(m_a) / len(m_a), 3)},
                        "plain_value": round(world * n / (sum(mp_t) / len(mp_t) * 1e-3), 1)})

    hbm_peak, peak_kind = peaks()
    work = work_model(fc, w, n)
    gpk = round(forest.gather_rate(Xd), 1)
    roofs = rooflines(trace, work, hbm_peak, peak_kind, args.steps, args.workload, gpk)
    roofs_p = rooflines(trace_p, work, hbm_peak, peak_kind, args.steps, args.workload, gpk)
    roof = None
    if roofs:
        top = roofs[0]
        roof = {k: top[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
        roof.update({"kernel": top["kernel"], "share": top["share"], "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": top["algorithmic_bytes_per_launch"],
                     "ms_per_launch": top["ms_per_launch"]})
        for k in ("l2_row_gather", "fp32_alu", "tensor_bf16"):
            if k in top:
                roof[k] = top[k]
    fc.close()
    fp.close()

    line = {
        "metric": "all-kNN queries/s at <=1% missing rate (chosen vs plain FP32 form)",
        "value": round(value, 1),
        "unit": "queries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "precision": "split decisions with FP64 semantics (certified FP32, FP64 fallback); "
                     "distances FP32 (canonical d32 key), BF16 tensor-core shortlist re-ranked "
                     "exactly",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "d": d, "n_trees": t_op,
                   "leaf_max": w.leaf_max, "k": w.k, "n_try": w.n_try, "split_rule": "uniform",
                   "form": "chosen",
                   "n_trees_rule": "smallest T of %s with missing rate <= 1 %% (nested "
                                   "ensembles, exact over all n points)" % (list(T_GRID),),
                   "configured_n_trees": w.n_trees,
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "missing_rate": round(miss, 6),
        "knn_distance_discrepancy": disc,
        "points_with_short_lists": short,
        "max_rel_distance_error_vs_fp64": rel,
        "accuracy": "missing rate and discrepancy over all %d points against exact brute force "
                    "(rpf_brute_knn); FP64 distance error on 2,000 rows" % n,
        "operating_point": {"n_trees": t_op, "stated_n_trees": stated,
                            "verified_smallest_in_grid": verified, "sweep_uniform": sweep_u},
        "stage_ms": {"build": round(sum(b_ms) / len(b_ms), 3),
                     "all_knn": round(sum(a_ms) / len(a_ms), 3)},
        "plain": {"value": round(world * n / (p_ms * 1e-3), 1), "ms_per_step": round(p_ms, 3),
                  "stage_ms": {"build": round(sum(p_b) / len(p_b), 3),
                               "all_knn": round(sum(p_a) / len(p_a), 3)}},
        "chosen_equals_plain": same,
        "autotune": tuned,
        "at_configured_n_trees": at_cfg,
        "median_split_rule": med,
        "forest": info,
        "e2e": {"value": round(world * n / e2e_s, 1), "unit": "queries/s",
                "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(n * w.k * 8)},
        "gpu_launches": int((l1 - l0) / args.steps),
        "gpu_launches_per_step": True,
        "roofline": roof,
        "kernel_rooflines": roofs,
        "plain_leaf_roofline": [r for r in roofs_p if r["kernel"] == "k_leaf_plain"],
        "work_model": work["_point_levels"],
        "kernels_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in
                                sorted(trace.items(), key=lambda kv: -kv[1]["ms"])},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_large:
        line["large_batched"] = run_large(args, dev)
    if rank == 0 and world == 1 and not args.no_sweep:
        line["ensemble_sweep"] = run_sweep(args, dev)
        line["n_try_ablation"] = run_ntry_ablation(args, dev)
        line["split_rules"] = run_split_rules(args, dev)
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cb = oracle_step(X, w, t_op, threads, seed=args.seed)
        cb["single_thread"] = oracle_single_thread(X, w, t_op, seed=args.seed)
        line["cpu_baseline"] = cb
    return line


SERVE_T_GRID = (32, 64, 128, 256, 384, 512)  # nested ensembles of the serving workload


def run_serving(args, dev, n_requests=300):
    """Serving on the resident-forest workload (2M x 96, leaf bound 128):
    saturation throughput (all requests at once), then Poisson arrivals at
    0.5 / 0.8 / 0.95 of it, for each K; p50 / p99 from arrival to results
    ready on the host.  Measured at the configured T = 32 and at the
    operating point: the forest grows (rpf_add_trees, nested ensembles) until
    the missing rate of 500 held-out queries at K = 10 is at most 1 %."""
    import torch
    from paper_1812_11689_gb300 import forest, serve, synth
    w = synth.WORKLOADS["mix50_d96"]
    X = torch.from_numpy(synth.make("mix50_d96", seed=args.seed)).to(dev)
    t0 = time.perf_counter()
    f = forest.Forest(X, n_trees=w.n_trees, leaf_max=w.leaf_max, n_try=w.n_try, seed=args.seed,
                      form=forest.FORM_CHOSEN)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sizes = synth.request_sizes(n_requests, seed=args.seed, max_size=w.extra["max_request"])
    Qs = torch.from_numpy(synth.queries("mix50_d96", 500, seed=args.seed, stream=9999)).to(dev)
    truth = {K: forest.brute_knn(X, Qs, K)[0].cpu().numpy() for K in w.extra["k_set"]}

    def missing(K):
        qi, _ = f.query(Qs, K)
        return round(float(missing_counts(qi.cpu().numpy(), truth[K]).sum()) / truth[K].size, 5)

    def make_reqs(K, stream0):
        return [serve.Request(i, synth.queries("mix50_d96", int(m), seed=args.seed,
                                               stream=stream0 + i), K, 0.0)
                for i, m in enumerate(sizes)]

    def runs_at():
        runs = {}
        mean_m = float(np.mean(sizes))
        for K in w.extra["k_set"]:
            tuned = f.autotune(K)  # the query scan of the chosen form, among others
            serve.Server(f, slots=4).run(make_reqs(K, 1000)[:20])  # warm-up
            srv = serve.Server(f, slots=4, max_batch=8192)
            sat = serve.latency_summary(srv.run(make_reqs(K, 2000)))
            r = {"saturation": sat}
            for load in (0.5, 0.8, 0.95):
                rate = load * sat["queries_per_s"] / mean_m
                arr = synth.poisson_arrivals(n_requests, rate_per_s=rate, seed=args.seed + 1)
                srv = serve.Server(f, slots=4, max_batch=8192)
                res = serve.latency_summary(srv.run(make_reqs(K, 3000), arr))
                res["offered_requests_per_s"] = round(rate, 1)
                res["batches"] = srv.n_batches
                r["load_%.2f" % load] = res
            r["missing_rate_sample_500"] = missing(K)
            r["autotune"] = tuned
            # the plain FP32 form of the same forest (identical lists), saturated
            f.set_form(forest.FORM_PLAIN)
            srv = serve.Server(f, slots=4, max_batch=8192)
            r["plain_saturation"] = serve.latency_summary(srv.run(make_reqs(K, 2000)))
            f.set_form(forest.FORM_CHOSEN)
            runs["K=%d" % K] = r
        return runs

    out = {"workload": "mix50_d96", "n": w.n, "d": w.d, "leaf_max": w.leaf_max,
           "requests_per_run": n_requests,
           "request_sizes": "floor(exp(U(0, ln 4097))) clamped to [1, 4096]",
           "build_s_32_trees": round(build_s, 3), "slots": 4, "max_batch": 8192,
           "accuracy_sample": "500 held-out queries vs exact brute force (rpf_brute_knn)",
           "configured": {"n_trees": w.n_trees, "runs": runs_at()}}
    sweep, t_op = [], None
    T = w.n_trees
    for Tn in SERVE_T_GRID:
        if Tn > T:
            t0 = time.perf_counter()
            f.add_trees(Tn - T)
            torch.cuda.synchronize()
            sweep.append({"added_trees": Tn - T, "add_s": round(time.perf_counter() - t0, 3)})
            T = Tn
        m10 = missing(10)
        sweep.append({"n_trees": T, "missing_rate_k10": m10})
        if m10 <= 0.01:
            t_op = T
            break
    out["sweep"] = sweep
    if t_op is not None:
        out["operating_point"] = {"n_trees": t_op, "runs": runs_at()}
    else:
        out["operating_point"] = {"not_reached_by_n_trees": max(SERVE_T_GRID)}
    f.close()
    return out


def run_sweep(args, dev, rows=2000):
    """Ensemble sweep (Sec. 5.2 accuracy experiments on synthetic data): one
    forest of 128 trees over the heavy-tailed workload answers all-kNN over
    its first T trees for every T of the sweep (nested ensembles), for
    nTry = 1 and 5, both forms; missing rate and kNN-distance discrepancy on
    a sample of points against exact brute force."""
    import torch
    from paper_1812_11689_gb300 import forest, synth
    w = synth.WORKLOADS["student3_d32"]
    Xh = synth.make("student3_d32", seed=args.seed)
    X = torch.from_numpy(Xh).to(dev)
    n = w.n
    r = torch.from_numpy(np.sort(np.random.default_rng(2).choice(n, rows, replace=False))
                         .astype(np.int32)).to(dev)
    bi, bd = forest.brute_knn(X, X[r.long()].contiguous(), w.k, self_idx=r)
    bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
    out = {"workload": "student3_d32", "n": n, "d": w.d, "leaf_max": w.leaf_max, "k": w.k,
           "sample": "%d points vs exact brute force" % rows, "n_try": {}}
    for ntry in (1, 5):
        f = {}
        for form in (forest.FORM_PLAIN, forest.FORM_CHOSEN):
            t0 = time.perf_counter()
            f[form] = forest.Forest(X, n_trees=max(w.extra["t_sweep"]), leaf_max=w.leaf_max,
                                    n_try=ntry, seed=args.seed, form=form)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
        rows_out, prev = [], None
        monotone = True
        for T in w.extra["t_sweep"]:
            res = {"n_trees": T}
            lists = {}
            for form, nm in ((forest.FORM_PLAIN, "plain"), (forest.FORM_CHOSEN, "chosen")):
                f[form].all_knn(w.k, n_trees=T)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                i, d = f[form].all_knn(w.k, n_trees=T)
                e1.record()
                torch.cuda.synchronize()
                res[nm + "_all_knn_ms"] = round(e0.elapsed_time(e1), 3)
                lists[nm] = (i, d)
            res["chosen_equals_plain"] = bool(torch.equal(lists["plain"][0], lists["chosen"][0])
                                              and torch.equal(lists["plain"][1], lists["chosen"][1]))
            ci = lists["chosen"][0][r.long()].cpu().numpy()
            cd = lists["chosen"][1][r.long()].cpu().numpy()
            miss = np.array([len(set(bi[q]) - set(ci[q])) for q in range(rows)])
            if prev is not None and np.any(miss > prev):
                monotone = False
            prev = miss
            res["missing_rate"] = round(float(miss.sum()) / bi.size, 5)
            res["knn_distance_discrepancy"], res["points_with_short_lists"] = \
                discrepancy_full(cd, bd)
            rows_out.append(res)
        out["n_try"][str(ntry)] = {"build_s_128_trees_chosen": round(build_s, 3), "by_T": rows_out,
                                   "missing_per_point_non_increasing_in_T": monotone}
        for v in f.values():
            v.close()
    return out


def run_large(args, dev, rows=1000):
    """All-kNN on the large batched workload (points near a 16-dimensional
    subspace, n = 1,000,000, d = 128, T = 64, leaf bound 256, K = 20): the
    chosen form's persistent tensor-core launch over every (tree, leaf) tile,
    against the plain form on the same forest shape."""
    import torch
    from paper_1812_11689_gb300 import forest, synth
    w = synth.WORKLOADS["subspace16_d128"]
    X = torch.from_numpy(synth.make("subspace16_d128", seed=args.seed)).to(dev)
    out = {"workload": "subspace16_d128", "n": w.n, "d": w.d, "n_trees": w.n_trees,
           "leaf_max": w.leaf_max, "k": w.k, "n_try": w.n_try}
    res = {}
    for form, nm in ((forest.FORM_CHOSEN, "chosen"), (forest.FORM_PLAIN, "plain")):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        f = forest.Forest(X, n_trees=w.n_trees, leaf_max=w.leaf_max, n_try=w.n_try,
                          seed=args.seed, form=form)
        e1.record()
        i, d = f.all_knn(w.k)
        e2.record()
        torch.cuda.synchronize()
        res[nm] = (i, d, e0.elapsed_time(e1), e1.elapsed_time(e2), f.counters())
        f.close()
    ci, cd, bc, ac, cnt = res["chosen"]
    pi, pd, bp, ap, _ = res["plain"]
    r = torch.from_numpy(np.sort(np.random.default_rng(3).choice(w.n, rows, replace=False))
                         .astype(np.int32)).to(dev)
    bi, _ = forest.brute_knn(X, X[r.long()].contiguous(), w.k, self_idx=r)
    bi, cis = bi.cpu().numpy(), ci[r.long()].cpu().numpy()
    out.update({
        "chosen": {"build_ms": round(bc, 2), "all_knn_ms": round(ac, 2),
                   "queries_per_s": round(w.n / ((bc + ac) * 1e-3), 1),
                   "certificate_fallback_rows": cnt.get("bf16_fallback_rows")},
        "plain": {"build_ms": round(bp, 2), "all_knn_ms": round(ap, 2),
                  "queries_per_s": round(w.n / ((bp + ap) * 1e-3), 1)},
        "chosen_equals_plain": bool(torch.equal(ci, pi) and torch.equal(cd, pd)),
        "missing_rate_sample": round(sum(len(set(bi[q]) - set(cis[q])) for q in range(rows))
                                     / float(bi.size), 5),
        "sample": "%d points vs exact brute force" % rows,
        "timing": "one cold step per form (build + all-kNN), CUDA events"})
    return out


def run_ntry_ablation(args, dev, rows=2000):
    """nTry ablation (Sec. 5.2 varies the projections tried per split): on the
    anisotropic workload (T = 40) and the heavy-tailed one (T = 32), the
    missing rate, discrepancy, build time and the share of split nodes the
    certified FP32 path had to settle in FP64, for nTry in {1, 3, 5, 10, 20}."""
    import torch
    from paper_1812_11689_gb300 import forest, synth
    out = {}
    for name, T in (("aniso20_d64", 40), ("student3_d32", 32)):
        w = synth.WORKLOADS[name]
        X = torch.from_numpy(synth.make(name, seed=args.seed)).to(dev)
        r = torch.from_numpy(np.sort(np.random.default_rng(4).choice(w.n, rows, replace=False))
                             .astype(np.int32)).to(dev)
        bi, bd = forest.brute_knn(X, X[r.long()].contiguous(), w.k, self_idx=r)
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
        res = []
        for ntry in (1, 3, 5, 10, 20):
            kw = dict(n_trees=T, leaf_max=w.leaf_max, n_try=ntry, seed=args.seed,
                      form=forest.FORM_CHOSEN)
            forest.Forest(X, **kw).close()  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = forest.Forest(X, **kw)
            e1.record()
            i, d = f.all_knn(w.k)
            torch.cuda.synchronize()
            info = f.info()
            ci, cd = i[r.long()].cpu().numpy(), d[r.long()].cpu().numpy()
            internal = (info["n_nodes"] - info["n_leaves"])
            res.append({"n_try": ntry, "build_ms": round(e0.elapsed_time(e1), 2),
                        "missing_rate": round(sum(len(set(bi[q]) - set(ci[q]))
                                                  for q in range(rows)) / float(bi.size), 5),
                        "knn_distance_discrepancy": discrepancy_full(cd, bd)[0],
                        "fp64_settled_split_share": round(info["n_exact_nodes"] / max(internal, 1), 5),
                        "max_depth": info["max_depth"]})
            f.close()
        out[name] = {"n_trees": T, "leaf_max": w.leaf_max, "k": w.k, "by_n_try": res,
                     "sample": "%d points vs exact brute force" % rows}
    return out


def run_split_rules(args, dev, rows=2000):
    """Split rules (Sec. 2): c uniform on [min, max] of the projections
    against the median, on the anisotropic (T = 40) and heavy-tailed (T = 32)
    workloads -- build time, depth, all-kNN time, missing rate."""
    import torch
    from paper_1812_11689_gb300 import forest, synth
    out = {}
    for name, T in (("aniso20_d64", 40), ("student3_d32", 32)):
        w = synth.WORKLOADS[name]
        X = torch.from_numpy(synth.make(name, seed=args.seed)).to(dev)
        r = torch.from_numpy(np.sort(np.random.default_rng(5).choice(w.n, rows, replace=False))
                             .astype(np.int32)).to(dev)
        bi, bd = forest.brute_knn(X, X[r.long()].contiguous(), w.k, self_idx=r)
        bi, bd = bi.cpu().numpy(), bd.cpu().numpy()
        res = {}
        for rule, nm in ((forest.SPLIT_UNIFORM, "uniform"), (forest.SPLIT_MEDIAN, "median")):
            kw = dict(n_trees=T, leaf_max=w.leaf_max, n_try=w.n_try, seed=args.seed,
                      form=forest.FORM_CHOSEN, split_rule=rule)
            forest.Forest(X, **kw).close()  # warm-up
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            f = forest.Forest(X, **kw)
            e1.record()
            i, d = f.all_knn(w.k)
            e2.record()
            torch.cuda.synchronize()
            info, cnt = f.info(), f.counters()
            ci, cd = i[r.long()].cpu().numpy(), d[r.long()].cpu().numpy()
            res[nm] = {"build_ms": round(e0.elapsed_time(e1), 2),
                       "all_knn_ms": round(e1.elapsed_time(e2), 2),
                       "queries_per_s": round(w.n / (e0.elapsed_time(e2) * 1e-3), 1),
                       "max_depth": info["max_depth"],
                       "phase_a_levels": cnt.get("phase_a_levels"),
                       "missing_rate": round(sum(len(set(bi[q]) - set(ci[q]))
                                                 for q in range(rows)) / float(bi.size), 5),
                       "knn_distance_discrepancy": discrepancy_full(cd, bd)[0]}
            f.close()
        out[name] = {"n_trees": T, "leaf_max": w.leaf_max, "k": w.k, "by_rule": res,
                     "sample": "%d points vs exact brute force" % rows}
    return out


def run_profile_step(args):
    import torch
    from paper_1812_11689_gb300 import forest, synth
    w = synth.WORKLOADS[args.workload]
    X = torch.from_numpy(synth.make(args.workload, seed=args.seed)).cuda()
    T = args.profile_trees or w.extra.get("n_trees_le_1pct", w.n_trees)
    kw = dict(n_trees=T, leaf_max=w.leaf_max, n_try=w.n_try, seed=args.seed,
              form=forest.FORM_CHOSEN)
    counts = []
    for _ in range(2):
        l0 = forest.Trace.launch_count()
        f = forest.Forest(X, **kw)
        f.all_knn(w.k)
        torch.cuda.synchronize()
        counts.append(forest.Trace.launch_count() - l0)
        f.close()
    return {"profile_step": True, "workload": args.workload, "n_trees": T,
            "launches_per_step": counts}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, as it stands, on the host cores, at
    the GPU arm's operating point (same workload and tree count); every step
    is one oracle_step (all trees grown in full, a quarter of the points
    answered).  Warm-up steps run the same function on a small sample (8
    trees, 1 % of the points) to page the data and the library in."""
    from paper_1812_11689_gb300 import synth
    if rank != 0:
        return None
    w = synth.WORKLOADS[args.workload]
    X = synth.make(args.workload, seed=args.seed)
    T = w.extra.get("n_trees_le_1pct", w.n_trees)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_step(X, w, min(8, T), threads, rows_fraction=0.01, seed=args.seed)
    res, step_s = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res.append(oracle_step(X, w, T, threads, seed=args.seed))
        step_s.append(time.perf_counter() - t0)
    v = statistics.median(r["value"] for r in res)
    cb = dict(res[-1])
    cb["value"] = v
    return {"impl": "reference", "metric": "all-kNN queries/s at <=1% missing rate "
            "(chosen vs plain FP32 form)", "value": round(v, 2), "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(step_s) / len(step_s), 3),
            "ms_per_step_is": "wall time of one oracle step (all trees, sampled answers); "
                              "value = n / the step's full-workload time",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "precision": "split decisions FP64, distances FP32 (canonical d32 key)",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": w.n, "d": w.d, "n_trees": T,
                       "leaf_max": w.leaf_max, "k": w.k, "n_try": w.n_try,
                       "split_rule": "uniform", "form": "oracle (exact union of leaves)"},
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 2), "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if args.impl == "gb300":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend=backend)
    if args.profile_step:
        line = run_profile_step(args)
    elif args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_gb300(args, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
