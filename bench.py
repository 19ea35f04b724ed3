"""Benchmark of the merged-index vector epsilon-join on one B300.

Metric: queries/s at recall >= 0.95 against the exact join, learned+BF16 arm
versus the plain FP32 arm.  One step = one join of every query of the
workload against the prebuilt merged index (the offline build is timed
separately, as the paper excludes indexing from join latency).

  plain FP32     MI+SWS (Alg. 1 with soft sharing) in FP32; CheckHybrid by the
                 d1/d2 rule; when that misses recall 0.95, hybrid search for
                 every query with the smallest queue size reaching it.
  learned+BF16   MI+SWS with the learned prologue: a predictor (trained here
                 on labels from the joins) routes each query to the BF16
                 tensor-core brute-force scan (exact after re-check) or gives
                 it a hybrid queue size; the route threshold is the largest
                 one reaching recall 0.95.

The default workload is 1M data x 100K queries x 128-d integer descriptors
(sift_like, degree 32, eps for a mean of 20 matches per query).  Prints one
JSON line.  --impl reference times the CPU oracle's join (FP64, one thread)
on whole MST subtrees of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at recall≥0.95 vs exact join: learned+BF16 vs plain FP32, one B300"


def _traffic(kernel, scale):
    """DRAM bytes per step of `kernel` from profiles/traffic.md (an ncu capture of the full-size learned
    step), or None when the workload is not the full-size one or the kernel's source changed since."""
    if scale != 1.0:
        return None
    import hashlib
    import re
    p = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        m = re.match(r"^\| (\S+) \| (\S+) \| ([0-9a-f]{64}) \| ([0-9.eE+]+) \|", line)
        if m and m.group(1) == kernel:
            src = os.path.join(ROOT, m.group(2))
            if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest() == m.group(3):
                return float(m.group(4))
    return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), d.get("bf16_tflops", 1800.0), "measured"
    return 6400.0, 1800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, idx=0):
        self.idx, self.rows, self.proc = idx, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_workload(name, scale):
    from paper_2603_16360_b300 import inputs
    if name == "sift_like":
        return inputs.sift_like(scale=scale)
    if name == "gauss_small":
        return inputs.gauss_small()
    if name == "angular_one":
        # one instance of the angular collection's recipe: 300K x 30K (times scale), d = 100 cosine
        nx, nq = int(3e5 * scale), int(3e4 * scale)
        return inputs.angular_instance(1239, 0, nx_range=(nx, nx + 1), nq_range=(nq, nq + 1))
    raise SystemExit(f"unknown workload {name}")


def calibrate_eps(vj, ix, w, target):
    """eps with a mean of `target` exact matches per query (exact GPU join)."""
    rng = np.random.default_rng(w.seed + 7)
    qs = w.Q[rng.choice(w.nq, size=min(200, w.nq), replace=False)].astype(np.float64)
    xs = w.X[rng.choice(w.nx, size=min(20000, w.nx), replace=False)].astype(np.float64)
    d2 = (qs ** 2).sum(1)[:, None] + (xs ** 2).sum(1)[None, :] - 2 * qs @ xs.T
    dd = np.sqrt(np.maximum(d2, 0)).ravel()
    guess = float(np.quantile(dd, min(8.0 * target / w.nx, 0.5)))
    for _ in range(12):
        ex = vj.vj_join_exact(ix, guess)
        if ex.offsets[-1] >= target * w.nq:
            break
        guess *= 1.25
    k = int(target * w.nq)
    return float(np.float32(np.partition(ex.dists, k)[k]))


def per_query_hits(r, ex, nx):
    """(hits per query, exact count per query) of result r against ex."""
    nq = len(ex.offsets) - 1
    qa = np.repeat(np.arange(nq, dtype=np.int64), np.diff(ex.offsets))
    qb = np.repeat(np.arange(nq, dtype=np.int64), np.diff(r.offsets))
    ka = qa * nx + ex.ids
    kb = qb * nx + r.ids
    common = np.intersect1d(ka, kb, assume_unique=True)
    hits = np.bincount(common // nx, minlength=nq)
    return hits, np.diff(ex.offsets)


def recall_of(r, ex, nx):
    hits, tot = per_query_hits(r, ex, nx)
    return float(hits.sum() / max(tot.sum(), 1))


def per_query_recall_mean(r, ex, nx):
    """Mean over queries of |R n E| / |E|; a query with an empty exact row counts 1."""
    hits, tot = per_query_hits(r, ex, nx)
    return float(np.where(tot > 0, hits / np.maximum(tot, 1), 1.0).mean())


def sample_subtrees(parent, order, target=1000):
    """Whole MST subtrees (children of the entry) totalling >= target queries, in order."""
    nq = len(parent)
    children = {}
    for q in range(nq):
        children.setdefault(int(parent[q]), []).append(q)
    chosen = set()
    for r0 in [q for q in order if parent[q] < 0]:
        stack = [int(r0)]
        while stack:
            a = stack.pop()
            chosen.add(a)
            stack.extend(children.get(a, []))
        if len(chosen) >= target:
            break
    return np.array([q for q in order if int(q) in chosen], np.int32)


def run_cpu_oracle(w, vj, ix, eps, sample_q=1000, mode="adapt", budget=256):
    import oracle
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    sub = sample_subtrees(parent, order, sample_q)
    t0 = time.perf_counter()
    oracle.join(w.X, w.Q, adj, entry, eps, work_sharing=oracle.WS_SOFT, adapt_hybrid=(mode == "adapt"),
                force_hybrid=(mode == "force"), hybrid_beam_size=budget, order=sub, parent=parent, queries=sub)
    return len(sub), time.perf_counter() - t0


def timed(vj, torch, ix, eps, budget, steps, warmup, tag="timed"):
    """Device-resident joins on torch's current stream: (ms per step, per-step stats).

    The timed steps run inside an NVTX range named `tag`, so a profiler can
    select exactly their kernels (ncu --nvtx --nvtx-include "<tag>/")."""
    stream = torch.cuda.current_stream()
    vj.vj_set_stream(ix, stream.cuda_stream)
    for _ in range(warmup):
        vj.vj_join_device(ix, eps, budget).free()
    torch.cuda.synchronize()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(tag)
    e0.record(stream)
    for _ in range(steps):
        dr = vj.vj_join_device(ix, eps, budget)
        s = dict(dr.stats)
        s["nnz"] = dr.nnz
        stats.append(s)
        dr.free()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, stats


def slowest_rank_ms(ms, dist, device):
    """The largest of the ranks' times (ms itself without a process group)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def collection_learned_arm(vj, ixs, eps, exs, nxs, nqs, pooled_recall, steps):
    """One predictor for the whole collection: trained on the labels of the
    six cheapest instances (per query: the smallest hybrid queue size on the
    ladder {0, 8, 32} reaching recall 0.95, and the route to the scan when none
    does or when the BFS costs more than a scan row), attached to every index,
    then the largest route threshold whose batched join reaches pooled recall
    0.95 (non-routed queries run the BFS closure)."""
    order = np.argsort([nq * nx for nq, nx in zip(nqs, nxs)], kind="stable")
    train_ids = [int(i) for i in order[:6]]
    Fs, yb, yr = [], [], []
    ladder = [0, 8, 32]
    for i in train_ids:
        ix, e, ex, nx = ixs[i], eps[i], exs[i], nxs[i]
        recs = {}
        for b in ladder:
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=int(b > 0),
                                  hybrid_beam=max(b, 1), learned=0)
            r = vj.vj_join(ix, e)
            h, tot = per_query_hits(r, ex, nx)
            recs[b] = np.where(tot > 0, h / np.maximum(tot, 1), 1.0)
            if b == 0:
                s0, st0 = r.steps.astype(np.float64), r.stats
        t_step = st0["ms_traverse"] / max(s0.sum(), 1.0)
        t_bf = ex.stats["ms_scan"] / len(s0)
        budget = np.full(len(s0), ladder[-1], np.int32)
        for b in reversed(ladder):
            budget = np.where(recs[b] >= 0.95, b, budget)
        route = (recs[ladder[-1]] < 0.95) | (s0 * t_step >= t_bf)
        Fs.append(vj.vj_features(ix, e))
        yb.append(np.log2(budget + 1.0))
        yr.append(route.astype(np.float32))
    F = np.concatenate(Fs)
    mlp = vj.MLP(F.shape[1], 256, 256, seed=7)
    t0 = time.perf_counter()
    loss = mlp.train(F, np.concatenate(yb).astype(np.float32), np.concatenate(yr), epochs=30, batch=256, lr=1e-3,
                     seed=7)
    train_s = time.perf_counter() - t0
    sweep, best = [], None
    for thr in (0.999, 0.99, 0.97, 0.9, 0.7, 0.5, 0.3):
        for ix in ixs:
            vj.vj_attach_predictor(ix, mlp, thr, 0)
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0, hybrid_beam=1,
                                  learned=1)
        vj.vj_join_batch(ixs, eps)
        t0 = time.perf_counter()
        rs = vj.vj_join_batch(ixs, eps)
        ms = 1e3 * (time.perf_counter() - t0)
        rec = pooled_recall(rs)
        routed = int(sum(int((r.hybrid == 2).sum()) for r in rs))
        sweep.append({"thr": thr, "recall": round(rec, 4), "ms": round(ms, 1), "routed": routed})
        if rec >= 0.95 and (best is None or ms < best[1]):
            best = (thr, ms)
    out = {"train_instances": train_ids, "train_queries": int(F.shape[0]), "train_s": round(train_s, 1),
           "final_loss": loss, "sweep": sweep}
    if best is not None:
        thr = best[0]
        for ix in ixs:
            vj.vj_attach_predictor(ix, mlp, thr, 0)
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            rs = vj.vj_join_batch(ixs, eps)
            ts.append(1e3 * (time.perf_counter() - t0))
        ms = statistics.median(ts)
        out.update({"thr": thr, "ms_per_step": ms, "queries_per_s": int(sum(nqs)) / (ms / 1e3),
                    "recall": pooled_recall(rs), "routed_frac": sum(int((r.hybrid == 2).sum()) for r in rs) / sum(nqs)})
    for ix in ixs:
        vj.vj_set_join_params(ix, learned=0)
        vj.vj_attach_predictor(ix, None, 0.5, 0)
    mlp.free()
    return out


def bench_collection(args, vj, torch):
    """A collection of independent join instances of very different sizes
    (angular_collection: |X| log-uniform 1e4..2e6 and |Q| 1e3..2e5, both times
    --scale, d = 100 cosine), joined by vj_join_batch (the traversal passes of
    all instances fused into one launch per pass) and, for comparison, by one
    vj_join per instance.  Plain MI+SWS (FP32); the d1/d2 rule, else forced
    hybrid search with the smallest queue size reaching pooled recall 0.95."""
    from paper_2603_16360_b300 import inputs
    lo = lambda v: max(int(v * args.scale), 2000)
    rng_kw = dict(nx_range=(lo(1e4), max(lo(2e6), lo(1e4) + 1)),
                  nq_range=(max(int(1e3 * args.scale), 100), max(int(2e5 * args.scale), 101)))
    ixs, eps, nqs, nxs, targets, exs = [], [], [], [], [], []
    t0 = time.perf_counter()
    build_total = 0.0
    for w in inputs.angular_collection(n=args.instances, **rng_kw):
        tb = time.perf_counter()
        ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
        build_total += time.perf_counter() - tb
        e = calibrate_eps(vj, ix, w, w.target_matches)
        ixs.append(ix)
        eps.append(e)
        nqs.append(w.nq)
        nxs.append(w.nx)
        targets.append(w.target_matches)
        exs.append(vj.vj_join_exact(ix, e))
        del w
    build_s = time.perf_counter() - t0
    total_q = int(sum(nqs))

    def pooled_recall(rs):
        hits = tot = 0
        for r, ex, nx in zip(rs, exs, nxs):
            h, t = per_query_hits(r, ex, nx)
            hits += int(h.sum())
            tot += int(t.sum())
        return hits / max(tot, 1)

    chosen = None
    sweep = []
    for mode, budget in [("adapt", 256)] + [("force", b) for b in (2, 4, 8, 16, 32, 64, 128, 256)]:
        for ix in ixs:
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=int(mode == "adapt"),
                                  force_hybrid=int(mode == "force"), hybrid_beam=budget, learned=0)
        t1 = time.perf_counter()
        rs = vj.vj_join_batch(ixs, eps)
        t1 = time.perf_counter() - t1
        rec = pooled_recall(rs)
        sweep.append({"hybrid": mode, "beam": budget, "recall": round(rec, 4), "ms": round(1e3 * t1, 1)})
        chosen = (mode, budget, rec, rs)
        if rec >= 0.95:
            break
    mode, budget, rec, rs = chosen
    pairs = int(sum(r.nnz for r in rs))
    for _ in range(args.warmup):
        vj.vj_join_batch(ixs, eps)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as cs:
        batch_ms, trav_ms = [], []
        for _ in range(args.steps):
            t1 = time.perf_counter()
            rb = vj.vj_join_batch(ixs, eps)
            batch_ms.append(1e3 * (time.perf_counter() - t1))
            trav_ms.append(rb[0].stats["ms_traverse"])
        seq_ms, seq_trav = [], []
        for _ in range(max(2, args.steps // 2)):
            t1 = time.perf_counter()
            tt = 0.0
            per_inst = []
            for k, (ix, e) in enumerate(zip(ixs, eps)):
                r1 = vj.vj_join(ix, e)
                st1 = r1.stats
                tt += st1["ms_traverse"]
                per_inst.append({"i": k, "nx": nxs[k], "nq": nqs[k], "ms_traverse": round(st1["ms_traverse"], 3),
                                 "ms_sws": [round(x, 3) for x in st1["ms_sws"]],
                                 "dist_per_query": round(st1["dist_computations"] / nqs[k], 1),
                                 "max_visited": int(r1.steps.max()), "restarts": st1["sws_restarts"],
                                 "spill_queries": st1["spill_queries"]})
            seq_ms.append(1e3 * (time.perf_counter() - t1))
            seq_trav.append(tt)
    b_ms = statistics.median(batch_ms)
    s_ms = statistics.median(seq_ms)
    d2h = int(sum(r.offsets.nbytes + r.ids.nbytes + r.dists.nbytes + r.steps.nbytes + r.cache.nbytes +
                  r.hybrid.nbytes for r in rb))
    line = {"metric": "queries/s of a collection of join instances at pooled recall≥0.95 vs exact join, one B300",
            "value": total_q / (b_ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"angular_collection: {len(ixs)} instances, |X| {min(nxs)}..{max(nxs)} "
                                   f"(sum {sum(nxs)}), |Q| {min(nqs)}..{max(nqs)} (sum {total_q}), d=100 cosine, "
                                   f"eps for a mean of {min(targets):g}..{max(targets):g} matches/query",
                       "arm": f"vj_join_batch, plain MI+SWS FP32, hybrid={mode} beam {budget}",
                       "recall": rec, "pairs": pairs, "sweep": sweep,
                       "prep_s": round(build_s, 1), "build_s": round(build_total, 2),
                       "fused_traversal_ms": statistics.median(trav_ms),
                       "one_join_per_instance": {"ms_per_step": s_ms, "queries_per_s": total_q / (s_ms / 1e3),
                                                 "traversal_ms_sum": statistics.median(seq_trav)},
                       "batch_vs_one_by_one": s_ms / b_ms,
                       "dist_computations": int(sum(r.stats["dist_computations"] for r in rb)),
                       "slowest_instances": sorted(per_inst, key=lambda x: -x["ms_traverse"])[:6],
                       "timing": "host wall time of the public call (host results, device-to-host copies inside)"},
            "e2e": {"value": total_q / (b_ms / 1e3), "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": d2h},
            "clocks": cs.summary()}
    if args.collection_learned:
        line["config"]["learned"] = collection_learned_arm(vj, ixs, eps, exs, nxs, nqs, pooled_recall,
                                                           max(3, args.steps))
    print(json.dumps(line), flush=True)
    for ix in ixs:
        ix.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sift_like")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-only", action="store_true")
    ap.add_argument("--instances", type=int, default=64, help="angular_collection: number of join instances")
    ap.add_argument("--collection-learned", action="store_true",
                    help="angular_collection: also time one shared predictor's learned route")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference" and rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    from paper_2603_16360_b300 import vj
    vj.load()
    if args.workload == "angular_collection":
        if rank == 0 and args.impl == "ours":
            bench_collection(args, vj, torch)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    w = make_workload(args.workload, args.scale)
    target = w.target_matches
    t0 = time.perf_counter()
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k))
    build_s = time.perf_counter() - t0
    info = ix.info()
    eps = calibrate_eps(vj, ix, w, target)
    ex = vj.vj_join_exact(ix, eps)
    wl_desc = (f"{w.name}: X={w.nx} Q={w.nq} d={w.d} {'L2' if w.metric == 0 else 'cosine'}, "
               f"eps for a mean of {target:g} matches/query")

    # ---- plain FP32 arm: operating point
    plain = None
    for mode, budget in [("adapt", 256)] + [("force", b) for b in (2, 4, 8, 16, 32, 64, 128, 256)]:
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=int(mode == "adapt"),
                              force_hybrid=int(mode == "force"), hybrid_beam=budget, learned=0)
        r = vj.vj_join(ix, eps)
        rec = recall_of(r, ex, w.nx)
        plain = (mode, budget, rec, r)
        if rec >= 0.95:
            break
    pmode, pbudget, prec, pr = plain

    if args.impl == "reference":
        n_s, dt = [], []
        for _ in range(args.warmup):
            run_cpu_oracle(w, vj, ix, eps, 200, pmode, pbudget)
        for _ in range(args.steps):
            n, t = run_cpu_oracle(w, vj, ix, eps, 1000, pmode, pbudget)
            n_s.append(n)
            dt.append(t)
        v = sum(n_s) / sum(dt)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dt) / len(dt),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": wl_desc, "arm": f"CPU oracle MI+SWS hybrid={pmode} beam {pbudget} "
                                                       "(Alg. 1), FP64, 1 thread", "eps": eps},
                "cpu_baseline": {"value": v, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                 "sample": f"whole MST subtrees, {n_s[0]} queries per step, on the GPU-built graph"},
                "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm, bf16, peak_kind = _peaks()
    # ---- time the plain arm
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=int(pmode == "adapt"),
                          force_hybrid=int(pmode == "force"), hybrid_beam=pbudget, learned=0)
    p_ms, p_stats = timed(vj, torch, ix, eps, pbudget, max(2, args.steps // 2), args.warmup, "plain_timed")
    plain_qps = w.nq / (p_ms / 1e3)

    learned = None
    if not args.plain_only:
        # ---- labels for the predictor on a seeded 10% training subset
        rng = np.random.default_rng(w.seed + 99)
        train = np.sort(rng.choice(w.nq, size=max(1, w.nq // 10), replace=False))
        ladder = [0, 8, 32]
        recs, steps_at, missed = {}, {}, {}
        for b in ladder:
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=int(b > 0),
                                  hybrid_beam=max(b, 1), learned=0)
            r = vj.vj_join(ix, eps)
            h, tot = per_query_hits(r, ex, w.nx)
            recs[b] = np.where(tot > 0, h / np.maximum(tot, 1), 1.0)
            missed[b] = (tot - h).astype(np.float64)
            steps_at[b] = r.stats, r.steps.astype(np.float64)
        st0, s0 = steps_at[0]
        t_step = st0["ms_traverse"] / max(s0.sum(), 1)             # ms per distance evaluation (BFS join)
        t_bf = ex.stats["ms_scan"] / w.nq                           # ms per query of the full scan
        budget_lab = np.full(w.nq, ladder[-1], np.int32)
        for b in reversed(ladder):
            budget_lab = np.where(recs[b] >= 0.95, b, budget_lab)
        # route labels: the routing a knapsack would choose on the training
        # queries for pooled recall 0.955 -- every query whose BFS costs more
        # than its scan row, then the others by missed pairs per unit of
        # extra cost, until the missed pairs left are within 4.5 %
        tot_all = np.diff(ex.offsets).astype(np.float64)
        c_bfs = s0 * t_step
        gain = np.where(c_bfs >= t_bf, np.inf, missed[0] / np.maximum(t_bf - c_bfs, 1e-12))
        route_lab = np.zeros(w.nq, bool)

        def knapsack(idx):
            left, allowed = missed[0][idx].sum(), 0.045 * tot_all[idx].sum()
            for qi in idx[np.argsort(-gain[idx], kind="stable")]:
                if left <= allowed and not np.isinf(gain[qi]):
                    break
                route_lab[qi] = missed[0][qi] > 0 or np.isinf(gain[qi])
                left -= missed[0][qi]

        held = np.setdiff1d(np.arange(w.nq), train)
        knapsack(train)
        knapsack(held)
        F = vj.vj_features(ix, eps)
        mlp = vj.MLP(F.shape[1], 256, 256, seed=w.seed)
        t_tr = time.perf_counter()
        final_loss = mlp.train(F[train], np.log2(budget_lab[train] + 1.0), route_lab[train].astype(np.float32),
                               epochs=30, batch=256, lr=1e-3, seed=w.seed)
        train_s = time.perf_counter() - t_tr
        pred = mlp.predict(F)
        route_acc = float(((pred[held, 1] > 0) == route_lab[held]).mean())
        # operating point: the fastest (route threshold, hybrid-queue cap) whose join reaches recall 0.95
        op, sweep = None, []
        grid = [(0, t) for t in (0.99, 0.97, 0.95, 0.9, 0.85, 0.8, 0.7, 0.6, 0.5, 0.4, 0.2)] + [(64, t) for t in (0.9, 0.6, 0.3)]
        for cap, thr in grid:
            vj.vj_attach_predictor(ix, mlp, thr, cap)
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0,
                                  hybrid_beam=max(cap, 1), learned=1)
            vj.vj_join(ix, eps)
            r = vj.vj_join(ix, eps)
            rec = recall_of(r, ex, w.nx)
            sweep.append({"thr": thr, "beam_cap": cap, "recall": round(rec, 4), "ms": round(r.stats["ms_total"], 2),
                          "routed": int((r.hybrid == 2).sum()), "ms_traverse": round(r.stats["ms_traverse"], 2),
                          "ms_route": round(r.stats["ms_route"], 2),
                          "ms_sws": [round(x, 2) for x in r.stats["ms_sws"]], "reruns": r.stats["sws_restarts"]})
            if rec >= 0.95 and (op is None or r.stats["ms_total"] < op[3]):
                op = (thr, rec, r, r.stats["ms_total"], cap)
        if op is None:  # nothing reached 0.95: route everything that the predictor doubts least
            op = (0.05, rec, r, r.stats["ms_total"], 64)
        thr, lrec, lr_, _, lcap = op
        vj.vj_attach_predictor(ix, mlp, thr, lcap)
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0,
                              hybrid_beam=max(lcap, 1), learned=1)
        l_ms, l_stats = timed(vj, torch, ix, eps, 0, args.steps, args.warmup, "learned_timed")
        learned = {"thr": thr, "beam_cap": lcap, "sweep": sweep, "recall": lrec, "ms": l_ms, "stats": l_stats,
                   "route_acc": route_acc,
                   "routed_frac": float((lr_.hybrid == 2).mean()), "train_s": train_s, "final_loss": final_loss,
                   "labels_route_frac": float(route_lab.mean()), "t_bf_ms": t_bf, "t_step_ms": t_step,
                   "recall_per_query_mean": per_query_recall_mean(lr_, ex, w.nx)}

    # ---- headline arm and its rooflines
    if learned is not None:
        step_ms, stats, rec = learned["ms"], learned["stats"], learned["recall"]
        arm = (f"learned+BF16: MI+SWS with the learned prologue, route threshold {learned['thr']}, "
               f"hybrid-queue cap {learned['beam_cap']}")
        dtype = "bf16"
    else:
        step_ms, stats, rec = p_ms, p_stats, prec
        arm = f"plain FP32 MI+SWS, hybrid={pmode} beam {pbudget}"
        dtype = "f32"
    value = world * w.nq / (step_ms / 1e3)
    t_tr = statistics.mean(s["ms_traverse"] for s in stats)
    t_sc = statistics.mean(s["ms_scan"] for s in stats)
    trav = {"kernel": "k_join (traversal)", "bound": "hbm", "unit": "GB/s", "peak": hbm,
            "achieved": statistics.mean(s["bytes_algorithmic"] for s in stats) / (t_tr / 1e3) / 1e9,
            "ms_per_launch": t_tr, "algorithmic_bytes_per_launch": statistics.mean(s["bytes_algorithmic"] for s in stats),
            "peak_kind": f"{peak_kind} hbm_gbs (burst)",
            "traffic": _traffic("k_join", args.scale) if learned is not None and args.workload == "sift_like" else None}
    trav["frac"] = trav["achieved"] / hbm
    rooflines = [trav]
    if learned is not None and t_sc > 0:
        nrouted = learned["routed_frac"] * w.nq
        flops = 2.0 * nrouted * w.nx * w.d
        scan = {"kernel": "k_tc_scan (tcgen05 BF16 brute-force scan)", "bound": "tensor", "unit": "TFLOP/s",
                "peak": bf16, "achieved": flops / (t_sc / 1e3) / 1e12, "ms_per_launch": t_sc,
                "algorithmic_flops_per_launch": flops, "peak_kind": f"{peak_kind} bf16_tflops (burst)",
                "traffic": _traffic("k_tc_scan_res", args.scale) if args.workload == "sift_like" else None}
        scan["frac"] = scan["achieved"] / bf16
        rooflines.append(scan)
    dominant = max(rooflines, key=lambda k: k["ms_per_launch"])

    # clocks during one more timed run of the headline arm
    with ClockSampler(torch.cuda.current_device()) as cs:
        time.sleep(0.3)
        timed(vj, torch, ix, eps, 0 if learned is not None else pbudget, args.steps, 1, "clock_run")
        time.sleep(0.2)

    # ---- end to end through the public call with a host result
    e2e_ms, e2e_gpu = [], []
    rh = None
    for _ in range(max(2, args.warmup)):  # untimed: page-locked result blocks enter the cache
        rh = vj.vj_join(ix, eps, 0 if learned is not None else pbudget)  # (two results alive at a time)
    for _ in range(max(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rh = vj.vj_join(ix, eps, 0 if learned is not None else pbudget)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_gpu.append(rh.stats["ms_total"])
    d2h = int(rh.offsets.nbytes + rh.ids.nbytes + rh.dists.nbytes + rh.steps.nbytes + rh.cache.nbytes +
              rh.hybrid.nbytes)
    # replicas: every rank joins the same workload; the job's time is the slowest rank's
    e2e_v = world * w.nq / (slowest_rank_ms(statistics.median(e2e_ms), dist, "cuda") / 1e3)
    if dist:
        step_ms = slowest_rank_ms(step_ms, dist, "cuda")
        value = world * w.nq / (step_ms / 1e3)
    rec_q = learned["recall_per_query_mean"] if learned is not None else per_query_recall_mean(pr, ex, w.nx)
    cfg = {"workload": wl_desc, "arm": arm, "recall": rec, "recall_per_query_mean": rec_q, "eps": eps,
           "degree": info["degree"],
           "knn_k": info["knn_k"], "mst_depth": info["max_depth"], "build_s": build_s,
           "pairs": int(stats[-1]["nnz"]), "pairs_per_s": world * stats[-1]["nnz"] / (step_ms / 1e3),
           "l2": "inputs larger than L2 (vectors %.0f MB)" % ((w.X.nbytes + w.Q.nbytes) / 1e6),
           "plain_fp32": {"qps": plain_qps, "ms_per_step": p_ms, "recall": prec, "hybrid": pmode,
                          "hybrid_beam": pbudget},
           "exact_join_ms": ex.stats["ms_total"], "exact_scan_ms": ex.stats["ms_scan"], "seed": w.seed,
           "e2e_detail": {"wall_ms": [round(x, 3) for x in e2e_ms], "join_stats_ms": [round(x, 3) for x in e2e_gpu],
                          "timed_step_join_stats_ms": round(statistics.mean(s["ms_total"] for s in stats), 3)}}
    if learned is not None:
        cfg["learned"] = {k: learned[k] for k in ("thr", "beam_cap", "sweep", "recall", "route_acc", "routed_frac",
                                                   "train_s", "final_loss", "labels_route_frac", "t_bf_ms", "t_step_ms")}
        cfg["learned"]["ms_prologue"] = statistics.mean(s["ms_prologue"] for s in stats)
        cfg["learned_vs_plain"] = value / plain_qps
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg, "roofline": dominant,
            "rooflines": rooflines,
            "e2e": {"value": e2e_v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
            "clocks": cs.summary(),
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
    if rank == 0 and not args.no_cpu_baseline:
        # a bounded sample: whole MST subtrees of about 15,000 queries, some seconds of one core
        n, dt = run_cpu_oracle(w, vj, ix, eps, 15000, pmode, pbudget)
        line["cpu_baseline"] = {"value": n / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} queries (whole MST subtrees) of the same workload on the GPU-built "
                                          f"graph, oracle MI+SWS join (hybrid={pmode}, beam {pbudget}), FP64, "
                                          "single thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    ix.free()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
