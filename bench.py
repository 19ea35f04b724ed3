"""Benchmark of the merged-index vector epsilon-join on one B300.

Metric: queries/s at recall >= 0.95 against the exact join, learned+BF16 arm
versus the plain FP32 arm.  One step = one join of every query of the index
(the offline build is timed separately, as the paper excludes indexing from
join latency).

Default workload: 10M data x 1M evaluated queries x 768-d unit vectors rounded
to BF16 (vmf_like: a 4,096-component von Mises-Fisher mixture, kappa 50, 20 %
of the queries from unseen components; cosine distance; eps for a mean of 10
matches per query; degree 32).  A further 100K held-out queries of the same
recipe are built into the same merged index: the learned arm trains on them
and picks its operating point on them; recall and queries/s count only the
evaluated queries (the held-out rows are joined in every step too).

  plain FP32     MI+SWS (Alg. 1 with soft sharing) with FP32 gathers: the
                 d1/d2 rule at several hybrid queue sizes, the rule with its
                 OOD queries routed to the tensor-core brute-force scan, and
                 forced hybrid search when none of those reaches 0.95; the
                 fastest setting reaching recall 0.95 is timed.
  learned+BF16   MI+SWS with the predictor's per-query plan (route to the
                 scan, no expansion, BFS or a hybrid queue size), trained by
                 the library on the held-out queries (vj_train_predictor), and
                 BF16 gathers (exact here: every coordinate is a BF16 value).

Before its timed steps each arm runs vj_autotune (untimed setup, like the
training): the traversal setting it keeps gives the same join, only faster.
--no-tune times both arms with the default setting.

Prints one JSON line.  --impl reference times the CPU oracle's join (FP64,
one thread) on whole MST subtrees of the same workload instead.
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
# queries (whole MST subtrees) in the CPU oracle's timed sample: the cpu_baseline and each step of the
# reference arm time the same subtrees
CPU_SAMPLE = 3000


def _traffic(kernel, workload):
    """DRAM bytes per step of `kernel` on `workload` ("name@scale") from profiles/traffic.md, or None when
    no capture of that workload is recorded or the kernel's source changed since."""
    import hashlib
    import re
    p = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        m = re.match(r"^\| (\S+) \| (\S+) \| (\S+) \| ([0-9a-f]{64}) \| ([0-9.eE+]+) \|", line)
        if m and m.group(1) == kernel and m.group(2) == workload:
            src = os.path.join(ROOT, m.group(3))
            if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest() == m.group(4):
                return float(m.group(5))
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


def make_workload(name, scale, replica=0):
    """The workload `name` (replica r > 0: the same recipe with seed + 1000 r)."""
    from paper_2603_16360_b300 import inputs
    if name == "vmf_like":
        return inputs.vmf_like(seed=1238 + 1000 * replica, scale=scale, device="cuda")
    if name == "sift_like":
        return inputs.sift_like(seed=1236 + 1000 * replica, scale=scale, nh=10_000)
    if name == "gauss_small":
        return inputs.gauss_small()
    if name == "gauss_wide":
        return inputs.gauss_wide(seed=1237 + 1000 * replica, scale=scale)
    if name == "angular_one":
        # one instance of the angular collection's recipe: 300K x 30K (times scale), d = 100 cosine
        nx, nq = int(3e5 * scale), int(3e4 * scale)
        return inputs.angular_instance(1239, 0, nx_range=(nx, nx + 1), nq_range=(nq, nq + 1))
    raise SystemExit(f"unknown workload {name}")


def host(a):
    """numpy copy of a workload array (host arrays pass through)."""
    return a.detach().cpu().numpy() if hasattr(a, "detach") else a


def n_eval(w):
    """Evaluated queries: the rows of Q before the held-out ones."""
    return w.nq - getattr(w, "nh", 0)


def calibrate_eps(vj, ix, w, target):
    """eps with a mean of `target` exact matches per evaluated query: an
    overestimate from a 200 x 20,000 sample, then the k-th distance of the
    exact GPU join."""
    rng = np.random.default_rng(w.seed + 7)
    ne = n_eval(w)
    qi = np.sort(rng.choice(ne, size=min(200, ne), replace=False))
    xi = np.sort(rng.choice(w.nx, size=min(20000, w.nx), replace=False))
    if hasattr(w.X, "detach"):
        import torch
        qs = w.Q[torch.from_numpy(qi).to(w.Q.device)].double().cpu().numpy()
        xs = w.X[torch.from_numpy(xi).to(w.X.device)].double().cpu().numpy()
    else:
        qs, xs = w.Q[qi].astype(np.float64), w.X[xi].astype(np.float64)
    if w.metric == 0:
        d2 = (qs ** 2).sum(1)[:, None] + (xs ** 2).sum(1)[None, :] - 2 * qs @ xs.T
        dd = np.sqrt(np.maximum(d2, 0)).ravel()
    else:
        qn = qs / np.linalg.norm(qs, axis=1, keepdims=True)
        xn = xs / np.linalg.norm(xs, axis=1, keepdims=True)
        dd = (1.0 - qn @ xn.T).ravel()
    guess = float(np.quantile(dd, min(8.0 * target / w.nx, 0.5)))
    for _ in range(12):
        ex = vj.vj_join_exact(ix, guess)
        if ex.offsets[ne] >= target * ne:
            break
        # grow: L2 by a factor, cosine by shrinking the similarity bound
        guess = guess * 1.25 if w.metric == 0 else 1.0 - (1.0 - guess) * 0.9
    k = int(target * ne)
    return float(np.float32(np.partition(ex.dists[:ex.offsets[ne]], k)[k]))


def per_query_hits(r, ex, nx, rows=None):
    """(hits, exact count) per query of result r against ex, over the query
    index range rows = (lo, hi) (all queries when None)."""
    lo, hi = (0, len(ex.offsets) - 1) if rows is None else rows
    qa = np.repeat(np.arange(lo, hi, dtype=np.int64), np.diff(ex.offsets[lo:hi + 1]))
    qb = np.repeat(np.arange(lo, hi, dtype=np.int64), np.diff(r.offsets[lo:hi + 1]))
    ka = qa * nx + ex.ids[ex.offsets[lo]:ex.offsets[hi]]
    kb = qb * nx + r.ids[r.offsets[lo]:r.offsets[hi]]
    common = np.intersect1d(ka, kb, assume_unique=True)
    hits = np.bincount(common // nx - lo, minlength=hi - lo)
    return hits, np.diff(ex.offsets[lo:hi + 1])


def recall_of(r, ex, nx, rows=None):
    hits, tot = per_query_hits(r, ex, nx, rows)
    return float(hits.sum() / max(tot.sum(), 1))


def per_query_recall_mean(r, ex, nx, rows=None):
    """Mean over queries of |R n E| / |E|; a query with an empty exact row counts 1."""
    hits, tot = per_query_hits(r, ex, nx, rows)
    return float(np.where(tot > 0, hits / np.maximum(tot, 1), 1.0).mean())


def sample_subtrees(parent, order, target=1000, limit=None):
    """Whole MST subtrees (children of the entry) totalling >= target queries,
    in processing order; with `limit`, only queries below it (their
    subtrees contain no other query)."""
    nq = len(parent)
    children = {}
    for q in range(nq):
        children.setdefault(int(parent[q]), []).append(q)
    chosen = set()
    for r0 in [q for q in order if parent[q] < 0]:
        stack, sub = [int(r0)], []
        while stack:
            a = stack.pop()
            sub.append(a)
            stack.extend(children.get(a, []))
        if limit is not None and max(sub) >= limit:
            continue
        chosen.update(sub)
        if len(chosen) >= target:
            break
    return np.array([q for q in order if int(q) in chosen], np.int32)


def run_cpu_oracle(w, vj, ix, eps, sample_q, mode, budget, Xh, Qh):
    """The oracle's MI+SWS join (FP64, one thread) on whole MST subtrees of
    evaluated queries of the GPU-built graph: (queries, seconds)."""
    import oracle
    adj, entry, parent, order, _ = vj.vj_export_graph(ix)
    sub = sample_subtrees(parent, order, sample_q, limit=n_eval(w))
    t0 = time.perf_counter()
    oracle.join(Xh, Qh, adj, entry, eps, metric=w.metric, work_sharing=oracle.WS_SOFT,
                adapt_hybrid=(mode == "adapt"), force_hybrid=(mode == "force"), hybrid_beam_size=budget,
                order=sub, parent=parent, queries=sub)
    return len(sub), time.perf_counter() - t0


def timed(vj, torch, ix, eps, budget, steps, warmup, tag="timed", clocks=False):
    """Device-resident joins on torch's current stream: (ms per step, per-step
    stats, clock summary or None).  The timed steps run inside an NVTX range
    named `tag` (ncu --nvtx --nvtx-include "<tag>/" selects their kernels);
    with clocks, nvidia-smi samples the SM clock during them."""
    stream = torch.cuda.current_stream()
    vj.vj_set_stream(ix, stream.cuda_stream)
    for _ in range(warmup):
        vj.vj_join_device(ix, eps, budget).free()
    torch.cuda.synchronize()
    stats = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cs = ClockSampler(torch.cuda.current_device()) if clocks else None
    if cs:
        cs.__enter__()
        time.sleep(0.3)  # the sampler's first rows before the timed region
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
    if cs:
        cs.__exit__()
    return e0.elapsed_time(e1) / steps, stats, (cs.summary() if cs else None)


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



def plain_arm(vj, ix, eps, ex, w, log):
    """The paper's method in FP32 (MI+SWS): the d1/d2 rule at several hybrid
    queue sizes, the rule with its OOD queries sent to the brute-force scan,
    and, when none of those reaches recall 0.95 on the evaluated queries,
    forced hybrid search at growing queue sizes.  Returns the fastest setting
    that reaches 0.95 (else the one with the best recall) and the sweep."""
    ne = n_eval(w)
    sweep, best, best_any = [], None, None

    def consider(name, setup):
        nonlocal best, best_any
        try:
            setup()
            vj.vj_join(ix, eps)
            r = vj.vj_join(ix, eps)
        except vj.VjError as e:
            sweep.append({"setting": name, "error": str(e)[:120]})
            vj.vj_set_plan(ix, None, None)
            return None
        rec = recall_of(r, ex, w.nx, (0, ne))
        ent = {"setting": name, "recall": round(rec, 4), "ms": round(r.stats["ms_total"], 3),
               "hybrid_queries": r.stats["hybrid_queries"], "routed": int((r.hybrid == 2).sum())}
        sweep.append(ent)
        log(f"plain {name}: recall {rec:.4f} ms {r.stats['ms_total']:.2f}")
        cand = (r.stats["ms_total"], name, setup, rec, r)
        if rec >= 0.95 and (best is None or cand[0] < best[0]):
            best = cand
        if best_any is None or rec > best_any[3]:
            best_any = cand
        return rec

    def rule(beam):
        return lambda: (vj.vj_set_plan(ix, None, None),
                        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=1, force_hybrid=0,
                                              hybrid_beam=beam, learned=0, gather=vj.VJ_PREC_FP32))

    for beam in (256, 32, 4):
        consider(f"rule, hybrid queue {beam}", rule(beam))
    # the rule's OOD queries (hybrid flag 1 under the rule) routed to the exact scan
    rule(256)()
    flags = vj.vj_join(ix, eps).hybrid
    route = (flags == 1).astype(np.uint8)

    def rule_route():
        vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0, hybrid_beam=1,
                              learned=0, gather=vj.VJ_PREC_FP32)
        vj.vj_set_plan(ix, route, np.zeros(w.nq, np.int32))

    consider(f"rule, its {int(route.sum())} OOD queries routed to the scan", rule_route)
    if best is None:
        for beam in (2, 4, 8, 16, 32, 64, 128, 256):
            rec = consider(f"forced hybrid, queue {beam}",
                           lambda beam=beam: (vj.vj_set_plan(ix, None, None),
                                              vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0,
                                                                    force_hybrid=1, hybrid_beam=beam, learned=0,
                                                                    gather=vj.VJ_PREC_FP32)))
            if rec is not None and rec >= 0.95:
                break
    return (best or best_any), sweep


def learned_arm(vj, ix, eps, ex, w, log, caps):
    """The learned route with BF16 gathers: a predictor trained by the library
    on the held-out queries' labels (vj_train_predictor), then the fastest
    (route threshold, hybrid-queue cap) whose join reaches recall 0.955 on
    the held-out queries.  The evaluated queries' recall is measured after."""
    ne = n_eval(w)
    rows = np.arange(ne, w.nq, dtype=np.int32)
    t0 = time.perf_counter()
    m, rep = vj.vj_train_predictor(ix, eps, rows, ladder=[-1, 0, 8], query_recall=0.95, pooled_recall=0.955,
                                   h1=256, h2=256, epochs=30, batch=256, lr=1e-3, seed=w.seed)
    train_s = time.perf_counter() - t0
    log(f"trained on {len(rows)} held-out queries in {train_s:.1f}s: {rep}")
    sweep, op = [], None
    for cap in caps:
        for thr in (0.99, 0.95, 0.9, 0.8, 0.7, 0.5, 0.3, 0.1):
            vj.vj_attach_predictor(ix, m, thr, cap)
            vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0,
                                  hybrid_beam=max(cap, 1), learned=1, gather=vj.VJ_PREC_BF16)
            try:
                vj.vj_join(ix, eps)
                r = vj.vj_join(ix, eps)
            except vj.VjError as e:
                sweep.append({"thr": thr, "beam_cap": cap, "error": str(e)[:120]})
                continue
            rh = recall_of(r, ex, w.nx, (ne, w.nq))
            ent = {"thr": thr, "beam_cap": cap, "heldout_recall": round(rh, 4), "ms": round(r.stats["ms_total"], 3),
                   "routed": int((r.hybrid == 2).sum()), "no_expansion": int((r.hybrid == 3).sum()),
                   "ms_traverse": round(r.stats["ms_traverse"], 3), "ms_route": round(r.stats["ms_route"], 3)}
            sweep.append(ent)
            log(f"learned {ent}")
            if rh >= 0.955 and (op is None or r.stats["ms_total"] < op[2]):
                op = (thr, cap, r.stats["ms_total"])
    if op is None:  # nothing reached the target on the held-out queries: route the most
        op = (0.01, caps[0], None)
    vj.vj_attach_predictor(ix, m, op[0], op[1])
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=0, force_hybrid=0, hybrid_beam=max(op[1], 1),
                          learned=1, gather=vj.VJ_PREC_BF16)
    return m, {"thr": op[0], "beam_cap": op[1], "sweep": sweep, "train_s": train_s, "train_report": rep}


def profile_modes(args, vj, ix, w, build_s, binfo):
    """--mode build / join: one JSON line per build or join, for profiling runs."""
    print(json.dumps({"mode": "build", "workload": w.name, "nx": w.nx, "nq": w.nq, "d": w.d, "build_s": build_s,
                      **binfo}), flush=True)
    if args.mode != "join":
        return
    # a threshold near the workload's: the exact join's calibration is not needed to time a traversal
    eps = calibrate_eps(vj, ix, w, w.target_matches)
    plan = {"none": -1, "bfs": 0}.get(args.plan)
    vj.vj_set_join_params(ix, work_sharing=vj.VJ_WS_SOFT, adapt_hybrid=int(plan is None), learned=0,
                          gather=vj.VJ_PREC_BF16)
    if plan is not None:
        vj.vj_set_plan(ix, None, np.full(w.nq, plan, np.int32))
    if args.tune:
        # the traversal settings the tuner tries, their join times, and the one it keeps
        print(json.dumps({"mode": "tune", "eps": eps, **vj.vj_autotune(ix, eps, reps=max(1, args.reps))}),
              flush=True)
    for i in range(args.reps):
        st = vj.vj_join(ix, eps).stats
        print(json.dumps({"mode": "join", "plan": args.plan, "rep": i, "eps": eps, "ms_total": st["ms_total"],
                          "ms_traverse": st["ms_traverse"], "ms_sws": st["ms_sws"],
                          "dist_per_query": st["dist_computations"] / w.nq,
                          "gbs_algorithmic": st["bytes_algorithmic"] / st["ms_traverse"] / 1e6}), flush=True)
    vj.vj_set_plan(ix, None, None)


def fp8_gemm_peak(torch):
    """Dense E4M3 GEMM throughput (TFLOP/s) of the library path (torch._scaled_mm, 8192^3, best of 10 by CUDA
    events): the measured FP8 denominator beside the nominal ratio (2x the measured BF16 peak)."""
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda")

        def f():
            return torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            f()
        best = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        return 2.0 * n ** 3 / best / 1e9, None
    except Exception as e:  # no FP8 GEMM in this torch build
        return None, str(e).splitlines()[0][:200]


def precision_mode(args, vj, torch, ix, w, build_s, binfo, log):
    """--mode precision: the exact join (the brute-force scan of every query,
    Sec. 3.2's NLJ) with BF16 and with FP8-e4m3 tiles on the same index.  Both
    re-decide every candidate from the FP32 vectors (FP64 near eps), so their
    rows are identical; the precision changes the tile throughput and the
    candidate count.  Per precision: scan kernel time, TFLOP/s and fraction of
    the tensor peak, candidates per query, whole-join time.  Error against FP64
    on sampled queries: pair ids outside the 1e-4 eps band and the largest
    relative distance error.  One JSON line."""
    hbm, bf16_peak, kind = _peaks()
    eps = calibrate_eps(vj, ix, w, w.target_matches)
    flops = 2.0 * w.nq * w.nx * w.d
    out = {"mode": "precision", "workload": f"{w.name}: X={w.nx} Q={w.nq} d={w.d} "
           f"{'L2' if w.metric == 0 else 'cosine'}, eps for a mean of {w.target_matches:g} matches/query",
           "eps": eps, "build_s": build_s, "build": binfo, "flops_per_scan": flops}
    f8_peak, f8_err = fp8_gemm_peak(torch)
    out["fp8_gemm_tflops_measured"] = f8_peak
    if f8_err:
        out["fp8_gemm_error"] = f8_err
    results = {}
    for name, prec, peak in (("bf16", vj.VJ_PREC_BF16, bf16_peak), ("fp8", vj.VJ_PREC_FP8, 2.0 * bf16_peak)):
        vj.vj_set_join_params(ix, scan=prec)
        r = vj.vj_join_exact(ix, eps)  # first call: the data-side tile rows and the candidate arrays
        reps = []
        for _ in range(max(1, args.reps)):
            r = vj.vj_join_exact(ix, eps)
            reps.append((r.stats["ms_scan"], r.stats["ms_total"]))
        ms_scan = statistics.median(x[0] for x in reps)
        ms_total = statistics.median(x[1] for x in reps)
        nnz = int(r.offsets[-1])
        results[name] = r
        out[name] = {"ms_scan": ms_scan, "ms_total": ms_total, "scan_tflops": flops / ms_scan / 1e9,
                     "peak_tflops": peak, "peak_kind": f"{kind} bf16 burst" + (" x 2 (nominal FP8:BF16)" if
                                                                              name == "fp8" else ""),
                     "frac": flops / ms_scan / 1e9 / peak,
                     "candidates_per_query": r.stats["scan_candidates"] / w.nq, "pairs": nnz,
                     "queries_per_s": w.nq / ms_total * 1e3}
        if name == "fp8" and f8_peak:
            out[name]["frac_of_measured_fp8_gemm"] = flops / ms_scan / 1e9 / f8_peak
        log(f"{name}: {out[name]}")
    vj.vj_set_join_params(ix, scan=vj.VJ_PREC_BF16)
    rb, r8 = results["bf16"], results["fp8"]
    out["same_rows"] = bool(np.array_equal(rb.offsets, r8.offsets) and np.array_equal(rb.ids, r8.ids))
    # FP64 check on sampled queries: distances to every data vector on the GPU in FP64
    rng = np.random.default_rng(w.seed + 11)
    qs = np.sort(rng.choice(w.nq, size=min(64, w.nq), replace=False))
    Xd = torch.from_numpy(host(w.X)).cuda()
    Qs = torch.from_numpy(host(w.Q)[qs]).cuda().double()
    band_n, diff_n, max_rel, checked = 0, 0, 0.0, 0
    for i, q in enumerate(qs):
        dd = torch.zeros(w.nx, dtype=torch.float64, device="cuda")
        for a in range(0, w.nx, 1 << 18):
            xb = Xd[a:a + (1 << 18)].double()
            if w.metric == 0:
                dd[a:a + len(xb)] = (xb - Qs[i]).pow(2).sum(1).sqrt()
            else:
                dd[a:a + len(xb)] = 1.0 - (xb @ Qs[i]) / (xb.norm(dim=1) * Qs[i].norm())
        d64 = dd.cpu().numpy()
        exp = set(np.nonzero(d64 < eps)[0].tolist())
        lo, hi = int(rb.offsets[q]), int(rb.offsets[q + 1])
        got = set(rb.ids[lo:hi].tolist())
        near = set(np.nonzero(np.abs(d64 - eps) <= 1e-4 * eps)[0].tolist())
        band_n += len(near)
        diff_n += len((got ^ exp) - near)
        for j in range(lo, hi):
            x = int(rb.ids[j])
            max_rel = max(max_rel, abs(float(rb.dists[j]) - d64[x]) / max(d64[x], 1e-30))
            checked += 1
    del Xd
    out["fp64_check"] = {"queries": len(qs), "pairs_checked": checked, "pairs_differing_outside_band": diff_n,
                         "pairs_in_band": band_n, "max_rel_dist_err": max_rel}
    print(json.dumps(out), flush=True)


VARIANT_SETTINGS = {
    "nnmap": [("BFS expansion", dict(work_sharing=0, adapt_hybrid=0, force_hybrid=0, hybrid_beam=256)),
              ("adaptive hybrid, queue 64", dict(work_sharing=0, adapt_hybrid=1, force_hybrid=0, hybrid_beam=64)),
              ("adaptive hybrid, queue 256", dict(work_sharing=0, adapt_hybrid=1, force_hybrid=0, hybrid_beam=256)),
              ("forced hybrid, queue 64", dict(work_sharing=0, adapt_hybrid=0, force_hybrid=1, hybrid_beam=64))],
    # Sec. 3.2's separate-index executions (the paper's INLJ / HWS / SWS baselines)
    "separate": [("INLJ (greedy from s_Y), BFS expansion", dict(work_sharing=0, force_hybrid=0)),
                 ("HWS (parent's row as seeds), BFS expansion", dict(work_sharing=1, force_hybrid=0)),
                 ("SWS (parent's cache as seed), BFS expansion", dict(work_sharing=2, force_hybrid=0)),
                 ("SWS, forced hybrid, queue 8", dict(work_sharing=2, force_hybrid=1, hybrid_beam=8))],
}


def variant_mode(args, vj, torch, ix, w, build_s, binfo, log):
    """--mode nnmap / separate: the joins of an NN-Map or a separate-index
    build at the workload's eps, one JSON line.  Each setting runs `steps`
    device-resident joins (CUDA events on the launching stream); recall is
    against the exact join over the evaluated queries.  `value` is the fastest
    setting reaching recall 0.95 (else the most accurate)."""
    ne = n_eval(w)
    eps = calibrate_eps(vj, ix, w, w.target_matches)
    ex = vj.vj_join_exact(ix, eps)
    hbm, _, peak_kind = _peaks()
    settings = VARIANT_SETTINGS[args.mode]
    arms, best = [], None
    for k, (name, kw) in enumerate(settings):
        vj.vj_set_join_params(ix, learned=0, gather=vj.VJ_PREC_BF16, **kw)
        try:
            r = vj.vj_join(ix, eps)
        except vj.VjError as e:  # e.g. a hybrid search that outgrows the per-query visited capacity
            arms.append({"setting": name, "error": str(e)[:160]})
            log(f"{args.mode} {name}: {e}")
            continue
        rec = recall_of(r, ex, w.nx, (0, ne))
        ms, stats, clk = timed(vj, torch, ix, eps, 0, args.steps, args.warmup, "nnmap_timed", clocks=(k == 0))
        t_tr = statistics.mean(s["ms_traverse"] for s in stats)
        byts = statistics.mean(s["bytes_algorithmic"] for s in stats)
        arm = {"setting": name, "recall": round(rec, 4),
               "recall_per_query_mean": round(per_query_recall_mean(r, ex, w.nx, (0, ne)), 4),
               "ms_per_step": ms, "qps": ne / (ms / 1e3), "ms_traverse": t_tr,
               "dist_per_query": statistics.mean(s["dist_computations"] for s in stats) / w.nq,
               "hybrid_queries": int((r.hybrid[:ne] == 1).sum()),
               "roofline": {"kernel": f"k_join ({args.mode})", "bound": "hbm", "unit": "GB/s", "peak": hbm,
                            "achieved": byts / (t_tr / 1e3) / 1e9, "frac": byts / (t_tr / 1e3) / 1e9 / hbm,
                            "algorithmic_bytes_per_launch": byts, "peak_kind": f"{peak_kind} hbm_gbs (burst)",
                            "traffic": None},
               "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
        if clk is not None:
            arm["clocks"] = clk
        log(f"{args.mode} {name}: recall {rec:.4f} {arm['qps']:.3e} q/s")
        arms.append(arm)
        if best is None:
            best = arm
        elif (arm["recall"] >= 0.95) != (best["recall"] >= 0.95):
            best = arm if arm["recall"] >= 0.95 else best
        elif arm["recall"] >= 0.95:
            best = arm if arm["qps"] > best["qps"] else best
        else:
            best = arm if arm["recall"] > best["recall"] else best
    if best is None:
        raise SystemExit(f"{args.mode}: no setting ran: {arms}")
    line = {"mode": args.mode, "metric": METRIC, "value": best["qps"], "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True,
            "dtype": "bf16", "data": "synthetic", "roofline": best["roofline"], "clocks": arms[0].get("clocks"),
            "gpu_launches": best["gpu_launches"],
            "config": {"workload": f"{w.name}: X={w.nx} Q={ne} (+{w.nq - ne} held out) d={w.d} "
                                   f"{'L2' if w.metric == 0 else 'cosine'}, eps for a mean of "
                                   f"{w.target_matches:g} matches/query",
                       "arm": f"{'NN-Map' if args.mode == 'nnmap' else 'separate indexes'}: {best['setting']}, "
                              f"BF16 gathers", "eps": eps,
                       "build": {"wall_s": round(build_s, 2), "ms_device": binfo["ms_build"],
                                 "ms_knn": binfo["ms_knn"], "knn_tensor_cores": binfo["knn_tensor_cores"],
                                 "knn_uncertified": binfo["knn_uncertified"]},
                       "settings": arms}}
    if args.mode == "nnmap":
        _, wd, ood = vj.vj_export_nnmap(ix)
        line["config"]["certified_empty_frac"] = float((wd[:ne] >= eps).mean())
        # the witness property: a row is certified empty exactly when the exact row is empty
        line["config"]["certified_empty_equals_exact_empty"] = bool(np.array_equal(
            wd[:ne] >= eps, np.diff(ex.offsets[:ne + 1]) == 0))
        line["config"]["ood_frac"] = float(ood[:ne].mean())
    else:
        line["config"]["mst_depth"] = ix.info()["max_depth"]
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vmf_like")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-only", action="store_true")
    ap.add_argument("--instances", type=int, default=64, help="angular_collection: number of join instances")
    ap.add_argument("--collection-learned", action="store_true",
                    help="angular_collection: also time one shared predictor's learned route")
    ap.add_argument("--quiet", action="store_true")
    ap.add_argument("--mode", default="bench", choices=["bench", "build", "join", "nnmap", "separate", "precision"],
                    help="build: generate the workload and build the index only (profiling the build); join: "
                         "also run --reps joins with every query planned --plan (profiling the traversal); "
                         "nnmap: build an NN-Map index instead and time its joins (BFS, adaptive and forced "
                         "hybrid expansion from the witnesses); separate: build separate per-set indexes and time "
                         "INLJ, HWS and SWS")
    ap.add_argument("--plan", default="none", choices=["none", "bfs", "rule"],
                    help="--mode join: none = no expansion (the learned step's plan here), bfs, or the d1/d2 rule")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune", action="store_true", help="--mode join: run vj_autotune first and print its report")
    ap.add_argument("--no-tune", action="store_true", help="bench: time both arms with the default traversal setting")
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

    def log(msg):
        if not args.quiet and rank == 0:
            print(f"[bench] {msg}", file=sys.stderr, flush=True)

    from paper_2603_16360_b300 import vj
    vj.load()
    if args.workload == "angular_collection":
        if rank == 0 and args.impl == "ours":
            bench_collection(args, vj, torch)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    t0 = time.perf_counter()
    # ranks run independent replicas: the same recipe, each rank its own seed
    w = make_workload(args.workload, args.scale, rank)
    gen_s = time.perf_counter() - t0
    ne = n_eval(w)
    target = w.target_matches
    log(f"workload {w.name}: X {w.nx} x {w.d}, Q {ne} evaluated + {w.nq - ne} held out ({gen_s:.1f}s)")
    t0 = time.perf_counter()
    ix = vj.vj_build(w.X, w.Q, metric=w.metric, params=vj.default_params(degree=w.degree, knn_k=w.knn_k),
                     nnmap=int(args.mode == "nnmap"), separate=int(args.mode == "separate"))
    build_s = time.perf_counter() - t0
    info, binfo = ix.info(), ix.build_info()
    log(f"build {build_s:.1f}s {binfo}")
    if args.mode in VARIANT_SETTINGS:
        variant_mode(args, vj, torch, ix, w, build_s, binfo, log)
        ix.free()
        return
    if args.mode == "precision":
        precision_mode(args, vj, torch, ix, w, build_s, binfo, log)
        ix.free()
        return
    if args.mode != "bench":
        profile_modes(args, vj, ix, w, build_s, binfo)
        ix.free()
        return
    eps = calibrate_eps(vj, ix, w, target)
    ex = vj.vj_join_exact(ix, eps)
    log(f"eps {eps}: exact pairs {ex.offsets[ne]} over {ne} evaluated queries, scan {ex.stats['ms_scan']:.1f} ms")
    wl_desc = (f"{w.name}: X={w.nx} Q={ne} (+{w.nq - ne} held-out queries in the index) d={w.d} "
               f"{'L2' if w.metric == 0 else 'cosine'}, eps for a mean of {target:g} matches/query")

    plain, psweep = plain_arm(vj, ix, eps, ex, w, log)
    p_ms_sweep, pname, psetup, prec, pr = plain

    if args.impl == "reference":
        Xh, Qh = host(w.X), host(w.Q)
        mode = "adapt" if pname.startswith("rule") else "force"
        pbeam = int(pname.split()[-1]) if "queue" in pname else 256
        n_s, dt = [], []
        run_cpu_oracle(w, vj, ix, eps, 200, mode, pbeam, Xh, Qh)
        for _ in range(max(args.warmup - 1, 0)):
            run_cpu_oracle(w, vj, ix, eps, 200, mode, pbeam, Xh, Qh)
        for _ in range(args.steps):
            n, t = run_cpu_oracle(w, vj, ix, eps, CPU_SAMPLE, mode, pbeam, Xh, Qh)
            n_s.append(n)
            dt.append(t)
        v = sum(n_s) / sum(dt)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dt) / len(dt),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": wl_desc, "arm": f"CPU oracle MI+SWS ({pname}), Alg. 1, FP64, 1 thread",
                           "eps": eps},
                "cpu_baseline": {"value": v, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                 "sample": f"whole MST subtrees of evaluated queries, {n_s[0]} queries per step (the "
                                           f"cpu_baseline's sample), on the GPU-built graph, {pname}"},
                "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        ix.free()
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    hbm, bf16, peak_kind = _peaks()
    # ---- time the plain arm (its setting re-applied)
    psetup()
    # each arm runs with the traversal setting vj_autotune picks for it (untimed setup)
    p_tune = None if args.no_tune else vj.vj_autotune(ix, eps, reps=2)
    p_ms, p_stats, _ = timed(vj, torch, ix, eps, 0, max(2, args.steps // 2), args.warmup, "plain_timed")
    plain_qps = ne / (p_ms / 1e3)
    vj.vj_set_plan(ix, None, None)
    vj.vj_set_tuning(ix)

    learned, m = None, None
    if not args.plain_only:
        m, learned = learned_arm(vj, ix, eps, ex, w, log, caps=(0,) if w.d > 256 else (0, 64))
        l_tune = None if args.no_tune else vj.vj_autotune(ix, eps, reps=2)
        if l_tune:
            log(f"learned arm tuning: {l_tune['settings'][l_tune['chosen']]}")
        learned["tune"] = l_tune
        l_ms, l_stats, clk = timed(vj, torch, ix, eps, 0, args.steps, args.warmup, "learned_timed", clocks=True)
        r = vj.vj_join(ix, eps)
        learned.update({"ms": l_ms, "stats": l_stats, "clocks": clk, "recall": recall_of(r, ex, w.nx, (0, ne)),
                        "recall_per_query_mean": per_query_recall_mean(r, ex, w.nx, (0, ne)),
                        "routed_frac": float((r.hybrid[:ne] == 2).mean()),
                        "no_expansion_frac": float((r.hybrid[:ne] == 3).mean())})

    # ---- headline arm and its rooflines
    if learned is not None:
        step_ms, stats, rec, clk = learned["ms"], learned["stats"], learned["recall"], learned["clocks"]
        arm = (f"learned+BF16: MI+SWS with the predictor's plan (route threshold {learned['thr']}, hybrid-queue cap "
               f"{learned['beam_cap']}), BF16 gathers")
        dtype = "bf16"
    else:
        psetup()
        step_ms, stats, clk = timed(vj, torch, ix, eps, 0, args.steps, 1, "plain_clock", clocks=True)
        rec = prec
        arm = f"plain FP32 MI+SWS, {pname}"
        dtype = "f32"
    value = ne / (step_ms / 1e3)
    t_tr = statistics.mean(s["ms_traverse"] for s in stats)
    t_sc = statistics.mean(s["ms_scan"] for s in stats)
    trav = {"kernel": "k_join (traversal)", "bound": "hbm", "unit": "GB/s", "peak": hbm,
            "achieved": statistics.mean(s["bytes_algorithmic"] for s in stats) / (t_tr / 1e3) / 1e9,
            "ms_per_launch": t_tr, "algorithmic_bytes_per_launch": statistics.mean(s["bytes_algorithmic"] for s in stats),
            "peak_kind": f"{peak_kind} hbm_gbs (burst)",
            "traffic": _traffic("k_join", f"{args.workload}@{args.scale}")}
    trav["frac"] = trav["achieved"] / hbm
    rooflines = [trav]
    if learned is not None and t_sc > 0:
        nrouted = learned["routed_frac"] * ne + float((r.hybrid[ne:] == 2).sum())
        flops = 2.0 * nrouted * w.nx * w.d
        scan = {"kernel": "k_tc_res / k_tc_wide (tcgen05 BF16 brute-force scan)", "bound": "tensor",
                "unit": "TFLOP/s", "peak": bf16, "achieved": flops / (t_sc / 1e3) / 1e12, "ms_per_launch": t_sc,
                "algorithmic_flops_per_launch": flops, "peak_kind": f"{peak_kind} bf16_tflops (burst)",
                "traffic": _traffic("k_tc_scan", f"{args.workload}@{args.scale}")}
        scan["frac"] = scan["achieved"] / bf16
        rooflines.append(scan)
    dominant = max(rooflines, key=lambda k: k["ms_per_launch"])
    n_all = w.nx + w.nq
    kp = (w.d + 63) // 64 * 64
    # the kNN sweeps' tensor work: the sample sweep over every 16th tile, then the threshold sweep,
    # which for rows wider than 128 columns computes each unordered pair once (symmetric tiles)
    knn_flops = 2.0 * n_all * n_all * kp / 16 + (1.0 if kp > 128 else 2.0) * n_all * n_all * kp
    exact_flops = 2.0 * w.nq * w.nx * w.d

    # ---- end to end through the public call with a host result
    e2e_ms, e2e_gpu = [], []
    rh = None
    for _ in range(max(2, args.warmup)):  # untimed: page-locked result blocks enter the cache
        rh = vj.vj_join(ix, eps, 0)
    for _ in range(max(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rh = vj.vj_join(ix, eps, 0)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_gpu.append(rh.stats["ms_total"])
    d2h = int(rh.offsets.nbytes + rh.ids.nbytes + rh.dists.nbytes + rh.steps.nbytes + rh.cache.nbytes +
              rh.hybrid.nbytes)
    e2e_v = world * ne / (slowest_rank_ms(statistics.median(e2e_ms), dist, "cuda") / 1e3)
    if dist:
        step_ms = slowest_rank_ms(step_ms, dist, "cuda")
        value = world * ne / (step_ms / 1e3)
    rec_q = learned["recall_per_query_mean"] if learned is not None else per_query_recall_mean(pr, ex, w.nx, (0, ne))
    pairs = int(ex.offsets[ne])
    cfg = {"workload": wl_desc, "arm": arm, "recall": rec, "recall_per_query_mean": rec_q, "eps": eps,
           "degree": info["degree"], "knn_k": info["knn_k"], "mst_depth": info["max_depth"],
           "queries_evaluated": ne, "queries_held_out": w.nq - ne,
           "build": {"wall_s": round(build_s, 2), "ms_device": binfo["ms_build"], "ms_knn": binfo["ms_knn"],
                     "knn_tensor_cores": binfo["knn_tensor_cores"], "knn_uncertified": binfo["knn_uncertified"],
                     "knn_tflops": knn_flops / (binfo["ms_knn"] / 1e3) / 1e12,
                     "knn_frac_of_bf16_peak": knn_flops / (binfo["ms_knn"] / 1e3) / 1e12 / bf16,
                     "knn_flops": knn_flops},
           "generate_s": round(gen_s, 2),
           "pairs_per_s": world * pairs / (step_ms / 1e3),
           "l2": "inputs larger than L2 (FP32 vectors %.1f GB, BF16 copy %.1f GB)" % (
               (w.nx + w.nq) * w.d * 4 / 1e9, (w.nx + w.nq) * kp * 2 / 1e9),
           "plain_fp32": {"qps": plain_qps, "ms_per_step": p_ms, "recall": prec, "setting": pname,
                          "sweep": psweep,
                          "tune": p_tune["settings"][p_tune["chosen"]] if p_tune else "default (--no-tune)"},
           "exact_join": {"ms": ex.stats["ms_total"], "ms_scan": ex.stats["ms_scan"],
                          "tflops": exact_flops / (ex.stats["ms_scan"] / 1e3) / 1e12},
           "seed": w.seed,
           "e2e_detail": {"wall_ms": [round(x, 3) for x in e2e_ms], "join_stats_ms": [round(x, 3) for x in e2e_gpu],
                          "timed_step_join_stats_ms": round(statistics.mean(s["ms_total"] for s in stats), 3)}}
    if learned is not None:
        cfg["learned"] = {k: learned[k] for k in ("thr", "beam_cap", "sweep", "recall", "routed_frac",
                                                   "no_expansion_frac", "train_s", "train_report")}
        cfg["learned"]["ms_prologue"] = statistics.mean(s["ms_prologue"] for s in stats)
        lt = learned.get("tune")
        cfg["learned"]["tune"] = {"chosen": lt["settings"][lt["chosen"]], "tried": lt["settings"]} if lt else \
            "default (--no-tune)"
        cfg["learned_vs_plain"] = value / plain_qps
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg, "roofline": dominant,
            "rooflines": rooflines,
            "e2e": {"value": e2e_v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
            "clocks": clk,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}
    if rank == 0 and not args.no_cpu_baseline:
        # a bounded sample: the reference arm's per-step sample (whole MST
        # subtrees of about CPU_SAMPLE evaluated queries), in the plain arm's mode
        Xh, Qh = host(w.X), host(w.Q)
        mode = "adapt" if pname.startswith("rule") else "force"
        pbeam = int(pname.split()[-1]) if "queue" in pname else 256
        n, dt = run_cpu_oracle(w, vj, ix, eps, CPU_SAMPLE, mode, pbeam, Xh, Qh)
        line["cpu_baseline"] = {"value": n / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n} evaluated queries (whole MST subtrees) of the same workload on the "
                                          f"GPU-built graph, oracle MI+SWS join ({pname}), FP64, single thread"}
        del Xh, Qh
    if rank == 0:
        print(json.dumps(line), flush=True)
    vj.vj_attach_predictor(ix, None, 0.5, 64)
    if m is not None:
        m.free()
    ix.free()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
