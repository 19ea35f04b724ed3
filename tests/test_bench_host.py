"""Host-side logic of bench.py that needs no GPU: recall against the exact
join, MST-subtree sampling for the CPU baseline, the stored DRAM traffic and
the clock summary."""
import hashlib
import os
import re

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _R:
    def __init__(self, rows):
        self.offsets = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
        self.ids = np.concatenate([np.asarray(r, np.int32) for r in rows]) if rows else np.zeros(0, np.int32)


def test_recall_matches_set_arithmetic():
    rng = np.random.default_rng(3)
    nx, nq = 500, 60
    ex_rows = [np.sort(rng.choice(nx, rng.integers(0, 30), replace=False)) for _ in range(nq)]
    got_rows = []
    for r in ex_rows:
        keep = r[rng.random(len(r)) < 0.8]
        extra = rng.choice(nx, 3, replace=False)
        got_rows.append(np.unique(np.concatenate([keep, extra])))
    ex, got = _R(ex_rows), _R(got_rows)
    hits, tot = bench.per_query_hits(got, ex, nx)
    for q in range(nq):
        assert hits[q] == len(set(ex_rows[q]) & set(got_rows[q]))
        assert tot[q] == len(ex_rows[q])
    want = sum(len(set(a) & set(b)) for a, b in zip(ex_rows, got_rows)) / sum(len(a) for a in ex_rows)
    assert abs(bench.recall_of(got, ex, nx) - want) < 1e-12


def test_sample_subtrees_are_closed_under_parents():
    rng = np.random.default_rng(4)
    nq = 400
    # a random forest below the entry: parent < child in BFS order
    order = np.arange(nq, dtype=np.int32)
    parent = np.array([-1 if q < 6 or rng.random() < 0.02 else int(rng.integers(0, q)) for q in range(nq)], np.int32)
    sub = bench.sample_subtrees(parent, order, 100)
    s = set(int(q) for q in sub)
    assert len(s) >= 100
    for q in s:  # every chosen query's ancestors are chosen: whole subtrees
        p = parent[q]
        assert p < 0 or p in s
    children = {}
    for q in range(nq):
        children.setdefault(int(parent[q]), []).append(q)
    for q in s:  # and its descendants too
        assert all(c in s for c in children.get(q, []))
    pos = {int(q): i for i, q in enumerate(sub)}
    assert all(parent[q] < 0 or pos[int(parent[q])] < pos[q] for q in s)  # parents first


def test_stored_traffic_is_keyed_to_the_kernel_sources():
    text = open(os.path.join(ROOT, "profiles", "traffic.md")).read()
    rows = re.findall(r"^\| (\S+) \| (\S+) \| (\S+) \| ([0-9a-f]{64}) \| ([0-9.eE+]+) \|", text, re.M)
    assert rows and {r[0] for r in rows} <= {"k_join", "k_tc_scan"}
    for kernel, wl, src, sha, val in rows:
        cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
        got = bench._traffic(kernel, wl)
        assert got == (float(val) if cur == sha else None)
        assert bench._traffic(kernel, wl + "0") is None  # only the captured workload


def test_clock_summary_flags_throttle_reasons():
    cs = bench.ClockSampler()
    assert cs.summary()["reasons"] == ["unsampled"]
    cs.rows = [["2032", "2032", "900.5", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["1980", "2032", "1090.0", "Not Active", "Not Active", "Not Active", "Active"],
               ["2010", "2032", "1000.0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = cs.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_slowest_rank_without_process_group():
    assert bench.slowest_rank_ms(3.5, None, "cpu") == 3.5


def test_per_query_recall_mean_counts_empty_rows_as_one():
    ex = _R([[1, 2, 3, 4], [], [7]])
    got = _R([[1, 2], [5], []])
    # 2/4, empty exact row -> 1, 0/1
    assert abs(bench.per_query_recall_mean(got, ex, 10) - (0.5 + 1.0 + 0.0) / 3) < 1e-12
    assert abs(bench.recall_of(got, ex, 10) - 2 / 5) < 1e-12


def test_profile_commands_run_committed_files_only():
    """Every profile summary gives its command, and the command runs files of
    this repository (bench.py), never a scratch script."""
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, f)).read()
        assert "_work" not in text, f
        for block in re.findall(r"```(.*?)```", text, re.S):
            for script in re.findall(r"python\S*\s+(\S+\.py)", block):
                assert os.path.exists(os.path.join(ROOT, script)), (f, script)
