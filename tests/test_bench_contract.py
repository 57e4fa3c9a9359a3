"""bench.py's reference arm on the CPU: the oracle on every host core, one JSON line with the
contract's keys; ranks other than 0 print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                           "--steps", "2", "--warmup", "3"], capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_json_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "tidset AND+popc GB/s" and d["unit"] == "GB/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == d["value"]
    assert isinstance(cb["cpu"], str) and cb["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "tiny" in d["config"]["workload"]


def test_reference_arm_other_ranks_are_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def _literal_bitmap_work(off, items, N, minsup):
    """Runs the bitmap Eclat literally, in row order (ascending support, ties by id), counting every
    support test (intersection), every class node that tests at least one candidate, and every prefix
    of two or more items whose bitmap is formed because it has at least two frequent extensions."""
    import numpy as np

    D = len(off) - 1
    supp = np.zeros(N, dtype=np.int64)
    tids = [set() for _ in range(N)]
    for t in range(D):
        for i in set(int(v) for v in items[off[t]:off[t + 1]]):
            tids[i].add(t)
            supp[i] += 1
    order = sorted(range(N), key=lambda i: (supp[i], i))  # row r holds item order[r]
    rows = [tids[i] for i in order]
    freq = [r for r in range(N) if len(rows[r]) >= minsup]
    count = {"I": 0, "C": 0, "M": 0}

    def node(X, tX, cands):
        if not cands:
            return
        count["C"] += 1
        surv = []
        for e in cands:
            count["I"] += 1
            t = tX & rows[e]
            if len(t) >= minsup:
                surv.append((e, t))
        if len(X) >= 2 and len(surv) >= 2:
            count["M"] += 1
        for k, (e, t) in enumerate(surv):
            node(X + (e,), t, [f for f, _ in surv[k + 1:]])

    for p, r in enumerate(freq):
        node((r,), rows[r], freq[p + 1:])
    return count["I"], count["C"], count["M"]


def test_algorithmic_work_counts_equal_a_literal_run():
    """The bench's unit of work (intersections, class nodes with candidates, materialised prefixes),
    recomputed from an oracle output alone, equals what a literal bitmap Eclat performs."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle

    rng = np.random.default_rng(7)
    for trial in range(6):
        N, D = int(rng.integers(3, 14)), int(rng.integers(20, 300))
        dens = rng.uniform(0.15, 0.7)
        txs = [np.nonzero(rng.random(N) < dens)[0] for _ in range(D)]
        off = np.cumsum([0] + [len(t) for t in txs]).astype(np.uint32)
        items = np.concatenate([t for t in txs] + [np.zeros(0, dtype=np.int64)]).astype(np.uint32)
        for minsup in (1, max(1, D // 6), max(1, D // 3)):
            so, si, _ = oracle.eclat(off, items, N, minsup)
            order = oracle.item_order(off, items, N, 0)
            rank = np.zeros(N, dtype=np.int64)
            rank[order] = np.arange(len(order))
            assert bench.bitmap_work(so, si, rank) == _literal_bitmap_work(off, items, N, minsup), (trial, minsup)


def test_cpu_baseline_record():
    """The main arm's cpu_baseline: the oracle on every host core and on one, medians of up to 5 runs,
    the host CPU named, in the metric's units."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2108_05038_gb300 import synth

    w = synth.make_workload("tiny")
    w["name"] = "tiny"
    bytes_alg, _ = bench.oracle_bytes(w["offsets"], w["items"], w["N"], w["D"], w["minsup"], w["word_bits"])
    cb = bench.cpu_baseline(w, bytes_alg, "tiny")
    assert cb["kind"] == "oracle" and cb["unit"] == "GB/s" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_core"]["value"] > 0 and cb["single_core"]["cores"] == 1
    assert "medians of" in cb["sample"] and "2624 itemsets" in cb["sample"] and cb["cpu"]


def test_result_digest_is_order_free_and_separates_results():
    """The serving comparison's per-request digest: the same itemsets and supports in any record order give
    the same digest; one support or one item changed gives another."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    class R:
        def __init__(self, sets):
            self.n_sets = len(sets)
            self.set_offsets = np.cumsum([0] + [len(s) for s, _ in sets]).astype(np.uint64)
            self.set_items = np.array([v for s, _ in sets for v in s], dtype=np.uint32)
            self.supports = np.array([c for _, c in sets], dtype=np.uint32)

    sets = [((1,), 50), ((2,), 40), ((1, 2), 30), ((1, 2, 7), 12), ((3,), 40)]
    d = bench.result_digest(R(sets))
    assert d[0] == 5
    assert bench.result_digest(R(sets[::-1])) == d
    assert bench.result_digest(R(sets[:3] + [((1, 2, 7), 13)] + sets[4:])) != d
    assert bench.result_digest(R(sets[:3] + [((1, 2, 8), 12)] + sets[4:])) != d
    assert bench.result_digest(R([])) == (0, 0)


def test_traffic_records_follow_the_sources():
    """A DRAM-traffic record is reported only while the CUDA sources hash to the value it was captured with."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.sources_sha256()
    assert len(h) == 64 and h == bench.sources_sha256()
    for name, rec in bench.CAPTURES.items():
        assert set(rec) >= {"sources_sha256", "date", "summary", "kernels", "step"}
        assert os.path.exists(os.path.join(ROOT, rec["summary"]))
        # the summary the record cites is the one of the same capture (it names the sources' hash)
        with open(os.path.join(ROOT, rec["summary"])) as f:
            assert rec["sources_sha256"][:12] in f.read(), (name, rec["summary"])
    saved = dict(bench.CAPTURES)
    try:
        bench.CAPTURES["x"] = {"sources_sha256": "0" * 64, "date": "d", "summary": "s", "kernels": {}, "step": 1}
        rec, why = bench.captured("x")
        assert rec is None and "changed" in why
        bench.CAPTURES["x"]["sources_sha256"] = h
        rec, why = bench.captured("x")
        assert rec is not None and h[:12] in why
        assert bench.captured("nothing")[0] is None
    finally:
        bench.CAPTURES.clear()
        bench.CAPTURES.update(saved)
