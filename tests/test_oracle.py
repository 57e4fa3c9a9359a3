"""Pins of the CPU oracle against facts fixed by the thesis and by mathematics.

Nothing here uses the GPU path.  Every check compares the oracle with
something other than itself: values printed in the thesis's worked examples,
closed forms, brute force over all subsets, an independent level-wise miner,
library-free recounts, and the published SplitMix64 stream.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2108_05038_gb300 import synth


def csr(txs):
    off = np.zeros(len(txs) + 1, dtype=np.uint32)
    items = []
    for i, t in enumerate(txs):
        items.extend(sorted(set(t)))
        off[i + 1] = len(items)
    return off, np.array(items, dtype=np.uint32)


def as_dict(res):
    so, si, sp = res
    return {tuple(int(v) for v in si[so[i]:so[i + 1]]): int(sp[i]) for i in range(len(sp))}


def brute_dict(txs, N, minsup):
    """Definition written out in Python: all non-empty subsets of the items present."""
    sets = [frozenset(t) for t in txs]
    present = sorted(set().union(*sets)) if sets else []
    out = {}
    for k in range(1, len(present) + 1):
        for c in itertools.combinations(present, k):
            s = sum(1 for t in sets if t.issuperset(c))
            if s >= minsup:
                out[c] = s
    return out


# ---------------------------------------------------------------- golden examples

@pytest.mark.parametrize("miner", [oracle.eclat, oracle.bruteforce, oracle.apriori])
def test_eclat_worked_example(golden, miner):
    """App. B.3.2: the 23 frequent itemsets and supports printed by the Eclat example."""
    minsup, txs, rows = golden("eclat_example.txt")
    off, items = csr(txs)
    got = as_dict(miner(off, items, 6, minsup))
    want = {s: v for f, s, v in rows if f == "F"}
    assert len(want) == 23
    assert got == want
    for f, s, v in rows:
        if f == "I":
            assert v < minsup and s not in got


@pytest.mark.parametrize("miner", [oracle.eclat, oracle.bruteforce, oracle.apriori])
def test_apriori_worked_example_corrected(golden, miner):
    """App. B.1 example database with its printed errors corrected (11 frequent itemsets)."""
    minsup, txs, rows = golden("apriori_example.txt")
    off, items = csr(txs)
    got = as_dict(miner(off, items, 6, minsup))
    want = {s: v for f, s, v in rows if f == "F"}
    assert len(want) == 11
    assert got == want


def test_golden_supports_by_python_definition(golden):
    """The fixtures themselves agree with the definition of support (Ch. 2)."""
    for name in ("eclat_example.txt", "apriori_example.txt"):
        minsup, txs, rows = golden(name)
        sets = [set(t) for t in txs]
        for f, s, v in rows:
            assert sum(1 for t in sets if set(s) <= t) == v
            assert (v >= minsup) == (f == "F")


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_identical_transactions(k):
    """D identical transactions of k items: 2^k - 1 frequent itemsets, each with support D."""
    D = 37
    off, items = csr([list(range(2, 2 + k))] * D)
    for miner in (oracle.eclat, oracle.apriori):
        got = as_dict(miner(off, items, k + 4, D))
        assert len(got) == 2 ** k - 1
        assert set(got.values()) == {D}


def test_disjoint_singletons():
    """Transactions of one item each: only singletons can be frequent."""
    N = 9
    txs = [[t % N] for t in range(100)]
    off, items = csr(txs)
    got = as_dict(oracle.eclat(off, items, N, 1))
    assert all(len(s) == 1 for s in got)
    assert got == {(i,): sum(1 for t in range(100) if t % N == i) for i in range(N)}


def test_minsup_above_D_is_empty():
    w = synth.make_workload("tiny", D=500)
    for miner in (oracle.eclat, oracle.apriori):
        so, si, sp = miner(w["offsets"], w["items"], w["N"], 501)
        assert len(sp) == 0


def test_minsup_zero_rejected():
    off, items = csr([[1, 2]])
    with pytest.raises(ValueError):
        oracle.eclat(off, items, 3, 0)


def test_item_out_of_range_rejected():
    off, items = csr([[1, 7]])
    with pytest.raises(ValueError):
        oracle.eclat(off, items, 5, 1)


def test_two_item_bernoulli_pair_count():
    """Two items in a Bernoulli pattern: supp({0,1}) is the number of rows holding both."""
    rng = np.random.default_rng(5)
    a = rng.random(3000) < 0.6
    b = rng.random(3000) < 0.45
    txs = [[0] * int(x) + [1] * int(y) for x, y in zip(a, b)]
    off, items = csr(txs)
    got = as_dict(oracle.eclat(off, items, 2, 1))
    assert got[(0,)] == int(a.sum()) and got[(1,)] == int(b.sum())
    assert got[(0, 1)] == int((a & b).sum())


def test_duplicate_items_count_once():
    """Set semantics (Def. Transaction): a repeated item inside a transaction counts once."""
    off = np.array([0, 4, 6], dtype=np.uint32)
    items = np.array([1, 1, 2, 2, 1, 1], dtype=np.uint32)
    got = as_dict(oracle.eclat(off, items, 3, 1))
    assert got == {(1,): 2, (2,): 1, (1, 2): 1}


def test_empty_transactions_count_toward_D():
    off, items = csr([[], [1, 2], [], [1]])
    got = as_dict(oracle.eclat(off, items, 3, 2))
    assert got == {(1,): 2}


# ---------------------------------------------------------------- brute force / independent miners

@pytest.mark.parametrize("seed", range(12))
def test_eclat_equals_bruteforce_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    N = int(rng.integers(3, 15))
    D = int(rng.integers(1, 400))
    dens = rng.uniform(0.1, 0.7)
    txs = [list(np.nonzero(rng.random(N) < dens)[0]) for _ in range(D)]
    off, items = csr(txs)
    for minsup in sorted({1, 2, max(1, D // 10), max(1, D // 3)}):
        e = as_dict(oracle.eclat(off, items, N, minsup))
        b = as_dict(oracle.bruteforce(off, items, N, minsup))
        a = as_dict(oracle.apriori(off, items, N, minsup))
        assert e == b == a


def test_bruteforce_equals_python_definition():
    rng = np.random.default_rng(7)
    txs = [list(np.nonzero(rng.random(8) < 0.4)[0]) for _ in range(60)]
    off, items = csr(txs)
    for minsup in (1, 3, 9):
        assert as_dict(oracle.bruteforce(off, items, 8, minsup)) == brute_dict(txs, 8, minsup)


@pytest.mark.parametrize("name,D", [("tiny", 3000), ("dense_deep", 2000)])
def test_eclat_equals_apriori_workloads(name, D):
    w = synth.make_workload(name, D=D)
    ms = synth.abs_minsup(w["rel_minsup"], D)
    e = oracle.eclat(w["offsets"], w["items"], w["N"], ms)
    a = oracle.apriori(w["offsets"], w["items"], w["N"], ms)
    for x, y in zip(e, a):
        assert np.array_equal(x, y)
    assert len(e[2]) > 50


def test_singletons_equal_histogram():
    w = synth.make_workload("sparse_mid", D=20000)
    so, si, sp = oracle.eclat(w["offsets"], w["items"], w["N"], 30)
    hist = np.bincount(w["items"], minlength=w["N"])  # generator writes distinct items per transaction
    single = {int(si[so[i]]): int(sp[i]) for i in range(len(sp)) if so[i + 1] - so[i] == 1}
    assert single == {i: int(c) for i, c in enumerate(hist) if c >= 30}


@pytest.mark.parametrize("seed,prefilter", [(0, 0), (1, 5), (2, 40), (3, 10 ** 6)])
def test_item_order_is_ascending_support_then_id(seed, prefilter):
    """The row order (reading 3: ascending support, ties by id; items below the prefilter dropped), as
    properties: a permutation of exactly the items whose support (library histogram of each
    transaction's distinct items) reaches the prefilter, supports non-decreasing, ties by id."""
    rng = np.random.default_rng(seed)
    N = 60
    txs = [list(rng.integers(0, N, size=rng.integers(0, 12))) for _ in range(800)]  # repeats inside allowed
    off = np.cumsum([0] + [len(t) for t in txs]).astype(np.uint32)  # raw CSR, repeats kept
    items = np.array([v for t in txs for v in t], dtype=np.uint32)
    supp = np.bincount(np.concatenate([np.unique(t) for t in txs if len(t)]), minlength=N)
    order = oracle.item_order(off, items, N, prefilter)
    assert sorted(order.tolist()) == [i for i in range(N) if supp[i] >= prefilter]
    s = supp[order]
    assert np.all(np.diff(s) >= 0)
    assert all(order[k] < order[k + 1] for k in range(len(order) - 1) if s[k] == s[k + 1])


def test_anti_monotone_along_prefixes():
    """Thm. 2.1 on an Eclat output: every set's prefix (minus last item) is output with >= support."""
    w = synth.make_workload("tiny", D=4000)
    d = as_dict(oracle.eclat(w["offsets"], w["items"], w["N"], 40))
    for s, v in d.items():
        if len(s) > 1:
            assert d[s[:-1]] >= v
            for drop in range(len(s)):
                sub = s[:drop] + s[drop + 1:]
                assert d[sub] >= v


# ---------------------------------------------------------------- certificate checker

def test_check_accepts_exact_and_rejects_planted_mistakes():
    w = synth.make_workload("tiny", D=3000)
    ms = 30
    off, items, N = w["offsets"], w["items"], w["N"]
    so, si, sp = oracle.eclat(off, items, N, ms)
    assert oracle.check(off, items, N, ms, so, si, sp)[0] == 0
    # wrong count
    sp2 = sp.copy()
    big = int(np.argmax(np.diff(so.astype(np.int64))))
    sp2[big] += 1
    assert oracle.check(off, items, N, ms, so, si, sp2)[0] in (1, 3)
    # dropped deepest set (its parent then misses a frequent extension)
    keep = np.ones(len(sp), dtype=bool)
    keep[big] = False
    so3 = np.concatenate([[0], np.cumsum(np.diff(so.astype(np.int64))[keep])]).astype(np.uint64)
    si3 = np.concatenate([si[so[i]:so[i + 1]] for i in range(len(sp)) if keep[i]])
    assert oracle.check(off, items, N, ms, so3, si3, sp[keep])[0] == 4
    # dropped singleton
    k1 = [i for i in range(len(sp)) if so[i + 1] - so[i] == 1][3]
    keep = np.ones(len(sp), dtype=bool)
    keep[k1] = False
    so4 = np.concatenate([[0], np.cumsum(np.diff(so.astype(np.int64))[keep])]).astype(np.uint64)
    si4 = np.concatenate([si[so[i]:so[i + 1]] for i in range(len(sp)) if keep[i]])
    assert oracle.check(off, items, N, ms, so4, si4, sp[keep])[0] in (3, 5)


# ---------------------------------------------------------------- counter-based generator

def test_splitmix64_published_stream():
    """SplitMix64 from state 1234567 (reference outputs of Steele et al.'s generator)."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423]
    assert synth.splitmix64_stream(1234567, 3) == want
    assert [oracle.splitmix64_at(1234567, k) for k in range(3)] == want


# ---------------------------------------------------------------- class-cost estimate

def _sample_brute_costs(txs, N, prefilter, rate, rel, seed, limit=0, return_minsup=False):
    """Estimate written out independently: sample by SplitMix64, brute-force mine, tally by first rank;
    the sample minsup doubles while the sample has more than ``limit`` frequent itemsets."""
    D = len(txs)
    supp = np.zeros(N, dtype=np.int64)
    for t in txs:
        for i in set(t):
            supp[i] += 1
    kept = [i for i in range(N) if supp[i] >= prefilter]
    kept.sort(key=lambda i: (supp[i], i))
    rank = {it: r for r, it in enumerate(kept)}
    m = max(math.ceil(rate * D), min(D, math.ceil(math.log(2 / 0.05) / (2 * 0.05 ** 2))))
    ms = max(1, math.ceil(rel * m))
    sample = []
    for k in range(m):
        x = oracle.splitmix64_at(seed, k)
        sample.append([i for i in txs[((x >> 32) * D) >> 32] if i in rank])
    fs = brute_dict(sample, N, ms)
    while limit and len(fs) > limit:
        ms *= 2
        fs = brute_dict(sample, N, ms)
    cnt = np.zeros(len(kept), dtype=np.int64)
    for s in fs:
        cnt[min(rank[i] for i in s)] += 1
    cost = cnt / len(fs) if fs else cnt.astype(float)
    if return_minsup:
        return cost, len(fs), ms
    return cost, len(fs)


@pytest.mark.parametrize("seed", [0, 1, 99])
def test_class_costs_match_independent_restatement(seed):
    rng = np.random.default_rng(seed + 40)
    N, D = 10, 300
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.2, 0.6))[0]) for _ in range(D)]
    off, items = csr(txs)
    for prefilter, rate, rel in ((0, 0.2, 0.1), (20, 0.5, 0.05), (0, 1.0, 0.3)):
        cost, order, nfs = oracle.class_costs(off, items, N, prefilter, rate, rel, seed)
        want, nfs2 = _sample_brute_costs(txs, N, prefilter, rate, rel, seed)
        assert nfs == nfs2
        assert np.array_equal(cost, want)
        keys = sorted(range(len(cost)), key=lambda r: (-cost[r], r))
        assert list(order) == keys


@pytest.mark.parametrize("limit", [1, 40, 150, 1023])
def test_class_costs_sample_limit_doubles_minsup(limit):
    """A sample with more than `limit` frequent itemsets is mined again at twice the minsup until it has no more."""
    rng = np.random.default_rng(7)
    N, D = 10, 400
    txs = [list(np.nonzero(rng.random(N) < 0.55)[0]) for _ in range(D)]
    off, items = csr(txs)
    cost, order, nfs, ms = oracle.class_costs(off, items, N, 0, 1.0, 0.01, 5, limit=limit, return_minsup=True)
    want, nfs2, ms2 = _sample_brute_costs(txs, N, 0, 1.0, 0.01, 5, limit=limit, return_minsup=True)
    assert (nfs, ms) == (nfs2, ms2)
    assert nfs <= limit
    assert np.array_equal(cost, want)
    if limit < 1023:  # minsup 4 (= ceil(0.01 * 400)) keeps almost every subset of 10 dense items
        assert ms > 4
    # limit 0: no doubling
    _, _, nfs0, ms0 = oracle.class_costs(off, items, N, 0, 1.0, 0.01, 5, limit=0, return_minsup=True)
    assert ms0 == 4 and nfs0 == _sample_brute_costs(txs, N, 0, 1.0, 0.01, 5)[1]


def test_sample_floor_is_theorem_size():
    """The sample is never smaller than the Theorem 6.1 size for eps = delta = 0.05 (738 rows), nor than rate * D."""
    assert math.ceil(math.log(2 / 0.05) / (2 * 0.05 ** 2)) == 738


def test_sample_support_within_chernoff_bound():
    """Sec. 6.1: with |D_s| >= ln(2/delta)/(2 eps^2), singleton relative supports err by <= eps w.p. >= 1-delta.

    A 10,000-row sample gives eps = 0.0136 at delta = 0.05; over 40 items and fixed
    seeds, the observed error stays inside the bound for at least 95% of items."""
    w = synth.make_workload("tiny", D=20000)
    off, items = w["offsets"], w["items"]
    D, N = 20000, w["N"]
    full = np.bincount(items, minlength=N) / D
    m = 10000
    eps = math.sqrt(math.log(2 / 0.05) / (2 * m))
    assert abs(eps - 0.0136) < 1e-3
    for seed in (3, 4):
        idx = np.array([(oracle.splitmix64_at(seed, k) >> 32) * D >> 32 for k in range(m)], dtype=np.int64)
        cnt = np.zeros(N)
        for t in idx:
            cnt[items[off[t]:off[t + 1]]] += 1
        err = np.abs(cnt / m - full)
        assert np.mean(err <= eps) >= 0.95


# ---------------------------------------------------------------- generator reproducibility

def test_generator_matches_stored_databases():
    """The seeded generator writes, bit for bit, the databases the stored oracle digests were computed on."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "digests.json")))
    for name, r in ref.items():
        if r["nnz"] > 3_000_000:
            continue  # the large database is checked by the GPU digest test
        w = synth.make_workload(name)
        assert synth.csr_digest(w["offsets"], w["items"]) == r["csr_sha256"], name


def _sample_intersection_costs(txs, N, prefilter, rate, rel, seed):
    """Counts, by running a literal Eclat on the sample in row order, the AND+popcount intersections of
    every one-item-prefix class: level 2 tries each later frequent row, a node [X | E] tries every e in E."""
    D = len(txs)
    supp = np.zeros(N, dtype=np.int64)
    for t in txs:
        for i in set(t):
            supp[i] += 1
    kept = sorted([i for i in range(N) if supp[i] >= prefilter], key=lambda i: (supp[i], i))
    rank = {it: r for r, it in enumerate(kept)}
    m = max(math.ceil(rate * D), min(D, math.ceil(math.log(2 / 0.05) / (2 * 0.05 ** 2))))
    ms = max(1, math.ceil(rel * m))
    sample = []
    for k in range(m):
        x = oracle.splitmix64_at(seed, k)
        sample.append({rank[i] for i in txs[((x >> 32) * D) >> 32] if i in rank})

    def tids(items):
        return {t for t, s in enumerate(sample) if items <= s}

    freq = [r for r in range(len(kept)) if len(tids({r})) >= ms]
    work = np.zeros(len(kept), dtype=np.int64)

    def expand(cls, X, cands):
        surv = []
        for e in cands:
            work[cls] += 1
            if len(tids(X | {e})) >= ms:
                surv.append(e)
        for k, s in enumerate(surv):
            if k + 1 < len(surv):
                expand(cls, X | {s}, surv[k + 1:])

    for pos, r in enumerate(freq):
        expand(r, {r}, freq[pos + 1:])
    total = work.sum()
    return work / total if total else work.astype(float)


@pytest.mark.parametrize("seed", [2, 5])
def test_intersection_costs_match_literal_eclat(seed):
    """The intersection-count class cost (kind 1) equals a literal count made by running Eclat on the sample."""
    rng = np.random.default_rng(seed + 90)
    N, D = 9, 250
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.25, 0.65))[0]) for _ in range(D)]
    off, items = csr(txs)
    for prefilter, rate, rel in ((0, 0.3, 0.1), (15, 0.6, 0.2)):
        cost, order, _ = oracle.class_costs(off, items, N, prefilter, rate, rel, seed, kind=1)
        want = _sample_intersection_costs(txs, N, prefilter, rate, rel, seed)
        assert np.allclose(cost, want, rtol=0, atol=1e-15)
        assert list(order) == sorted(range(len(cost)), key=lambda r: (-cost[r], r))


# ---------------------------------------------------------------- extension supports

def test_extension_supports_worked_example(golden):
    """Every printed support of the App. B.3.2 example (frequent and infrequent rows) is reached as
    supp(P u {c}) for P = the set minus its last item (minus nothing for a singleton: P = {c})."""
    minsup, txs, rows = golden("eclat_example.txt")
    off, items = csr(txs)
    for _f, s, v in rows:
        prefix = s[:-1] if len(s) > 1 else s
        got = oracle.extension_supports(off, items, 6, prefix, [s[-1]])
        assert int(got[0]) == v, (s, v)


@pytest.mark.parametrize("seed", [3, 4])
def test_extension_supports_equal_eclat_outputs(seed):
    """At minsup 1 Eclat outputs every itemset with nonzero support: each extension of an output set
    by any item is either output with that support or absent with support 0."""
    rng = np.random.default_rng(seed)
    N = 12
    txs = [list(rng.choice(N, size=rng.integers(0, 6), replace=False)) for _ in range(300)]
    off, items = csr(txs)
    d = as_dict(oracle.eclat(off, items, N, 1))
    for s in list(d)[:: 7]:
        got = oracle.extension_supports(off, items, N, list(s), np.arange(N))
        for c in range(N):
            want = d.get(tuple(sorted(set(s) | {c})), 0)
            assert int(got[c]) == want, (s, c)


def test_extension_supports_closed_forms():
    """An item in every transaction: supp({0, c}) = supp(c); a candidate inside P gives supp(P);
    disjoint halves give 0; repeats inside a transaction or P count once."""
    D, N = 500, 9
    rng = np.random.default_rng(11)
    txs = [[0] + list(rng.choice(np.arange(1, N), size=rng.integers(0, 4), replace=False)) for _ in range(D)]
    off, items = csr(txs)
    hist = np.bincount(items, minlength=N)
    assert list(oracle.extension_supports(off, items, N, [0], np.arange(N))) == list(hist)
    assert list(oracle.extension_supports(off, items, N, [0, 0], [0, 0])) == [D, D]
    lo = [[1, 2]] * 5 + [[3, 4, 4]] * 7 + [[]] * 2  # raw CSR: the repeated 4 stays in
    off2 = np.cumsum([0] + [len(t) for t in lo]).astype(np.uint32)
    items2 = np.array([i for t in lo for i in t], dtype=np.uint32)
    assert list(oracle.extension_supports(off2, items2, 5, [1], [2, 3, 4])) == [5, 0, 0]
    assert list(oracle.extension_supports(off2, items2, 5, [4, 4], [3, 4, 1])) == [7, 7, 0]
    with pytest.raises(ValueError):
        oracle.extension_supports(off2, items2, 5, [], [1])
    with pytest.raises(ValueError):
        oracle.extension_supports(off2, items2, 5, [1], [5])


# ---------------------------------------------------------------- threaded driver

@pytest.mark.parametrize("threads", [1, 2, 5, 64])
def test_threaded_eclat_equals_sequential(threads):
    """The threaded driver runs the same recursion per one-item class: identical canonical output,
    also with more threads than classes."""
    for name, D in (("tiny", 4000), ("dense_deep", 3000)):
        w = synth.make_workload(name, D=D)
        ms = synth.abs_minsup(w["rel_minsup"], D)
        a = oracle.eclat(w["offsets"], w["items"], w["N"], ms)
        b = oracle.eclat_mt(w["offsets"], w["items"], w["N"], ms, threads)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    rng = np.random.default_rng(threads)
    txs = [list(rng.choice(15, size=rng.integers(0, 8), replace=False)) for _ in range(200)]
    off, items = csr(txs)
    assert as_dict(oracle.eclat_mt(off, items, 15, 2, threads)) == brute_dict(txs, 15, 2)


# ---------------------------------------------------------------- closed and maximal itemsets

def _brute_closed_maximal(txs, N, minsup):
    """Definitions written out over all subsets: closure = items of every transaction containing the set."""
    sets = [frozenset(t) for t in txs]
    d = brute_dict(txs, N, minsup)
    out = {}
    for s, v in d.items():
        cover = [t for t in sets if set(s) <= t]
        closure = frozenset.intersection(*cover) if cover else frozenset()
        closed = closure == frozenset(s)
        maximal = not any(set(s) < set(o) for o in d)
        out[s] = (1 if closed else 0) | (2 if maximal else 0)
    return out


def _flags_dict(res):
    so, si, sp, fl = res
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(fl[k]) for k in range(len(sp))}


@pytest.mark.parametrize("seed", range(6))
def test_closed_maximal_equal_definitions_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    N = int(rng.integers(3, 11))
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.2, 0.8))[0]) for _ in range(int(rng.integers(5, 60)))]
    off, items = csr(txs)
    for minsup in (1, 2, max(1, len(txs) // 4)):
        assert _flags_dict(oracle.closed_maximal(off, items, N, minsup)) == _brute_closed_maximal(txs, N, minsup)


def test_closed_maximal_closed_forms():
    """k identical transactions: only the full set is closed and maximal; nested transactions
    {0} c {0,1} c {0,1,2}: every prefix closed (supports 3, 2, 1), only the longest maximal at minsup 1;
    disjoint singletons: each both."""
    off, items = csr([[0, 1, 2, 3]] * 5)
    f = _flags_dict(oracle.closed_maximal(off, items, 4, 5))
    assert f[(0, 1, 2, 3)] == 3 and all(v == 0 for k, v in f.items() if k != (0, 1, 2, 3))
    off, items = csr([[0], [0, 1], [0, 1, 2]])
    f = _flags_dict(oracle.closed_maximal(off, items, 3, 1))
    assert f[(0,)] == 1 and f[(0, 1)] == 1 and f[(0, 1, 2)] == 3 and f[(1,)] == 0 and f[(1, 2)] == 0
    off, items = csr([[0], [1], [2]])
    assert set(_flags_dict(oracle.closed_maximal(off, items, 3, 1)).values()) == {3}
