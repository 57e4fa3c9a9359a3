"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Counts are integers, so the bar is bit-exact: the same set of itemsets and the
same supports.  The output order of the GPU is unspecified; sets are compared
as canonical dictionaries (items ascending inside a set).
"""
import json
import math
import time
import os

import numpy as np
import pytest

import canon
import oracle
from paper_2108_05038_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2108_05038_gb300 import fim  # noqa: E402


def csr(txs):
    off = np.zeros(len(txs) + 1, dtype=np.uint32)
    items = []
    for i, t in enumerate(txs):
        items.extend(sorted(set(int(v) for v in t)))
        off[i + 1] = len(items)
    return off, np.array(items, dtype=np.uint32)


def odict(res):
    so, si, sp = res
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(len(sp))}


def gpu_mine(off, items, N, minsup, word_bits=64, prefilter=0, **kw):
    """Build + mine through the C ABI (kw: fim_mine options)."""
    db = fim.build_vertical_db(off, items, N, word_bits=word_bits, prefilter_minsup=prefilter)
    try:
        return db.mine(minsup, **kw)
    finally:
        db.free()


def assert_same(got: dict, want: dict):
    if got != want:
        missing = [k for k in want if k not in got][:5]
        extra = [k for k in got if k not in want][:5]
        wrong = [(k, got[k], want[k]) for k in want if k in got and got[k] != want[k]][:5]
        raise AssertionError(f"{len(got)} vs {len(want)} itemsets; missing {missing} extra {extra} wrong {wrong}")


# ---------------------------------------------------------------- golden and tiny cases

def test_eclat_worked_example_on_gpu(golden):
    minsup, txs, rows = golden("eclat_example.txt")
    off, items = csr(txs)
    for wb in (32, 64):
        got = gpu_mine(off, items, 6, minsup, word_bits=wb).as_dict()
        assert_same(got, {s: v for f, s, v in rows if f == "F"})


@pytest.mark.parametrize("seed", range(16))
def test_random_tiny_vs_bruteforce(seed):
    rng = np.random.default_rng(1000 + seed)
    N = int(rng.integers(2, 15))
    D = int(rng.integers(1, 700))
    dens = rng.uniform(0.05, 0.8)
    txs = [list(np.nonzero(rng.random(N) < dens)[0]) for _ in range(D)]
    off, items = csr(txs)
    for minsup in sorted({1, 2, max(1, D // 7), max(1, D // 2)}):
        want = odict(oracle.bruteforce(off, items, N, minsup))
        got = gpu_mine(off, items, N, minsup, word_bits=32 if seed % 2 else 64,
                       dfs_mode=(0, 1, 3, 4, 5)[(seed // 2) % 5]).as_dict()
        assert_same(got, want)


@pytest.mark.parametrize("D", [1, 31, 32, 33, 63, 64, 65, 1000, 4096 + 37])
def test_ragged_D(D):
    """D not a multiple of the word / row padding: tail bits stay zero."""
    rng = np.random.default_rng(D)
    txs = [list(np.nonzero(rng.random(12) < 0.6)[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = max(1, D // 5)
    assert_same(gpu_mine(off, items, 12, minsup).as_dict(), odict(oracle.eclat(off, items, 12, minsup)))


@pytest.mark.parametrize("k,mode,depth", [(11, 0, 0), (16, 0, 8), (11, 1, 4), (16, 1, 0), (11, 3, 0), (16, 3, 4),
                                          (11, 4, 0), (16, 4, 4), (11, 5, 0), (16, 5, 4)])
def test_identical_transactions_closed_form(k, mode, depth):
    """2^k - 1 itemsets of support D; with a first DFS stack of 4 or 8 the depth of 9 or 14 forces the
    regrown retry, with 0 the stack has the full depth at once."""
    D = 300
    off, items = csr([list(range(k))] * D + [[k]])
    got = gpu_mine(off, items, k + 1, D, dfs_mode=mode, dfs_depth_first=depth).as_dict()
    assert len(got) == 2 ** k - 1 and set(got.values()) == {D}


@pytest.mark.parametrize("mode", [0, 1, 3, 4, 5])
def test_single_and_empty_transactions(mode):
    """One transaction of 5 items: every non-empty subset (31) with support 1; only empty transactions:
    nothing is frequent (no item has support); one item in every transaction: only that singleton."""
    off, items = csr([[4, 0, 2, 3, 1]])
    got = gpu_mine(off, items, 5, 1, dfs_mode=mode).as_dict()
    assert len(got) == 31 and set(got.values()) == {1}
    off, items = csr([[] for _ in range(100)])
    assert gpu_mine(off, items, 7, 1, dfs_mode=mode).n_sets == 0
    off, items = csr([[3]] * 40)
    assert gpu_mine(off, items, 8, 40, dfs_mode=mode).as_dict() == {(3,): 40}


def test_many_items_global_histogram():
    """N = 20,000 items (above the 12,288 counted in shared memory per CTA): counts from global atomics."""
    rng = np.random.default_rng(31)
    D, N = 3000, 20000
    hot = rng.choice(N, 30, replace=False)
    txs = [list(set(rng.choice(N, 5).tolist()) | set(hot[rng.random(30) < 0.3].tolist())) for _ in range(D)]
    off, items = csr(txs)
    want = odict(oracle.eclat(off, items, N, 40))
    assert_same(gpu_mine(off, items, N, 40).as_dict(), want)


def test_degenerate_cases():
    off, items = csr([[0], [1], [2], [0, 1]])
    assert gpu_mine(off, items, 3, 5).n_sets == 0             # minsup > D: empty
    assert gpu_mine(off, items, 3, 2).as_dict() == {(0,): 2, (1,): 2}  # {0,1} has support 1
    off, items = csr([[], [], [4]])
    assert gpu_mine(off, items, 5, 1).as_dict() == {(4,): 1}  # empty transactions count toward D
    off, items = csr([[1, 2]] * 3)
    assert gpu_mine(off, items, 3, 3).as_dict() == {(1,): 3, (2,): 3, (1, 2): 3}  # n1 = 2: no DFS launch


def test_duplicate_items_count_once():
    off = np.array([0, 4, 6], dtype=np.uint32)
    items = np.array([1, 1, 2, 2, 1, 1], dtype=np.uint32)
    assert gpu_mine(off, items, 3, 1).as_dict() == {(1,): 2, (2,): 1, (1, 2): 1}


def test_item_supports_with_repeats_in_any_order():
    """Set semantics of the item count (Ch. 2: a transaction supports an item once) on 2,000 transactions of
    0-200 ids drawn with replacement: short ones (counted by one thread each) sorted or not, with repeats,
    and long ones (more than 64 ids, counted by a warp) with repeats across 32-id chunks.  Minsup 60 keeps
    the 1,500 singletons (about 133 transactions each) and no pair (about 9 on average)."""
    rng = np.random.default_rng(12)
    N, D = 1500, 2000
    lens = rng.integers(0, 201, D)
    off = np.zeros(D + 1, dtype=np.uint32)
    off[1:] = np.cumsum(lens)
    items = rng.integers(0, N, int(off[-1])).astype(np.uint32)
    for d in range(0, D, 3):
        items[off[d]:off[d + 1]].sort()
    want = odict(oracle.eclat(off, items, N, 60))
    assert len(want) == N and all(len(k) == 1 for k in want)
    assert_same(gpu_mine(off, items, N, 60).as_dict(), want)


def test_invalid_inputs():
    off, items = csr([[1, 7]])
    with pytest.raises(fim.FimError) as e:
        fim.build_vertical_db(off, items, 5)
    assert e.value.status == fim.FIM_ERR_INVALID
    off, items = csr([[1, 2]])
    db = fim.build_vertical_db(off, items, 3)
    with pytest.raises(fim.FimError) as e:
        db.mine(0)
    assert e.value.status == fim.FIM_ERR_INVALID
    with pytest.raises(fim.FimError):
        db.estimate_class_costs(0.0, 0.1, 1)
    db.free()


@pytest.mark.parametrize("offsets,why", [([0, 100, 5], "non-decreasing"), ([3, 4, 5], "[0] must be 0"),
                                         ([0, 6, 5], "non-decreasing")])
def test_invalid_device_offsets_rejected_before_reading_items(offsets, why):
    """Device input: a range past tx_offsets[D] or a nonzero first offset is reported, and the count kernel
    reads no item past tx_offsets[D] (the items buffer holds exactly 5 ids here)."""
    d_off = torch.tensor(offsets, dtype=torch.int32, device="cuda")
    d_it = torch.tensor([0, 1, 2, 1, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(fim.FimError) as e:
        fim.build_vertical_db_device(d_off, d_it, len(offsets) - 1, 3)
    assert e.value.status == fim.FIM_ERR_INVALID and why in str(e.value)
    ok = fim.build_vertical_db_device(torch.tensor([0, 2, 5], dtype=torch.int32, device="cuda"), d_it, 2, 3)
    assert ok.mine(1).as_dict() == {(0,): 2, (1,): 2, (2,): 1, (0, 1): 2, (0, 2): 1, (1, 2): 1, (0, 1, 2): 1}
    ok.free()


# ---------------------------------------------------------------- named workloads

@pytest.mark.parametrize("name,mode", [("tiny", 0), ("dense_deep", 0), ("dense_exact37", 0), ("tiny", 1), ("tiny", 4),
                                       ("dense_deep", 1), ("tiny", 3), ("dense_deep", 3), ("tiny", 5),
                                       ("dense_deep", 5)])
def test_workload_full_size_exact(name, mode):
    w = synth.make_workload(name)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], w["minsup"]))
    got = gpu_mine(w["offsets"], w["items"], w["N"], w["minsup"], word_bits=w["word_bits"], dfs_mode=mode).as_dict()
    assert_same(got, want)


@pytest.mark.parametrize("mode", [0, 1, 3, 5])
def test_sparse_mid_full_size_exact(mode):
    w = synth.make_workload("sparse_mid")
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], w["minsup"]))
    res = gpu_mine(w["offsets"], w["items"], w["N"], w["minsup"], word_bits=64, dfs_mode=mode)
    assert_same(res.as_dict(), want)
    st = res.stats
    assert st["n_frequent"] == len(want)
    assert st["n_pair_intersections"] == st["n_frequent_items"] * (st["n_frequent_items"] - 1) // 2


@pytest.mark.parametrize("threads,vec,donate,order,mode", [(128, 1, True, "uniform", 0), (256, 2, False, "uniform", 0),
                                                             (512, 8, True, "estimate", 0),
                                                             (512, 4, False, "estimate", 0),
                                                             (128, 1, False, "uniform", 1), (256, 4, False, "estimate", 1),
                                                             (512, 8, False, "estimate", 1), (128, 4, False, "estimate", 3),
                                                             (256, 8, False, "uniform", 3), (512, 2, False, "estimate", 3)])
def test_launch_shapes_and_orders_identical(threads, vec, donate, order, mode):
    """Item order, class order, CTA shape and donation never change the output (Sec. 8.2)."""
    w = synth.make_workload("dense_deep", D=20000)
    ms = 12000
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    if order == "estimate":
        db.estimate_class_costs(0.02, 0.6, 5)
    got = db.mine(ms, class_order=order, threads_per_cta=threads, vec_per_lane=vec, donate=donate,
                  dfs_mode=mode).as_dict()
    db.free()
    assert_same(got, want)


def test_sparse_mode_mixes_listed_and_dense_prefixes():
    """300,000 transactions: five items in ~90% of them give prefixes with more nonzero words than a
    shared-memory list holds (dense, counted from the stack), 25 items in ~0.5% give listed ones;
    every DFS mode gives the oracle's answer."""
    rng = np.random.default_rng(17)
    D = 300_000
    dense = rng.random((D, 5)) < 0.9
    sparse = rng.random((D, 25)) < 0.005
    txs = [list(np.nonzero(dense[t])[0]) + list(5 + np.nonzero(sparse[t])[0]) for t in range(D)]
    off, items = csr(txs)
    ms = 300
    want = odict(oracle.eclat(off, items, 30, ms))
    for mode in (3, 0, 1):
        assert_same(gpu_mine(off, items, 30, ms, dfs_mode=mode).as_dict(), want)


def test_pair_lists_for_sparse_leading_rows():
    """150,000 transactions, 150 rare items co-occurring in fixed pairs (supports ~200, below a quarter
    of the 1,176 16-byte words of a row: their pairs are counted from nonzero-word lists) and 50 common
    ones (tiles); the counts, and so the itemsets, equal the oracle's."""
    rng = np.random.default_rng(29)
    D = 150_000
    common = rng.random((D, 50)) < rng.uniform(0.02, 0.1, 50)
    pat = np.where(rng.random(D) < 0.1, rng.integers(0, 75, D), -1)
    txs = []
    for t in range(D):
        tx = list(150 + np.nonzero(common[t])[0])
        if pat[t] >= 0:
            tx += [2 * int(pat[t]), 2 * int(pat[t]) + 1]
        txs.append(tx)
    off, items = csr(txs)
    ms = 50
    want = odict(oracle.eclat(off, items, 200, ms))
    assert any(k == (0, 1) for k in want)  # rare pairs are frequent
    for mode in (2, 0):
        assert_same(gpu_mine(off, items, 200, ms, dfs_mode=mode).as_dict(), want)


def test_work_counters_match_output_and_modes():
    """Intersections, class nodes and materialised prefixes reported by both DFS modes equal the counts
    derived from the oracle's output alone (bench.bitmap_work)."""
    import bench
    w = synth.make_workload("dense_deep", D=30000)
    ms = 18000
    so, si, sp = oracle.eclat(w["offsets"], w["items"], w["N"], ms)
    order = oracle.item_order(w["offsets"], w["items"], w["N"], 0)
    rank = np.zeros(w["N"], dtype=np.int64)
    rank[order] = np.arange(len(order))
    I, Cn, M = bench.bitmap_work(so, si, rank)
    for mode in (0, 1, 3, 4):
        st = gpu_mine(w["offsets"], w["items"], w["N"], ms, dfs_mode=mode).stats
        assert st["n_intersections"] == I
        rb = (30000 + 63) // 64 * 8
        assert st["bytes_algorithmic"] == (I + Cn + M) * rb


def test_prefilter_and_device_input():
    w = synth.make_workload("tiny", D=6000)
    ms = 90
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    assert_same(gpu_mine(w["offsets"], w["items"], w["N"], ms, prefilter=50).as_dict(), want)
    d_off = torch.from_numpy(w["offsets"].astype(np.int32)).cuda()
    d_it = torch.from_numpy(w["items"].astype(np.int32)).cuda()
    torch.cuda.synchronize()
    db = fim.build_vertical_db_device(d_off, d_it, 6000, w["N"], 32, 0)
    got = db.mine(ms).as_dict()
    db.free()
    assert_same(got, want)


def test_fixed_capacity_overflow_then_retry():
    w = synth.make_workload("tiny", D=5000)
    ms = 50
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    with pytest.raises(fim.FimError) as e:
        db.mine(ms, out_capacity_sets=100, out_capacity_items=150)
    assert e.value.status == fim.FIM_ERR_OUTPUT_OVERFLOW
    need_sets, need_items = e.value.needed
    assert need_sets == len(want) and need_items == sum(len(k) for k in want)
    got = db.mine(ms, out_capacity_sets=need_sets, out_capacity_items=need_items).as_dict()
    db.free()
    assert_same(got, want)


@pytest.mark.parametrize("mode", [0, 1, 3, 4, 5])
def test_itemset_limit_aborts_early(mode):
    """max_itemsets stops the mine once the output passes it (FIM_ERR_OUTPUT_OVERFLOW); the db stays usable."""
    off, items = csr([list(range(20))] * 50 + [[20]])
    db = fim.build_vertical_db(off, items, 21)
    with pytest.raises(fim.FimError) as e:
        db.mine(2, max_itemsets=5000, dfs_mode=mode)
    assert e.value.status == fim.FIM_ERR_OUTPUT_OVERFLOW
    got = db.mine(50, dfs_mode=mode).as_dict()
    db.free()
    assert len(got) == 2 ** 20 - 1


@pytest.mark.parametrize("mode", [0, 1, 3, 4, 5])
def test_output_regrowth_reuses_pair_counts(mode):
    """2^20 - 1 itemsets of length up to 20 overflow the first output buffer and a 3-deep first DFS
    stack: the repeated runs skip the pair kernel (its counts stay in the workspace) and still give
    the exact closed-form answer."""
    off, items = csr([list(range(20))] * 50 + [[20]])
    db = fim.build_vertical_db(off, items, 21)
    res = db.mine(50, dfs_mode=mode, collect_times=True, dfs_depth_first=3)  # depth 20 > 3: stack grows too
    st = res.stats
    got = res.as_dict()
    db.free()
    assert len(got) == 2 ** 20 - 1 and all(v == 50 for v in got.values())
    assert st["ms_pair_kernel"] > 0 and st["ms_device_total"] >= st["ms_dfs_kernel"] > 0


@pytest.mark.parametrize("mode", [0, 1, 3, 4, 5])
def test_cta_busy_times_are_consistent(mode):
    """collect_times records every persistent CTA's resident time: 0 < mean <= max <= the kernel's time."""
    w = synth.make_workload("dense_deep", D=20_000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    st = db.mine(12_000, dfs_mode=mode, collect_times=True).stats
    db.free()
    assert 0 < st["dfs_cta_busy_mean_ms"] <= st["dfs_cta_busy_max_ms"] <= st["ms_dfs_kernel"] * 1.05 + 0.01


def _literal_class_work(txs, N, minsup):
    """Intersections per one-row class of a literal Eclat in the row order (ascending support, ties by id):
    level 2 tries every later frequent row, a node [X | E] tries every e in E, and a child is expanded
    when it has a later survivor."""
    supp = np.zeros(N, dtype=np.int64)
    sets = [set(t) for t in txs]
    for t in sets:
        for i in t:
            supp[i] += 1
    rows = sorted(range(N), key=lambda i: (supp[i], i))
    sets = [{rows.index(i) for i in t} for t in sets]

    def sup(X):
        return sum(1 for t in sets if X <= t)

    freq = [r for r in range(N) if sup({r}) >= minsup]
    work = np.zeros(N, dtype=np.uint64)

    def expand(cls, X, cands):
        surv = []
        for e in cands:
            work[cls] += 1
            if sup(X | {e}) >= minsup:
                surv.append(e)
        for k, e in enumerate(surv):
            if k + 1 < len(surv):
                expand(cls, X | {e}, surv[k + 1:])

    for pos, r in enumerate(freq):
        expand(r, {r}, freq[pos + 1:])
    return work


@pytest.mark.parametrize("seed,mode", [(0, 0), (1, 1), (2, 0), (3, 1), (4, 3), (5, 3), (6, 4), (7, 4), (8, 5),
                                       (9, 5)])
def test_class_work_matches_literal_eclat(seed, mode):
    """class_work_out: intersections per one-row class equal a literal Eclat's count, and sum to the total."""
    rng = np.random.default_rng(700 + seed)
    N, D = 12, 400
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.2, 0.7))[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = int(rng.integers(15, 60))
    db = fim.build_vertical_db(off, items, N, word_bits=32 if seed % 2 else 64)
    res = db.mine(minsup, dfs_mode=mode, class_work=True)
    db.free()
    want = _literal_class_work(txs, N, minsup)
    assert np.array_equal(res.class_work, want)
    assert int(res.class_work.sum()) == res.stats["n_intersections"]


def test_workspaces_pass_between_databases():
    """A freed database's device workspace serves the next build (larger, smaller, other data): every
    result stays exact."""
    for name, D, ms in (("sparse_mid", 30_000, 75), ("tiny", 4000, 40), ("dense_deep", 20_000, 12_000),
                        ("sparse_mid", 60_000, 150), ("tiny", 2000, 20)):
        w = synth.make_workload(name, D=D)
        want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
        db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
        db.estimate_class_costs(0.05, ms / D, 3)
        got = db.mine(ms).as_dict()
        db.free()
        assert_same(got, want)


def test_repeated_mines_reuse_workspace():
    w = synth.make_workload("tiny", D=8000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    for ms in (400, 80, 200, 80):
        assert_same(db.mine(ms).as_dict(), odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms)))
    db.free()


# ---------------------------------------------------------------- class-cost estimate

@pytest.mark.parametrize("name,D,rate,rel,seed", [("tiny", 10000, 0.05, 0.01, 3), ("dense_deep", 20000, 0.01, 0.6, 9),
                                                   ("sparse_mid", 50000, 0.02, 0.005, 1)])
def test_estimate_matches_oracle(name, D, rate, rel, seed):
    w = synth.make_workload(name, D=D)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    cost, order = db.estimate_class_costs(rate, rel, seed)
    nfs, m, ms = db.estimate_sample_size()
    db.free()
    ocost, oorder, onfs = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, rate, rel, seed)
    assert m == max(math.ceil(rate * D), min(D, 738)) and nfs == onfs
    assert np.array_equal(cost, ocost)
    assert np.array_equal(order, oorder)


@pytest.mark.parametrize("name,D,rate,rel,seed", [("tiny", 10000, 0.05, 0.01, 3), ("dense_deep", 20000, 0.02, 0.6, 4),
                                                   ("sparse_mid", 50000, 0.02, 0.005, 1)])
def test_intersection_cost_estimate_matches_oracle(name, D, rate, rel, seed):
    w = synth.make_workload(name, D=D)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    cost, order = db.estimate_class_costs(rate, rel, seed, cost="intersections")
    db.free()
    ocost, oorder, _ = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, rate, rel, seed, kind=1)
    assert np.array_equal(cost, ocost)
    assert np.array_equal(order, oorder)


@pytest.mark.parametrize("rel,limit,kind", [(0.2, 20000, "itemsets"), (0.3, 20000, "intersections"),
                                            (0.45, 300, "itemsets"), (0.6, 0, "intersections")])
def test_estimate_sample_limit_matches_oracle(rel, limit, kind):
    """The sample minsup doubles while the sample has more than `limit` frequent itemsets, as in the oracle
    (dense_deep, 8,000 rows: 148 -> 592, 222 -> 444, 333 -> 666, and no limit at 443)."""
    w = synth.make_workload("dense_deep", D=8000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    cost, order = db.estimate_class_costs(0.05, rel, 11, cost=kind, max_sample_itemsets=limit)
    nfs, m, ms = db.estimate_sample_size()
    db.free()
    k = {"itemsets": 0, "intersections": 1}[kind]
    ocost, oorder, onfs, oms = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, 0.05, rel, 11, kind=k,
                                                  limit=limit, return_minsup=True)
    assert (nfs, ms) == (onfs, oms)
    assert np.array_equal(cost, ocost)
    assert np.array_equal(order, oorder)


def test_estimate_of_exploding_sample_is_bounded():
    """minsup 0.1% on 30-of-100-item transactions, 30% of them holding an 18-item core: at the start
    minsup (1) the sample's itemsets explode; the limit doubles the sample minsup until the sample mines
    within it.  Limit 2^16: parity with the oracle (1 -> 256, 128 itemsets); default limit: bounded time."""
    rng = np.random.default_rng(3)
    N, D = 100, 20000
    txs = [list(rng.choice(N, size=30, replace=False)) for _ in range(D)]
    for t in txs[: int(D * 0.3)]:
        t[:] = sorted(set(t) | set(range(18)))
    off, items = csr(txs)
    db = fim.build_vertical_db(off, items, N)
    cost, order = db.estimate_class_costs(0.01, 0.001, 2, max_sample_itemsets=1 << 16)
    nfs, m, ms = db.estimate_sample_size()
    ocost, oorder, onfs, oms = oracle.class_costs(off, items, N, 0, 0.01, 0.001, 2, limit=1 << 16,
                                                  return_minsup=True)
    assert (nfs, ms) == (onfs, oms) and ms > 1
    assert np.array_equal(cost, ocost) and np.array_equal(order, oorder)
    t0 = time.perf_counter()
    db.estimate_class_costs(0.01, 0.001, 2)
    dt = time.perf_counter() - t0
    nfs, m, ms = db.estimate_sample_size()
    db.free()
    assert nfs <= fim.SAMPLE_ITEMSET_LIMIT and ms > 1
    assert dt < 20.0


def test_row_order_matches_oracle():
    w = synth.make_workload("sparse_mid", D=20000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], prefilter_minsup=3)
    ri, sp = db.rows()
    db.free()
    assert np.array_equal(ri, oracle.item_order(w["offsets"], w["items"], w["N"], 3))
    assert np.all(np.diff(sp.astype(np.int64)) >= 0)


@pytest.mark.parametrize("name,D,ms", [("sparse_mid", 30000, 80), ("dense_deep", 20000, 12000)])
def test_output_independent_of_sample_rate_and_seed(name, D, ms):
    """The estimate only orders the classes (Sec. 8.2): after estimates at different sample rates,
    seeds, relative minsups and cost measures, every mine returns the oracle's itemsets."""
    w = synth.make_workload(name, D=D)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        for rate, seed, rel, cost in [(0.005, 1, ms / D, "itemsets"), (0.05, 7, ms / D, "itemsets"),
                                      (1.0, 2, ms / D, "intersections"), (0.01, 3, 1.5 * ms / D, "itemsets")]:
            db.estimate_class_costs(rate, rel, seed, cost=cost)
            assert_same(db.mine(ms).as_dict(), want)
    finally:
        db.free()


# ---------------------------------------------------------------- full sizes against stored oracle digests

DIGESTS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "digests.json")))


@pytest.mark.parametrize("name", sorted(DIGESTS))
def test_full_size_digest(name):
    """Every named workload at full size: the generated database is the one the oracle mined
    (CSR SHA-256), and the GPU's canonical output hashes to the oracle's (tests/golden/make_digests.py)."""
    ref = DIGESTS[name]
    w = synth.make_workload(name)
    assert synth.csr_digest(w["offsets"], w["items"]) == ref["csr_sha256"]
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=w["word_bits"])
    db.estimate_class_costs(0.01, w["rel_minsup"], 3)
    res = db.mine(w["minsup"])
    db.free()
    assert canon.digest(res.set_offsets, res.set_items, res.supports) == ref["oracle"]


def test_large_sparse_certificate():
    """large_sparse at full size: the oracle's certificate (recount, parents, completeness) on sampled sets."""
    w = synth.make_workload("large_sparse")
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    res = db.mine(w["minsup"], class_order="uniform")
    db.free()
    code, bad = oracle.check(w["offsets"], w["items"], w["N"], w["minsup"], res.set_offsets, res.set_items,
                             res.supports, stride=20011)
    assert code == 0, (oracle.CHECK_CODES[code], bad)


# ---------------------------------------------------------------- warp DFS (rows of at most 512 words)

@pytest.mark.parametrize("name,D,ms_scale", [("tiny", 10000, 1.0), ("sparse_mid", 16000, 1.0), ("dense_deep", 16000, 1.0),
                                             ("large_sparse", 10000, 1.0), ("sparse_mid", 1000, 1.0),
                                             ("dense_deep", 738, 1.0)])
def test_warp_dfs_workload_laws(name, D, ms_scale):
    """Every row-width class of the warp DFS (1, 2, 4, 8, 16 words per lane) on the workloads' laws at
    sample-like sizes, against the oracle."""
    w = synth.make_workload(name, D=D)
    ms = max(2, int(synth.abs_minsup(w["rel_minsup"], D) * ms_scale))
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    res = gpu_mine(w["offsets"], w["items"], w["N"], ms, dfs_mode=4)
    assert_same(res.as_dict(), want)
    st = res.stats
    assert st["n_frequent"] == len(want)


@pytest.mark.parametrize("D", [32, 64, 128, 1000, 2048, 4096, 8192, 16384])
def test_warp_dfs_words_per_lane(D):
    """Row widths 32 ... 512 words (D up to 16,384 bits): deep dense classes through the warp stack."""
    rng = np.random.default_rng(D + 5)
    N = 14
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.3, 0.9))[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = max(1, D // 8)
    want = odict(oracle.eclat(off, items, N, minsup))
    for wb in (32, 64):
        assert_same(gpu_mine(off, items, N, minsup, word_bits=wb, dfs_mode=4).as_dict(), want)


def test_warp_dfs_falls_back_on_wide_rows():
    """FIM_DFS_WARP on rows wider than 512 words runs the sparse node mode: same output."""
    w = synth.make_workload("sparse_mid", D=30000)
    ms = 75
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    assert_same(gpu_mine(w["offsets"], w["items"], w["N"], ms, dfs_mode=4).as_dict(), want)


def test_host_result_arrays_outlive_the_result():
    """A host result's arrays view the result's own pinned memory: they stay valid after Result.free() and
    after the Result object is gone (the memory goes back to the pool only when the last array does), and
    results made meanwhile reuse pooled blocks without touching them."""
    import gc

    w = synth.make_workload("tiny", D=6000)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], 60))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    res = db.mine(60)
    off, items, supp = res.set_offsets, res.set_items, res.supports
    res.free()
    del res
    gc.collect()
    for _ in range(3):  # more results while the arrays above are alive
        other = db.mine(90)
        assert other.n_sets < len(want)
        del other
        gc.collect()
    got = {tuple(int(v) for v in items[off[k]:off[k + 1]]): int(supp[k]) for k in range(len(supp))}
    assert got == want
    db.free()
