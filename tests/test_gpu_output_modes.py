"""GPU output modes: only the maximal itemsets (the DFS writes its leaves, the candidates on an MFI of the
DFS-MFI-Schema, Ch. 7, and a superset pass keeps the maximal ones) or only the closed ones, against the
oracle's definitions (oracle.closed_maximal: closure by the item counts over each itemset's transactions).
Counts are integers: the bar is the exact set of itemsets and supports."""
import numpy as np
import pytest

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


def want_sets(off, items, N, minsup):
    so, si, sp, fl = oracle.closed_maximal(off, items, N, minsup)
    sets = {tuple(int(v) for v in si[so[k]:so[k + 1]]): (int(sp[k]), int(fl[k])) for k in range(len(sp))}
    closed = {s: c for s, (c, f) in sets.items() if f & 1}
    maximal = {s: c for s, (c, f) in sets.items() if f & 2}
    return closed, maximal


def assert_same(got, want):
    if got != want:
        missing = [k for k in want if k not in got][:5]
        extra = [k for k in got if k not in want][:5]
        raise AssertionError(f"{len(got)} vs {len(want)}; missing {missing} extra {extra}")


@pytest.mark.parametrize("seed", range(10))
def test_random_databases(seed):
    rng = np.random.default_rng(9100 + seed)
    N = int(rng.integers(3, 14))
    D = int(rng.integers(1, 600))
    dens = rng.uniform(0.05, 0.85)
    txs = [list(np.nonzero(rng.random(N) < dens)[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = int(rng.integers(1, max(2, D // 3)))
    closed, maximal = want_sets(off, items, N, minsup)
    db = fim.build_vertical_db(off, items, N, word_bits=32 if seed % 2 else 64)
    assert_same(db.mine(minsup, output="maximal").as_dict(), maximal)
    assert_same(db.mine(minsup, output="closed").as_dict(), closed)
    db.free()


@pytest.mark.parametrize("name,D,minsup", [("tiny", 10_000, 100), ("dense_deep", 5_000, 3_000),
                                           ("sparse_mid", 20_000, 50)])
def test_workloads(name, D, minsup):
    w = synth.make_workload(name, D=D)
    closed, maximal = want_sets(w["offsets"], w["items"], w["N"], minsup)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=w["word_bits"])
    db.estimate_class_costs(0.05, minsup / D, 2)
    res = db.mine(minsup, output="maximal")
    assert_same(res.as_dict(), maximal)
    assert res.stats["n_frequent"] == len(maximal)
    assert_same(db.mine(minsup, output="closed").as_dict(), closed)
    db.free()


@pytest.mark.parametrize("kw", [{}, {"proj_bitmap_words": 1}, {"proj_split_words": 1}, {"proj_stack_words": 256}])
def test_maximal_under_every_split(kw):
    """The leaves are written by the projected DFS, by its sparse fallback (every class past a one-word
    budget), by warps that take handed-out frames (every frame handed out) and across stack regrowth."""
    w = synth.make_workload("sparse_mid", D=20_000)
    closed, maximal = want_sets(w["offsets"], w["items"], w["N"], 40)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    assert_same(db.mine(40, output="maximal", **kw).as_dict(), maximal)
    db.free()


def test_closed_forms():
    """k identical transactions of m items: one maximal and one closed itemset, the whole set; disjoint
    single-item transactions: every frequent singleton is maximal and closed."""
    off, items = csr([list(range(9))] * 30)
    db = fim.build_vertical_db(off, items, 9)
    assert db.mine(5, output="maximal").as_dict() == {tuple(range(9)): 30}
    assert db.mine(5, output="closed").as_dict() == {tuple(range(9)): 30}
    db.free()
    off, items = csr([[i % 7] for i in range(70)])
    db = fim.build_vertical_db(off, items, 7)
    assert db.mine(10, output="maximal").as_dict() == {(i,): 10 for i in range(7)}
    db.free()


def test_maximal_of_a_wide_database_equals_the_full_result_flags():
    """On 70,000 transactions of the large-sparse laws (about 3,900 frequent rows: the automatic projected DFS)
    the maximal output equals the maximal itemsets that the flags pass finds in the complete result,
    itself pinned to the oracle's definitions on the smaller cases (tests/test_gpu_flags.py)."""
    w = synth.make_workload("large_sparse", D=70_000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    full = db.mine(40)
    fl = full.flags()
    d = full.as_dict()
    keys = list(d.keys())
    want = {keys[k]: d[keys[k]] for k in range(len(keys)) if fl[k] & 2}
    got = db.mine(40, output="maximal")
    assert_same(got.as_dict(), want)
    assert got.n_sets < full.n_sets
    db.free()
