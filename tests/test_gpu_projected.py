"""GPU parity of the projected DFS (FIM_DFS_PROJECTED) against the CPU oracle.

The projected traversal builds, for every one-item class [i | S_i], the bitmaps
of the survivors S_i over the transactions of i (Phase 3 of the thesis on the
device) and mines every two-item class from those short bitmaps (Phase 4);
classes past its budgets go to a second queue mined by the sparse node mode.
Counts are integers: the bar is the oracle's exact set of itemsets and supports,
for every split of the classes between the two queues.
"""
import numpy as np
import pytest

import oracle
from paper_2108_05038_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2108_05038_gb300 import fim  # noqa: E402

PROJ = 5


def odict(res):
    so, si, sp = res
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(len(sp))}


def assert_same(got: dict, want: dict):
    if got != want:
        missing = [k for k in want if k not in got][:5]
        extra = [k for k in got if k not in want][:5]
        wrong = [(k, got[k], want[k]) for k in want if k in got and got[k] != want[k]][:5]
        raise AssertionError(f"{len(got)} vs {len(want)} itemsets; missing {missing} extra {extra} wrong {wrong}")


def csr(txs):
    off = np.zeros(len(txs) + 1, dtype=np.uint32)
    items = []
    for i, t in enumerate(txs):
        items.extend(sorted(set(int(v) for v in t)))
        off[i + 1] = len(items)
    return off, np.array(items, dtype=np.uint32)


@pytest.mark.parametrize("seed", range(8))
def test_random_small_vs_bruteforce(seed):
    """Random databases (supports from 1 to all transactions, minsup down to 1) against brute force."""
    rng = np.random.default_rng(4200 + seed)
    N = int(rng.integers(3, 14))
    D = int(rng.integers(1, 900))
    dens = rng.uniform(0.05, 0.8)
    txs = [list(np.nonzero(rng.random(N) < dens)[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = int(rng.integers(1, max(2, D // 4)))
    want = odict(oracle.bruteforce(off, items, N, minsup))
    db = fim.build_vertical_db(off, items, N, word_bits=32 if seed % 2 else 64)
    got = db.mine(minsup, dfs_mode=PROJ).as_dict()
    db.free()
    assert_same(got, want)


# (workload, D, minsup): rows of up to 200,000 transactions; the large-sparse laws have about 3,900 frequent
# rows, so the automatic mode takes the projected traversal itself there
CASES = [("large_sparse", 200_000, 100), ("large_sparse", 70_000, 40), ("sparse_mid", 100_000, 250),
         ("dense_deep", 50_000, 30_000), ("tiny", 10_000, 100)]


@pytest.fixture(scope="module")
def wants():
    out = {}
    for name, D, ms in CASES:
        w = synth.make_workload(name, D=D)
        out[(name, D, ms)] = (w, odict(oracle.eclat_mt(w["offsets"], w["items"], w["N"], ms, 0)))
    return out


@pytest.mark.parametrize("case", CASES)
def test_workloads_exact(case, wants):
    w, want = wants[case]
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=w["word_bits"])
    db.estimate_class_costs(0.01, case[2] / case[1], 1)
    mode = None if case[0] == "large_sparse" else PROJ  # the automatic choice with 1,024 or more frequent rows
    res = db.mine(case[2], dfs_mode=mode)
    db.free()
    assert_same(res.as_dict(), want)


@pytest.mark.parametrize("budget", [("bitmap", 1), ("bitmap", 20_000), ("row", 8), ("row", 40), ("stack", 64),
                                    ("stack", 4096), ("split", 1), ("split", 64), ("split", 2048)])
def test_budget_splits_stay_exact(budget, wants):
    """Small budgets send some classes (or all) to the fallback queue, a small first stack forces the
    doubling retries, and a small split threshold hands almost every frame to other warps with its own
    database part: the output is the oracle's in every case, with the same class nodes and
    intersections as the sparse node mode alone."""
    case = ("large_sparse", 70_000, 40)
    w, want = wants[case]
    kind, v = budget
    kw = {"bitmap": {"proj_bitmap_words": v}, "row": {"proj_max_row_words": v},
          "stack": {"proj_stack_words": v}, "split": {"proj_split_words": v}}[kind]
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    ref = db.mine(case[2], dfs_mode=3, class_order="uniform").stats
    res = db.mine(case[2], dfs_mode=PROJ, class_order="uniform", **kw)
    db.free()
    assert_same(res.as_dict(), want)
    st = res.stats
    for key in ("n_intersections", "n_classes", "n_queue_entries", "n_frequent", "max_len"):
        assert st[key] == ref[key], key


def test_class_work_equals_sparse_mode(wants):
    """Intersections per one-row class are the same in the projected traversal as in the sparse node
    mode (same nodes, same candidates), in estimate order."""
    case = ("large_sparse", 200_000, 100)
    w, want = wants[case]
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    db.estimate_class_costs(0.01, case[2] / case[1], 1)
    a = db.mine(case[2], dfs_mode=3, class_work=True)
    b = db.mine(case[2], dfs_mode=PROJ, class_work=True, collect_times=True)
    db.free()
    assert np.array_equal(a.class_work, b.class_work)
    assert int(b.class_work.sum()) == b.stats["n_intersections"]
    assert b.stats["ms_dfs_kernel"] > 0 and 0 < b.stats["dfs_cta_busy_mean_ms"] <= b.stats["dfs_cta_busy_max_ms"]


def test_result_on_device_and_itemset_limit(wants):
    """The device-resident result equals the host one; a limit below |F| stops the mine with
    FIM_ERR_OUTPUT_OVERFLOW and leaves the database usable."""
    case = ("large_sparse", 70_000, 40)
    w, want = wants[case]
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    with pytest.raises(fim.FimError) as e:
        db.mine(case[2], dfs_mode=PROJ, max_itemsets=len(want) // 3)
    assert e.value.status == fim.FIM_ERR_OUTPUT_OVERFLOW
    res = db.mine(case[2], dfs_mode=PROJ, result_on_device=True)
    assert res.on_device and res.n_sets == len(want) == res.stats["n_frequent"]
    res.free()
    assert_same(db.mine(case[2], dfs_mode=PROJ).as_dict(), want)
    db.free()


@pytest.mark.parametrize("seed", range(6))
def test_diffset_frames_random_vs_bruteforce(seed):
    """Every frame of the projected DFS held as diffsets (dEclat: d(PXY) = d(PY) minus d(PX), supp(PXY) =
    supp(PX) - |d(PXY)|): the same itemsets and supports as brute force, dense and sparse databases alike."""
    rng = np.random.default_rng(5300 + seed)
    N = int(rng.integers(3, 14))
    D = int(rng.integers(1, 900))
    dens = rng.uniform(0.05, 0.95)
    txs = [list(np.nonzero(rng.random(N) < dens)[0]) for _ in range(D)]
    off, items = csr(txs)
    minsup = int(rng.integers(1, max(2, D // 3)))
    want = odict(oracle.bruteforce(off, items, N, minsup))
    db = fim.build_vertical_db(off, items, N, word_bits=64)
    for mode in (1, 2):
        assert_same(db.mine(minsup, dfs_mode=PROJ, diffsets=mode).as_dict(), want)
    db.free()


@pytest.mark.parametrize("name,D,minsup", [("dense_deep", 50_000, 30_000), ("dense_deep", 200_000, 120_000),
                                           ("large_sparse", 70_000, 40), ("sparse_mid", 100_000, 250)])
def test_diffset_frames_workloads(name, D, minsup):
    """The deep dense workload, its law at 200,000 transactions (rows of 6,250 words), and two sparse ones:
    tidset and diffset frames give the oracle's output, with the same class nodes and intersections; the
    operand bytes per node of both forms are reported by the stats."""
    w = synth.make_workload(name, D=D)
    want = odict(oracle.eclat_mt(w["offsets"], w["items"], w["N"], minsup, 0))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    ref = db.mine(minsup, dfs_mode=PROJ, diffsets=0)
    assert_same(ref.as_dict(), want)
    for mode in (1, 2):
        res = db.mine(minsup, dfs_mode=PROJ, diffsets=mode)
        assert_same(res.as_dict(), want)
        for key in ("n_intersections", "n_classes", "n_frequent"):
            assert res.stats[key] == ref.stats[key], key
    db.free()
