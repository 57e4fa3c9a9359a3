"""The estimate left on the device (fim_estimate_class_costs_ex with NULL outputs): the sample's mine, its
per-class counts and the LPT order of the classes (Sec. 8.2) stay on the device until a mine or a query
reads them.  Checked against the oracle: the mine's output, and the costs, order and sample size that
fim_estimate_result / fim_estimate_sample_size report afterwards, including a sample past its itemset
limit (redone by the synchronous path after the mine), a replaced estimate, a uniform-order mine and a
plan created while the estimate is pending."""
import math

import numpy as np
import pytest

import oracle
from paper_2108_05038_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2108_05038_gb300 import fim  # noqa: E402


def odict(res):
    so, si, sp = res
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(len(sp))}


def deferred(w, rate, rel):
    """Whether the documented condition for a device-resident estimate holds (without a prefilter every
    item is a row): at most 4,096 rows and at least 3/4 of them with supp * m / D >= minsup_s."""
    D = w["offsets"].size - 1
    supp = np.bincount(w["items"].astype(np.int64), minlength=w["N"])
    m = max(math.ceil(rate * D), min(D, 738))
    ms = max(1, math.ceil(rel * m))
    pred = int(np.sum(supp * m / D >= ms))
    return supp.size <= 4096 and 4 * pred >= 3 * supp.size


CASES = [("tiny", 10000, 0.05, 0.01, 3, 0), ("sparse_mid", 100000, 0.01, 0.0025, 1, 0),
         ("sparse_mid", 50000, 0.02, 0.005, 1, 1), ("dense_deep", 8000, 0.05, 0.3, 4, 1)]


@pytest.mark.parametrize("name,D,rate,rel,seed,kind", CASES)
def test_deferred_estimate_matches_oracle(name, D, rate, rel, seed, kind):
    w = synth.make_workload(name, D=D)
    assert deferred(w, rate, rel)
    minsup = max(1, math.ceil(rel * D))
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], minsup))
    ocost, oorder, onfs = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, rate, rel, seed, kind=kind)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        costk = ("itemsets", "intersections")[kind]
        assert db.estimate_class_costs(rate, rel, seed, cost=costk, outputs=False) is None
        assert db.mine(minsup).as_dict() == want
        cost, order = db.estimate_result()
        assert np.array_equal(cost, ocost)
        assert np.array_equal(order, oorder)
        nfs, m, _ = db.estimate_sample_size()
        assert nfs == onfs and m == max(math.ceil(rate * D), min(D, 738))
        assert db.mine(minsup).as_dict() == want  # the second mine takes the host copies
    finally:
        db.free()


@pytest.mark.parametrize("rel,limit,kind", [(0.45, 300, "itemsets"), (0.3, 20000, "intersections")])
def test_deferred_sample_past_its_limit_is_redone(rel, limit, kind):
    """dense_deep, 8,000 rows: the sample at the start minsup has more itemsets than the limit, so the
    synchronous path doubles its minsup (as the oracle does) after the first mine, which stays exact."""
    w = synth.make_workload("dense_deep", D=8000)
    assert deferred(w, 0.05, rel)
    minsup = math.ceil(rel * 8000)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], minsup))
    k = {"itemsets": 0, "intersections": 1}[kind]
    ocost, oorder, onfs, oms = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, 0.05, rel, 11, kind=k,
                                                  limit=limit, return_minsup=True)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        db.estimate_class_costs(0.05, rel, 11, cost=kind, max_sample_itemsets=limit, outputs=False)
        assert db.mine(minsup).as_dict() == want
        nfs, _, ms = db.estimate_sample_size()
        assert (nfs, ms) == (onfs, oms)
        cost, order = db.estimate_result()
        assert np.array_equal(cost, ocost)
        assert np.array_equal(order, oorder)
    finally:
        db.free()


def test_replaced_estimate_uniform_mine_and_plan():
    w = synth.make_workload("sparse_mid", D=60000)
    rel = 0.004
    minsup = math.ceil(rel * 60000)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], minsup))
    ocost, oorder, _ = oracle.class_costs(w["offsets"], w["items"], w["N"], 0, 0.02, rel, 7)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        assert deferred(w, 0.01, rel) and deferred(w, 0.02, rel)
        db.estimate_class_costs(0.01, rel, 5, outputs=False)
        db.estimate_class_costs(0.02, rel, 7, outputs=False)  # replaces the first while it may be pending
        assert db.mine(minsup, class_order="uniform").as_dict() == want
        cost, order = db.estimate_result()
        assert np.array_equal(cost, ocost) and np.array_equal(order, oorder)
        db.estimate_class_costs(0.02, rel, 7, outputs=False)
        plan = db.plan(minsup)  # reads the pending estimate on the host
        plan.launch()
        assert plan.result().as_dict() == want
        plan.free()
        db.estimate_class_costs(0.02, rel, 7, outputs=False)
        res = db.mine(minsup, result_on_device=True)
        assert res.n_sets == len(want)
        res.free()
    finally:
        db.free()


# Samples with more than 1,024 frequent rows: the automatic DFS mines them with the projected DFS (and the
# sparse node mode for the classes left out), whose count-only mines check the itemset limit at their polls.
# (12,000 x 1,400: 1,079 of the 1,400 rows predicted frequent in the 6,000-transaction sample, so the sample is
# mined over all rows; start minsup 9 gives 26,822 itemsets, past a limit of 20,000: 18 gives 10,538.
# 20,000 x 1,500 at rate 1/4: 73% predicted, so the sample is mined over its frequent rows; 11,480 itemsets at
# minsup 10, past 5,000: 3,476 at 20.)
PROJ_CASES = [(12000, 1400, 12.0, 0.5, 0.0015, 0, 0, False), (12000, 1400, 12.0, 0.5, 0.0015, 20000, 0, False),
              (12000, 1400, 12.0, 0.5, 0.0015, 20000, 1, True), (20000, 1500, 10.0, 0.25, 0.002, 5000, 0, True)]


@pytest.mark.parametrize("D,N,TL,rate,rel,limit,kind,outputs", PROJ_CASES)
def test_sample_mined_by_the_projected_dfs_matches_oracle(D, N, TL, rate, rel, limit, kind, outputs):
    off, items = synth.pattern_db(7, D, N, TL, 5.0, 500 if D == 12000 else 600)
    w = {"offsets": off, "items": items, "N": N}
    assert deferred(w, rate, rel) == (D == 12000)
    ocost, oorder, onfs, oms = oracle.class_costs(off, items, N, 0, rate, rel, 5, kind=kind, limit=limit,
                                                  return_minsup=True)
    assert onfs > 1024 and (limit == 0 or oms > max(1, math.ceil(rel * math.ceil(rate * D))))
    minsup = math.ceil(rel * D)
    want = odict(oracle.eclat(off, items, N, minsup))
    db = fim.build_vertical_db(off, items, N)
    try:
        costk = ("itemsets", "intersections")[kind]
        if outputs:
            cost, order = db.estimate_class_costs(rate, rel, 5, cost=costk, max_sample_itemsets=limit)
        else:
            assert db.estimate_class_costs(rate, rel, 5, cost=costk, max_sample_itemsets=limit, outputs=False) is None
            assert db.mine(minsup).as_dict() == want
            cost, order = db.estimate_result()
        nfs, m, ms = db.estimate_sample_size()
        assert (nfs, ms, m) == (onfs, oms, math.ceil(rate * D))
        assert np.array_equal(cost, ocost)
        assert np.array_equal(order, oorder)
        assert db.mine(minsup).as_dict() == want
    finally:
        db.free()
