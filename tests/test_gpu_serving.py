"""Serving: jobs on different databases and minsups admitted into a
continuous-batching loop give, in the mix, exactly the result each gives alone
(and the oracle's)."""
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


def small_requests(n):
    # the serving laws with bounded transaction lengths and minsup >= 1%: small outputs the oracle mines quickly
    reqs = synth.serving_requests(n, seed=77, D_range=(2_000, 40_000), N_range=(50, 600), TL_range=(4.0, 12.0),
                                  rel_range=(0.01, 0.05))
    out = []
    for r in reqs:
        off, items = synth.request_db(r)
        ms = max(2, r["minsup"])
        out.append((off, items, r["N"], ms))
    return out


def test_mix_equals_alone_and_oracle():
    reqs = small_requests(12)
    alone = []
    for off, items, N, ms in reqs:
        db = fim.build_vertical_db(off, items, N, prefilter_minsup=ms)
        alone.append(db.mine(ms).as_dict())
        db.free()
    srv = fim.Server(slots=4, ctas_per_sm=1)
    ids = [srv.submit(off, items, N, ms, sample_rate=0.05) for off, items, N, ms in reqs]
    for k, jid in enumerate(ids):
        res, lat, svc = srv.wait(jid)
        assert lat >= svc >= 0
        got = res.as_dict()
        assert got == alone[k]
        off, items, N, ms = reqs[k]
        assert got == odict(oracle.eclat(off, items, N, ms))
    st = srv.stats()
    assert st["in_flight"] == 0 and st["queued"] == 0 and st["peak_in_flight"] >= 1
    srv.free()


def test_budget_forces_one_at_a_time_and_stays_exact():
    reqs = small_requests(5)
    srv = fim.Server(hbm_budget_bytes=1, slots=4)  # every job exceeds the budget: they run alone
    ids = [srv.submit(off, items, N, ms) for off, items, N, ms in reqs]
    for k, jid in enumerate(ids):
        res, _, _ = srv.wait(jid)
        off, items, N, ms = reqs[k]
        assert res.as_dict() == odict(oracle.eclat(off, items, N, ms))
    assert srv.stats()["peak_in_flight"] == 1
    srv.free()


def test_bad_job_reports_error_others_unaffected():
    reqs = small_requests(3)
    srv = fim.Server(slots=2)
    off, items, N, ms = reqs[0]
    bad_items = items.copy()
    bad_items[0] = N + 5  # item id out of range: the job fails with FIM_ERR_INVALID
    bad = srv.submit(off, bad_items, N, ms)
    good = srv.submit(*reqs[1])
    with pytest.raises(fim.FimError) as e:
        srv.wait(bad)
    assert e.value.status == fim.FIM_ERR_INVALID
    res, _, _ = srv.wait(good)
    off, items, N, ms = reqs[1]
    assert res.as_dict() == odict(oracle.eclat(off, items, N, ms))
    srv.free()


def test_itemset_limit_stops_exploding_job():
    """A request whose output explodes (long transactions, tiny minsup) is stopped at the per-job limit
    with FIM_ERR_OUTPUT_OVERFLOW; the next job is unaffected."""
    txs_len = 24
    D = 400
    rng = np.random.default_rng(9)
    base = rng.choice(60, size=txs_len, replace=False)
    off = np.arange(0, (D + 1) * txs_len, txs_len, dtype=np.uint32)
    items = np.tile(np.sort(base), D).astype(np.uint32)  # every transaction identical: 2^24 - 1 itemsets
    srv = fim.Server(slots=2, max_itemsets=100_000)
    bad = srv.submit(off, items, 60, 2)
    good_req = small_requests(1)[0]
    good = srv.submit(*good_req)
    with pytest.raises(fim.FimError) as e:
        srv.wait(bad)
    assert e.value.status == fim.FIM_ERR_OUTPUT_OVERFLOW
    res, _, _ = srv.wait(good)
    off2, items2, N2, ms2 = good_req
    assert res.as_dict() == odict(oracle.eclat(off2, items2, N2, ms2))
    srv.free()


def test_long_jobs_overlap_on_the_device_and_stay_exact():
    """Continuous batching, not a queue alone: two long jobs submitted together run on the device at the
    same time (their device intervals, from CUDA events on their slots' streams, intersect), and each
    result equals the job's result alone and the oracle's."""
    jobs = []
    for seed, D in ((11, 60_000), (12, 60_000)):
        w = synth.make_workload("sparse_mid", D=D, seed=seed)
        ms = synth.abs_minsup(w["rel_minsup"], D)
        jobs.append((w["offsets"], w["items"], w["N"], ms))
    alone = []
    for off, items, N, ms in jobs:
        db = fim.build_vertical_db(off, items, N, prefilter_minsup=ms)
        alone.append(db.mine(ms).as_dict())
        db.free()
    srv = fim.Server(slots=2, ctas_per_sm=1)
    ids = [srv.submit(off, items, N, ms, sample_rate=0.01) for off, items, N, ms in jobs]
    spans = []
    for k, jid in enumerate(ids):
        res, lat, svc, (t0, t1) = srv.wait_ex(jid)
        assert 0 <= t0 < t1
        spans.append((t0, t1))
        got = res.as_dict()
        assert got == alone[k]
        off, items, N, ms = jobs[k]
        assert got == odict(oracle.eclat(off, items, N, ms))
    assert srv.stats()["peak_in_flight"] == 2
    srv.free()
    (a0, a1), (b0, b1) = spans
    assert max(a0, b0) < min(a1, b1), spans  # the two device intervals intersect
