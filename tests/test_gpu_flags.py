"""fim_result_flags (closed and maximal itemsets, Ch. 2) against the oracle's definitions on the same
seeded inputs: bit-exact flags for every itemset, host and device results."""
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
    off = np.cumsum([0] + [len(t) for t in txs]).astype(np.uint32)
    items = np.array([int(i) for t in txs for i in t], dtype=np.uint32)
    return off, items


def gpu_flags(off, items, N, minsup, **kw):
    db = fim.build_vertical_db(off, items, N)
    try:
        res = db.mine(minsup, **kw)
        fl = res.flags()
        so, si = res.set_offsets, res.set_items
        out = {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(fl[k]) for k in range(res.n_sets)}
        res.free()
        return out
    finally:
        db.free()


def oracle_flags(off, items, N, minsup):
    so, si, sp, fl = oracle.closed_maximal(off, items, N, minsup)
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(fl[k]) for k in range(len(sp))}


@pytest.mark.parametrize("seed", range(8))
def test_random_small_databases(seed):
    rng = np.random.default_rng(900 + seed)
    N = int(rng.integers(3, 16))
    txs = [list(np.nonzero(rng.random(N) < rng.uniform(0.1, 0.8))[0]) for _ in range(int(rng.integers(10, 400)))]
    off, items = csr(txs)
    for minsup in (1, max(1, len(txs) // 10)):
        assert gpu_flags(off, items, N, minsup) == oracle_flags(off, items, N, minsup)


@pytest.mark.parametrize("name,D", [("tiny", 10000), ("dense_deep", 4000), ("sparse_mid", 20000)])
def test_workload_laws(name, D):
    w = synth.make_workload(name, D=D)
    ms = synth.abs_minsup(w["rel_minsup"], D)
    assert gpu_flags(w["offsets"], w["items"], w["N"], ms) == oracle_flags(w["offsets"], w["items"], w["N"], ms)


def test_closed_forms_and_device_result():
    """Identical transactions: only the full set is closed and maximal (2^12 - 1 itemsets); the same
    counts from a device-resident result."""
    off, items = csr([list(range(12))] * 40)
    f = gpu_flags(off, items, 12, 40)
    assert len(f) == 4095 and f[tuple(range(12))] == 3 and sum(1 for v in f.values() if v) == 1
    db = fim.build_vertical_db(off, items, 12)
    try:
        res = db.mine(40, result_on_device=True)
        fl = res.flags()
        assert len(fl) == 4095 and int((fl == 3).sum()) == 1 and int((fl != 0).sum()) == 1
        res.free()
    finally:
        db.free()
