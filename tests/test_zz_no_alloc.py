"""The allocation-free entry point fim_mine_pairs_noalloc, called through the C ABI.

Some callers cannot allocate device memory while they run (memory reserved up
front by another allocator, or a serving loop that must not call cudaMalloc,
which can synchronise the device).  This file runs last so that a failure here
stops a -x run only after every other test has run.  It checks the entry
point's pairs against the 2-itemsets of fim_mine on the same database and
against the oracle's, on two calls in a row (the shared scratch keeps the
previous call's contents), and that the second call allocates nothing: the
device's free memory, the library pool's use and reservation, PyTorch's
allocations and the database's workspace stay as they were.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2108_05038_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2108_05038_gb300 import fim  # noqa: E402


def pairs_of(result_dict):
    return {k: v for k, v in result_dict.items() if len(k) == 2}


def call_noalloc(lib, db, minsup, d_pairs, d_supp, cap):
    n = ctypes.c_uint64()
    status = lib.fim_mine_pairs_noalloc(ctypes.c_void_p(db.handle), minsup, ctypes.c_void_p(d_pairs.data_ptr()),
                                        ctypes.c_void_p(d_supp.data_ptr()), cap, ctypes.byref(n))
    return status, n.value


@pytest.mark.parametrize("name,D,minsup", [("sparse_mid", 100_000, 250), ("tiny", 10_000, 60)])
def test_noalloc_pairs_match_mine_twice(name, D, minsup):
    w = synth.make_workload(name, D=D)
    lib = fim.load()
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=64)
    want = pairs_of(db.mine(minsup).as_dict())
    so, si, sp = oracle.eclat(w["offsets"], w["items"], w["N"], minsup)
    want_oracle = {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(len(sp))
                   if so[k + 1] - so[k] == 2}
    assert want == want_oracle and len(want) > 10
    cap = len(want) + 16
    d_pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    d_supp = torch.zeros(cap, dtype=torch.int32, device="cuda")
    dev = torch.cuda.current_device()
    for call in range(2):
        d_pairs.fill_(-1)
        d_supp.fill_(-1)
        torch.cuda.synchronize()
        before = (torch.cuda.mem_get_info(dev)[0], fim.pool_memory(dev), torch.cuda.memory_allocated(dev),
                  db.info()["device_bytes"])
        status, n = call_noalloc(lib, db, minsup, d_pairs, d_supp, cap)
        torch.cuda.synchronize()
        after = (torch.cuda.mem_get_info(dev)[0], fim.pool_memory(dev), torch.cuda.memory_allocated(dev),
                 db.info()["device_bytes"])
        assert status == fim.FIM_OK, lib.fim_last_error()
        assert n == len(want)
        if call == 1:  # the first call may set up the scratch address; the second allocates nothing
            assert after == before
        p = d_pairs[: 2 * n].cpu().numpy().astype(np.int64).reshape(-1, 2)
        s = d_supp[:n].cpu().numpy().astype(np.int64)
        got = {(int(a), int(b)): int(c) for (a, b), c in zip(p, s)}
        assert got == want
    db.free()


def test_noalloc_rejects_too_many_items_and_small_capacity():
    w = synth.make_workload("large_sparse", D=20_000)
    lib = fim.load()
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    d_pairs = torch.zeros(2, dtype=torch.int32, device="cuda")
    d_supp = torch.zeros(1, dtype=torch.int32, device="cuda")
    status, _ = call_noalloc(lib, db, 2, d_pairs, d_supp, 1)  # thousands of frequent items at minsup 2
    assert status == fim.FIM_ERR_INVALID
    assert b"1024" in lib.fim_last_error()
    db.free()
    w = synth.make_workload("tiny", D=5_000)
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    status, n = call_noalloc(lib, db, 30, d_pairs, d_supp, 1)
    assert status == fim.FIM_ERR_OUTPUT_OVERFLOW and n > 1
    db.free()
