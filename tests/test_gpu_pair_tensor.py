"""Level-2 pair counts on the tensor cores (FIM_PAIR_TENSOR: packed e2m1 operands; FIM_PAIR_TENSOR_E4M3:
byte operands; FIM_PAIR_TENSOR_FUSED: the raw bits widened to e4m3 in shared memory inside the kernel)
against the oracle: named workloads at
full size, ragged numbers of frequent rows around the 128 x 256 tile edges, supports past 2^24 (fp32
exactness needs the K range split), graph replays, and the integer-pipe kernel on the same inputs."""
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


def csr(txs):
    off = np.cumsum([0] + [len(t) for t in txs]).astype(np.uint32)
    items = np.array([int(i) for t in txs for i in t], dtype=np.uint32)
    return off, items


TENSOR = [fim.FIM_PAIR_TENSOR, fim.FIM_PAIR_TENSOR_E4M3, fim.FIM_PAIR_TENSOR_FUSED]


@pytest.mark.parametrize("pk", TENSOR)
@pytest.mark.parametrize("name", ["tiny", "dense_deep", "dense_exact37", "sparse_mid"])
def test_workloads_exact_on_tensor_cores(name, pk):
    w = synth.make_workload(name)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], w["minsup"]))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], word_bits=w["word_bits"])
    try:
        res = db.mine(w["minsup"], pair_kernel=pk)
        assert res.stats["pair_kernel"] == pk
        assert res.as_dict() == want
        cores = db.mine(w["minsup"], pair_kernel=fim.FIM_PAIR_CORES)
        assert cores.stats["pair_kernel"] == fim.FIM_PAIR_CORES
        assert cores.as_dict() == want
    finally:
        db.free()


@pytest.mark.parametrize("pk", TENSOR)
@pytest.mark.parametrize("n1", [2, 3, 127, 128, 129, 255, 256, 257, 383, 385, 600])
@pytest.mark.parametrize("D", [700, 4097])
def test_ragged_frequent_rows(n1, D, pk):
    """Every item frequent (minsup 1), transactions of at most 4 items: all pairs that occur, and
    the deeper itemsets, equal the oracle; tile edges at 128 (i) and 256 (j) rows."""
    rng = np.random.default_rng(n1 * 7 + D)
    txs = [list(rng.choice(n1, size=rng.integers(1, min(5, n1 + 1)), replace=False)) for _ in range(D)]
    txs += [[k, (k + 1) % n1] for k in range(n1)]  # every item occurs
    off, items = csr(txs)
    want = odict(oracle.eclat(off, items, n1, 1))
    db = fim.build_vertical_db(off, items, n1)
    try:
        assert db.mine(1, pair_kernel=pk).as_dict() == want
    finally:
        db.free()


@pytest.mark.parametrize("pk", TENSOR)
def test_supports_past_fp32_integer_range(pk):
    """D = 2^24 + 1 identical transactions of 12 items: every one of the 4,095 itemsets has support
    2^24 + 1, which fp32 cannot hold, so the K range must be split into exact partial sums."""
    D, N = (1 << 24) + 1, 12
    d_off = (torch.arange(D + 1, dtype=torch.int64, device="cuda") * N).to(torch.int32)
    d_items = torch.arange(N, dtype=torch.int32, device="cuda").repeat(D)
    torch.cuda.synchronize()
    db = fim.build_vertical_db_device(d_off, d_items, D, N, 64, 0)
    try:
        res = db.mine(D, pair_kernel=pk)
        got = res.as_dict()
        assert len(got) == (1 << N) - 1
        assert set(got.values()) == {D}
    finally:
        db.free()
        del d_off, d_items


@pytest.mark.parametrize("pk", [fim.FIM_PAIR_TENSOR, fim.FIM_PAIR_TENSOR_FUSED])
def test_graph_replay_on_tensor_cores(pk):
    w = synth.make_workload("sparse_mid", D=30000)
    ms = 80
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        plan = db.plan(ms, pair_kernel=pk)
        for _ in range(3):
            plan.launch()
            assert plan.result().as_dict() == want
        plan.free()
    finally:
        db.free()


def test_estimate_and_mine_with_automatic_choice():
    """The automatic choice (tensor cores on sparse_mid's 988 rows of 12.5 KB; fused, since a mine's
    frequent rows are consecutive) keeps the output exact through the sample estimate and the mine."""
    w = synth.make_workload("sparse_mid")
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], w["minsup"]))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        db.estimate_class_costs(0.01, w["rel_minsup"], 1)
        res = db.mine(w["minsup"])
        assert res.stats["pair_kernel"] in (fim.FIM_PAIR_CORES, fim.FIM_PAIR_TENSOR_FUSED)
        assert res.as_dict() == want
    finally:
        db.free()


@pytest.mark.parametrize("pk", [fim.FIM_PAIR_TENSOR, fim.FIM_PAIR_TENSOR_FUSED])
def test_pair_kernel_wait_runs_out_and_context_survives(pk):
    """Failure detection on the GPU: with fault_pair_wait every stage of the tensor pair kernel waits for
    16 bytes that never arrive, so its bounded mbarrier waits (about 1 s each) run out; the kernel
    flags the timeout, lets its copies and MMAs finish, frees its TMEM and returns, nothing below
    level 2 runs on the incomplete counts, and the call reports FIM_ERR_TIMEOUT.  The same database
    then mines exactly."""
    w = synth.make_workload("sparse_mid", D=20000)
    ms = 50
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        with pytest.raises(fim.FimError) as e:
            db.mine(ms, pair_kernel=pk, fault_pair_wait=True)
        assert e.value.status == fim.FIM_ERR_TIMEOUT
        assert db.mine(ms, pair_kernel=pk).as_dict() == want
        torch.cuda.synchronize()  # the context is intact
    finally:
        db.free()


def test_fused_kernel_needs_no_widened_rows():
    """The fused kernel takes no scratch for widened rows: the database's device bytes (its bitmaps and
    workspace) grow by nothing on a fused mine after an integer-pipe mine of the same minsup, while the
    widened kernel's scratch (rows x padded words x 16 bytes) adds to them."""
    w = synth.make_workload("sparse_mid")
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    try:
        db.mine(w["minsup"], pair_kernel=fim.FIM_PAIR_CORES)
        base = db.info()["device_bytes"]
        res = db.mine(w["minsup"], pair_kernel=fim.FIM_PAIR_TENSOR_FUSED)
        assert res.stats["pair_kernel"] == fim.FIM_PAIR_TENSOR_FUSED
        assert db.info()["device_bytes"] == base
        db.mine(w["minsup"], pair_kernel=fim.FIM_PAIR_TENSOR)
        assert db.info()["device_bytes"] > base
    finally:
        db.free()
