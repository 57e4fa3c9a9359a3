"""fim_extension_supports against the oracle's definition of support (Ch. 2) on the same seeded
inputs: bit-exact counts, one-item and multi-item prefixes, ragged D, dense and sparse prefixes."""
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


def check(off, items, N, prefixes, word_bits=64, prefilter=0, cands=None):
    db = fim.build_vertical_db(off, items, N, word_bits=word_bits, prefilter_minsup=prefilter)
    try:
        kept = db.rows()[0]
        cands = kept if cands is None else np.asarray(cands, dtype=np.uint32)
        for p in prefixes:
            got = db.extension_supports(p, cands)
            want = oracle.extension_supports(off, items, N, p, cands)
            assert np.array_equal(got.astype(np.uint64), want), (p, np.flatnonzero(got != want)[:5])
    finally:
        db.free()


@pytest.mark.parametrize("D", [1, 63, 64, 1000, 4097, 40_001])
@pytest.mark.parametrize("word_bits", [32, 64])
def test_random_prefixes_vs_oracle(D, word_bits):
    rng = np.random.default_rng(D + word_bits)
    N = 40
    txs = [list(rng.choice(N, size=rng.integers(0, 9), replace=False)) for _ in range(D)]
    txs[0] = [0, 1, 2]
    off, items = csr(txs)
    db = fim.build_vertical_db(off, items, N, word_bits=word_bits)
    kept = db.rows()[0]
    db.free()
    prefixes = [[int(kept[k % len(kept)])] for k in range(3)]
    prefixes += [list(rng.choice(kept, size=s, replace=True)) for s in (2, 3, 5)]
    check(off, items, N, prefixes, word_bits)


def test_many_word_tiles_dense_prefix_closed_form():
    """Item 0 in every transaction of a 300,001-transaction database (each row spans several
    loop trips of a CTA and ends in a ragged word): supp({0, c}) = supp(c) for every kept c."""
    D, N = 300_001, 300
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 6, size=D)
    off = np.zeros(D + 1, dtype=np.uint32)
    off[1:] = np.cumsum(lens + 1)
    items = np.empty(int(off[-1]), dtype=np.uint32)
    items[off[:-1]] = 0
    rest = np.ones(int(off[-1]), dtype=bool)
    rest[off[:-1]] = False
    items[rest] = rng.integers(1, N, size=int(rest.sum()))  # repeats inside a transaction count once
    db = fim.build_vertical_db(off, items, N)
    try:
        kept, supp = db.rows()
        got = db.extension_supports([0], kept)
        assert np.array_equal(got, supp)
        assert np.array_equal(got.astype(np.uint64), oracle.extension_supports(off, items, N, [0], kept))
        want = oracle.extension_supports(off, items, N, [0, 7, 9], kept)
        assert np.array_equal(db.extension_supports([9, 0, 7], kept).astype(np.uint64), want)
    finally:
        db.free()


def test_sparse_prefix_skips_zero_words():
    """A prefix item present only in a block of transactions (most 16-byte words of t(P) are zero)
    and at scattered positions: counts stay exact."""
    w = synth.make_workload("sparse_mid", D=120_000)
    off, items, N = w["offsets"], w["items"], w["N"]
    D = off.size - 1
    txs = [list(items[off[i]:off[i + 1]]) for i in range(D)]
    for i in list(range(5000, 5400)) + list(range(0, D, 997)):
        txs[i] = txs[i] + [N]  # item N: the block plus a stride of transactions
    off2, items2 = csr(txs)
    check(off2, items2, N + 1, [[N], [N, int(items[0])]])


def test_workload_prefilter_and_candidate_inside_prefix():
    w = synth.make_workload("tiny", D=6000)
    off, items, N = w["offsets"], w["items"], w["N"]
    db = fim.build_vertical_db(off, items, N, prefilter_minsup=60)
    kept = db.rows()[0]
    db.free()
    p = [int(kept[-1]), int(kept[-2])]
    check(off, items, N, [p, p[:1]], prefilter=60, cands=list(kept) + p)


def test_errors_and_empty_candidates():
    off, items = csr([[1, 2], [2, 3], [1]])
    db = fim.build_vertical_db(off, items, 5, prefilter_minsup=2)  # items 1 and 2 kept, 3 dropped
    try:
        assert db.extension_supports([1], []).size == 0
        assert list(db.extension_supports([1], [2, 1])) == [1, 2]
        for p, c in (([], [1]), ([7], [1]), ([1], [5]), ([3], [1]), ([1], [3]), ([0], [1])):
            with pytest.raises(fim.FimError) as e:
                db.extension_supports(p, c)
            assert e.value.status == fim.FIM_ERR_INVALID
        assert list(db.extension_supports([2, 1], [1, 2])) == [1, 1]  # still usable after errors
    finally:
        db.free()
