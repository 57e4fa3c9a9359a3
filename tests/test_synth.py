"""The seeded input generator follows the stated recipe (CPU): the laws of the thesis's workload
shapes that the synthetic databases stand in for (pattern-embedded databases with Poisson lengths
and uniform or Zipf(1.1) item popularity, the Bernoulli and exactly-k dense laws, and the serving
request law), checked as statistical properties of the generated data."""
import math

import numpy as np
import pytest

from paper_2108_05038_gb300 import synth


def lengths(w):
    return np.diff(w["offsets"].astype(np.int64))


def assert_set_semantics(w):
    """Items of a transaction are distinct, ascending and below N."""
    off, it = w["offsets"].astype(np.int64), w["items"].astype(np.int64)
    assert off[0] == 0 and off[-1] == len(it) and np.all(np.diff(off) >= 0)
    assert it.size == 0 or (it.min() >= 0 and it.max() < w["N"])
    inner = np.ones(len(it), dtype=bool)
    inner[off[:-1][off[:-1] < len(it)]] = False  # the first item of every non-empty transaction
    assert np.all(np.diff(it)[inner[1:]] > 0)


@pytest.mark.parametrize("name,D", [("tiny", None), ("sparse_mid", None), ("large_sparse", 100_000)])
def test_pattern_databases_have_poisson_lengths(name, D):
    """Transaction lengths come from Poisson(TL), cut only by the fill limit: mean within 2% of TL."""
    w = synth.make_workload(name, D=D)
    assert len(w["offsets"]) - 1 == w["D"]
    assert_set_semantics(w)
    L = lengths(w)
    assert abs(L.mean() - w["TL"]) < 0.02 * w["TL"]
    assert L.var() < 1.5 * w["TL"]  # Poisson: variance = mean (the fill cut only lowers it)


def test_uniform_and_zipf_item_popularity():
    """Uniform popularity: item counts vary little; Zipf(1.1): counts fall as a power of the rank with
    exponent near -1.1 (fitted over ranks 10-1000) and the top 1% of items hold about half the items."""
    for name in ("tiny", "sparse_mid"):
        w = synth.make_workload(name)
        f = np.bincount(w["items"], minlength=w["N"]).astype(float)
        assert f.std() / f.mean() < 0.5, name
    w = synth.make_workload("large_sparse", D=100_000)
    f = np.sort(np.bincount(w["items"], minlength=w["N"]))[::-1].astype(float)
    r = np.arange(1, len(f) + 1)
    m = (r >= 10) & (r <= 1000)
    slope = np.polyfit(np.log(r[m]), np.log(f[m]), 1)[0]
    assert -1.3 < slope < -0.9
    assert f[: len(f) // 100].sum() / f.sum() > 0.4


def test_bernoulli_dense_law():
    """dense_deep: item i is in each transaction independently with p_i = 0.3 + 0.65 i / 74, so every
    item's frequency lies within 5 standard errors of p_i and the mean length near sum p_i = 46.875."""
    w = synth.make_workload("dense_deep", D=20_000)
    assert_set_semantics(w)
    D, N = w["D"], w["N"]
    p = 0.3 + 0.65 * np.arange(N) / (N - 1)
    freq = np.bincount(w["items"], minlength=N) / D
    assert np.all(np.abs(freq - p) < 5 * np.sqrt(p * (1 - p) / D))
    L = lengths(w)
    assert abs(L.mean() - p.sum()) < 5 * math.sqrt((p * (1 - p)).sum() / D)


def test_exactly_k_dense_law():
    """dense_exact37: every transaction holds exactly 37 distinct items, drawn with weights rising with i."""
    w = synth.make_workload("dense_exact37", D=5_000)
    assert_set_semantics(w)
    assert np.all(lengths(w) == 37)
    f = np.bincount(w["items"], minlength=w["N"])
    assert f[-10:].mean() > f[:10].mean()


def test_serving_request_law():
    """2,000 requests: D log-uniform on [1e4, 5e5], N uniform on [100, 5000], TL uniform on [5, 30],
    relative minsup log-uniform on [0.1%, 5%] with minsup = ceil(rel D), Poisson arrivals at 20/s,
    request k seeded 1000 + k; every sample mean within 5 standard errors of the law's."""
    n = 2000
    reqs = synth.serving_requests(n, rate=20.0)
    assert [r["k"] for r in reqs] == list(range(n)) and [r["seed"] for r in reqs] == [1000 + k for k in range(n)]
    D = np.array([r["D"] for r in reqs], dtype=float)
    N = np.array([r["N"] for r in reqs], dtype=float)
    TL = np.array([r["TL"] for r in reqs])
    rel = np.array([r["rel_minsup"] for r in reqs])
    arr = np.array([r["arrival_s"] for r in reqs])
    assert D.min() >= 1e4 and D.max() <= 5e5 and N.min() >= 100 and N.max() <= 5000
    assert TL.min() >= 5 and TL.max() <= 30 and rel.min() >= 0.001 and rel.max() <= 0.05
    assert all(r["minsup"] == max(1, math.ceil(r["rel_minsup"] * r["D"] - 1e-9)) for r in reqs)
    assert all(r["npat"] == 2 * r["N"] and r["PL"] == 4.0 for r in reqs)

    def near_uniform(x, lo, hi):  # sample mean of a uniform variable on [lo, hi]
        return abs(x.mean() - (lo + hi) / 2) < 5 * (hi - lo) / math.sqrt(12 * len(x))

    assert near_uniform(np.log(D), math.log(1e4), math.log(5e5))
    assert near_uniform(N, 100, 5000)
    assert near_uniform(TL, 5, 30)
    assert near_uniform(np.log(rel), math.log(0.001), math.log(0.05))
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() - 0.05) < 5 * 0.05 / math.sqrt(n)  # exponential gaps: sd = mean


def test_relative_minsup_is_exact_decimal_ceiling():
    """Reading 8: minsup = ceil(rel D) computed on the decimal value of rel, at least 1: the workloads'
    absolute minsups (100, 250, 30,000, 500), and cases where binary floating point would round wrong
    (0.07 x 100 = 7.000000000000001 in doubles, whose ceiling is 8)."""
    assert [synth.make_workload(n)["minsup"] for n in ("tiny", "sparse_mid", "dense_deep", "large_sparse")] == \
        [100, 250, 30_000, 500]
    assert synth.abs_minsup(0.07, 100) == 7
    assert synth.abs_minsup(0.29, 100) == 29
    assert synth.abs_minsup(0.071, 100) == 8
    assert synth.abs_minsup(0.0001, 100) == 1
    assert synth.abs_minsup(0.0, 100) == 1
