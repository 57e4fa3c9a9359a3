"""Seeded synthetic transaction databases (input generation only).

The generator lives in ``synth.c`` (plain C, SplitMix64 streams) and holds none
of the mining arithmetic; the CPU oracle and the GPU path both read the CSR
arrays it returns.  The shared library is compiled with gcc on first use (and
by ``__graft_entry__.build()``).

Workload recipes.  The thesis measures on databases from the IBM generator
(Sec. 11.2: transactions built from embedded patterns, parametrised by average
transaction length, item count, pattern count and pattern length); those files
are not available, and the pattern-embedding recipe in ``synth.c`` stands in
for them with the following shapes:

* ``tiny``         D=10,000  N=100    TL=10 PL=4 npat=200    uniform, seed 0, minsup 100
* ``sparse_mid``   D=100,000 N=1,000  TL=10 PL=4 npat=2,000  uniform, seed 1, minsup 250
* ``dense_deep``   D=50,000  N=75     Bernoulli p_i=0.3+0.65*i/74, seed 2, minsup 30,000
* ``large_sparse`` D=1,000,000 N=10,000 TL=20 PL=6 npat=20,000 Zipf(1.1), seed 3, minsup 500
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libfimsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into libfimsynth.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, dbl, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
            lib.synth_pattern_db.restype = P
            lib.synth_pattern_db.argtypes = [u64, u32, u32, dbl, dbl, u32, i32, dbl, dbl, dbl]
            lib.synth_dense_bernoulli.restype = P
            lib.synth_dense_bernoulli.argtypes = [u64, u32, u32, dbl, dbl]
            lib.synth_dense_fixed.restype = P
            lib.synth_dense_fixed.argtypes = [u64, u32, u32, u32, dbl, dbl]
            lib.synth_num_tx.restype = u32
            lib.synth_num_tx.argtypes = [P]
            lib.synth_nnz.restype = u64
            lib.synth_nnz.argtypes = [P]
            lib.synth_copy.restype = None
            lib.synth_copy.argtypes = [P, P, P]
            lib.synth_free.restype = None
            lib.synth_free.argtypes = [P]
            lib.synth_exp.restype = dbl
            lib.synth_exp.argtypes = [dbl]
            lib.synth_log.restype = dbl
            lib.synth_log.argtypes = [dbl]
            lib.synth_splitmix64_next.restype = u64
            lib.synth_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
            _lib = lib
    return _lib


def _take(handle):
    lib = _load()
    if not handle:
        raise MemoryError("synthetic generator failed")
    try:
        D = lib.synth_num_tx(handle)
        nnz = lib.synth_nnz(handle)
        offsets = np.empty(D + 1, dtype=np.uint32)
        items = np.empty(max(nnz, 1), dtype=np.uint32)
        lib.synth_copy(handle, offsets.ctypes.data, items.ctypes.data)
        return offsets, items[:nnz]
    finally:
        lib.synth_free(handle)


def pattern_db(seed: int, D: int, N: int, TL: float, PL: float, npat: int, popularity: str = "uniform",
               zipf_s: float = 1.1, q_noise: float = 0.2, keep_p: float = 0.8):
    """Pattern-embedded database; returns (tx_offsets u32[D+1], tx_items u32[nnz])."""
    zipf = {"uniform": 0, "zipf": 1}[popularity]
    return _take(_load().synth_pattern_db(seed, D, N, TL, PL, npat, zipf, zipf_s, q_noise, keep_p))


def dense_bernoulli(seed: int, D: int, N: int, p_lo: float = 0.3, p_hi: float = 0.95):
    """Item i present independently with p_i = p_lo + (p_hi - p_lo) * i / (N - 1)."""
    return _take(_load().synth_dense_bernoulli(seed, D, N, p_lo, p_hi))


def dense_fixed(seed: int, D: int, N: int, k: int, p_lo: float = 0.3, p_hi: float = 0.95):
    """Exactly k distinct items per transaction, weighted draws without replacement."""
    return _take(_load().synth_dense_fixed(seed, D, N, k, p_lo, p_hi))


def splitmix64_stream(state: int, n: int):
    """First n outputs of SplitMix64 from the given state (for pinning the generator)."""
    lib = _load()
    s = ctypes.c_uint64(state)
    return [lib.synth_splitmix64_next(ctypes.byref(s)) for _ in range(n)]


def csr_digest(offsets, items) -> str:
    """SHA-256 of a CSR database (little-endian u32 offsets then items)."""
    import hashlib
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(offsets, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(items, dtype="<u4").tobytes())
    return h.hexdigest()


# ---------------------------------------------------------------------------
# Named workloads.  Each returns a dict with the CSR arrays and the absolute
# minimum support; ``make_workload(name, D=...)`` keeps the laws and changes D.

WORKLOADS = {
    "tiny": dict(kind="pattern", seed=0, D=10_000, N=100, TL=10.0, PL=4.0, npat=200, popularity="uniform",
                 rel_minsup=0.01, word_bits=32),
    "sparse_mid": dict(kind="pattern", seed=1, D=100_000, N=1_000, TL=10.0, PL=4.0, npat=2_000,
                       popularity="uniform", rel_minsup=0.0025, word_bits=64),
    "dense_deep": dict(kind="bernoulli", seed=2, D=50_000, N=75, p_lo=0.3, p_hi=0.95, rel_minsup=0.60,
                       word_bits=64),
    "dense_exact37": dict(kind="fixed", seed=2, D=50_000, N=75, k=37, p_lo=0.3, p_hi=0.95, rel_minsup=0.60,
                          word_bits=64),
    "large_sparse": dict(kind="pattern", seed=3, D=1_000_000, N=10_000, TL=20.0, PL=6.0, npat=20_000,
                         popularity="zipf", rel_minsup=0.0005, word_bits=64),
}


def abs_minsup(rel: float, D: int) -> int:
    """ceil(rel * D) in exact decimal arithmetic (rel given as a decimal fraction), at least 1."""
    from fractions import Fraction
    v = math.ceil(Fraction(repr(rel)) * D)
    return max(1, int(v))


def make_workload(name: str, D: int | None = None, seed: int | None = None):
    """Generate a named workload, optionally with another D (the laws stay the same)."""
    w = dict(WORKLOADS[name])
    if D is not None:
        w["D"] = D
    if seed is not None:
        w["seed"] = seed
    kind = w["kind"]
    if kind == "pattern":
        off, items = pattern_db(w["seed"], w["D"], w["N"], w["TL"], w["PL"], w["npat"], w["popularity"])
    elif kind == "bernoulli":
        off, items = dense_bernoulli(w["seed"], w["D"], w["N"], w["p_lo"], w["p_hi"])
    else:
        off, items = dense_fixed(w["seed"], w["D"], w["N"], w["k"], w["p_lo"], w["p_hi"])
    w["offsets"] = off
    w["items"] = items
    w["minsup"] = abs_minsup(w["rel_minsup"], w["D"])
    return w


def serving_requests(n: int, seed: int = 4, rate: float = 20.0, D_range=(10_000, 500_000), N_range=(100, 5_000),
                     TL_range=(5.0, 30.0), rel_range=(0.001, 0.05)):
    """Request specs for the serving workload: Poisson arrivals and per-request database laws.

    Request k uses database seed 1000 + k; arrivals, sizes and minsups come from a
    SplitMix64 stream seeded with ``seed``.  Returns a list of dicts (no databases
    are generated here; call ``request_db`` for each)."""
    st = [int(seed * 0x2545F4914F6CDD1D + 0xABCDEF) & (2**64 - 1)]

    def unit():
        v = splitmix64_stream(st[0], 1)[0]
        st[0] = (st[0] + 0x9E3779B97F4A7C15) & (2**64 - 1)
        return ((v >> 11) + 1) / 9007199254740992.0

    t = 0.0
    reqs = []
    for k in range(n):
        t += -math.log(unit()) / rate
        D = int(round(math.exp(math.log(D_range[0]) + unit() * (math.log(D_range[1]) - math.log(D_range[0])))))
        N = int(N_range[0] + min(N_range[1] - N_range[0], int(unit() * (N_range[1] - N_range[0] + 1))))
        TL = TL_range[0] + unit() * (TL_range[1] - TL_range[0])
        rel = math.exp(math.log(rel_range[0]) + unit() * (math.log(rel_range[1]) - math.log(rel_range[0])))
        reqs.append(dict(k=k, arrival_s=t, seed=1000 + k, D=D, N=N, TL=TL, PL=4.0, npat=2 * N, rel_minsup=rel,
                         minsup=max(1, math.ceil(rel * D))))
    return reqs


def request_db(req):
    """Generate the database of one serving request (pattern-embedded, uniform popularity)."""
    return pattern_db(req["seed"], req["D"], req["N"], req["TL"], req["PL"], req["npat"], "uniform")
