"""CPU oracle for frequent-itemset mining -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It never imports the GPU package and the GPU
package never imports it; the C code in ``fim_oracle.c`` shares nothing with
the CUDA sources.  See ``fim_oracle.c`` for the cited definitions.

Functions return results as ``(set_offsets u64[n+1], set_items u32[...],
supports u32[n])`` sorted canonically: items ascending inside a set, sets in
the thesis's lexicographic order (Ch. 9), counts exact.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fim_oracle.c")
_LIB = os.path.join(_HERE, "libfimoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fim_oracle.c with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            PP = ctypes.POINTER(ctypes.c_void_p)
            for name in ("oracle_eclat", "oracle_bruteforce", "oracle_apriori"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int
                f.argtypes = [P, P, u32, u32, u32, PP]
            lib.oracle_eclat_mt.restype = ctypes.c_int
            lib.oracle_eclat_mt.argtypes = [P, P, u32, u32, u32, u32, PP]
            lib.oracle_result_free.restype = None
            lib.oracle_result_free.argtypes = [P]
            lib.oracle_result_sort.restype = ctypes.c_int
            lib.oracle_result_sort.argtypes = [P]
            lib.oracle_result_n_sets.restype = u64
            lib.oracle_result_n_sets.argtypes = [P]
            lib.oracle_result_n_items.restype = u64
            lib.oracle_result_n_items.argtypes = [P]
            lib.oracle_result_copy.restype = None
            lib.oracle_result_copy.argtypes = [P, P, P, P]
            lib.oracle_check.restype = ctypes.c_int
            lib.oracle_check.argtypes = [P, P, u32, u32, u32, u64, P, P, P, u64, ctypes.POINTER(u64)]
            lib.oracle_item_order.restype = ctypes.c_int
            lib.oracle_item_order.argtypes = [P, P, u32, u32, u32, P, ctypes.POINTER(u32)]
            lib.oracle_class_costs.restype = ctypes.c_int
            lib.oracle_class_costs.argtypes = [P, P, u32, u32, u32, dbl, dbl, u64, P, P, ctypes.POINTER(u32),
                                               ctypes.POINTER(u64)]
            lib.oracle_class_costs_kind.restype = ctypes.c_int
            lib.oracle_class_costs_kind.argtypes = [P, P, u32, u32, u32, dbl, dbl, u64, ctypes.c_int, P, P,
                                                    ctypes.POINTER(u32), ctypes.POINTER(u64)]
            lib.oracle_class_costs_limit.restype = ctypes.c_int
            lib.oracle_class_costs_limit.argtypes = [P, P, u32, u32, u32, dbl, dbl, u64, ctypes.c_int, u64, P, P,
                                                     ctypes.POINTER(u32), ctypes.POINTER(u64), ctypes.POINTER(u32)]
            lib.oracle_splitmix64_at.restype = u64
            lib.oracle_splitmix64_at.argtypes = [u64, u64]
            _lib = lib
    return _lib


def _csr(offsets, items):
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    items = np.ascontiguousarray(items, dtype=np.uint32)
    if items.size == 0:
        items = np.zeros(1, dtype=np.uint32)
    return offsets, items


def _run(fname, offsets, items, N, minsup, *extra):
    lib = _load()
    offsets, items = _csr(offsets, items)
    D = offsets.size - 1
    h = ctypes.c_void_p()
    rc = getattr(lib, fname)(offsets.ctypes.data, items.ctypes.data, D, N, minsup, *extra, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"{fname} failed with code {rc}")
    try:
        if lib.oracle_result_sort(h) != 0:
            raise MemoryError("oracle sort failed")
        n = lib.oracle_result_n_sets(h)
        ni = lib.oracle_result_n_items(h)
        so = np.empty(n + 1, dtype=np.uint64)
        si = np.empty(max(ni, 1), dtype=np.uint32)
        sp = np.empty(max(n, 1), dtype=np.uint32)
        lib.oracle_result_copy(h, so.ctypes.data, si.ctypes.data, sp.ctypes.data)
        return so, si[:ni], sp[:n]
    finally:
        lib.oracle_result_free(h)


def eclat(offsets, items, N: int, minsup: int):
    """O1: Eclat-DFS over sorted tidlists (App. B.3.2)."""
    return _run("oracle_eclat", offsets, items, N, minsup)


def eclat_mt(offsets, items, N: int, minsup: int, threads: int = 0):
    """O1 with the one-item classes spread over ``threads`` host threads (0: every core); same output."""
    return _run("oracle_eclat_mt", offsets, items, N, minsup, threads or (os.cpu_count() or 1))


def bruteforce(offsets, items, N: int, minsup: int):
    """O2: every non-empty subset, counted by scanning (N <= 20)."""
    return _run("oracle_bruteforce", offsets, items, N, minsup)


def apriori(offsets, items, N: int, minsup: int):
    """O3: level-wise Apriori (App. B.1)."""
    return _run("oracle_apriori", offsets, items, N, minsup)


CHECK_CODES = {
    0: "ok", 1: "support differs from recount", 2: "support below minsup", 3: "parent missing or smaller support",
    4: "frequent extension missing", 5: "singleton missing or wrong", 6: "duplicate or malformed set",
}


def check(offsets, items, N: int, minsup: int, set_offsets, set_items, supports, stride: int = 1):
    """O4: certificate check of an output; returns (code, bad_index); code 0 = exact."""
    lib = _load()
    offsets, items = _csr(offsets, items)
    so = np.ascontiguousarray(set_offsets, dtype=np.uint64)
    si = np.ascontiguousarray(set_items, dtype=np.uint32)
    sp = np.ascontiguousarray(supports, dtype=np.uint32)
    if si.size == 0:
        si = np.zeros(1, dtype=np.uint32)
    if sp.size == 0:
        sp = np.zeros(1, dtype=np.uint32)
    bad = ctypes.c_uint64(0)
    rc = lib.oracle_check(offsets.ctypes.data, items.ctypes.data, offsets.size - 1, N, minsup, so.size - 1,
                          so.ctypes.data, si.ctypes.data, sp.ctypes.data, stride, ctypes.byref(bad))
    if rc < 0:
        raise MemoryError("oracle check failed to allocate")
    return rc, bad.value


def item_order(offsets, items, N: int, prefilter_minsup: int = 0):
    """Kept items (support >= prefilter) by ascending support, ties by id."""
    lib = _load()
    offsets, items = _csr(offsets, items)
    out = np.empty(max(N, 1), dtype=np.uint32)
    nk = ctypes.c_uint32(0)
    rc = lib.oracle_item_order(offsets.ctypes.data, items.ctypes.data, offsets.size - 1, N, prefilter_minsup,
                               out.ctypes.data, ctypes.byref(nk))
    if rc != 0:
        raise ValueError(f"item_order failed {rc}")
    return out[: nk.value]


SAMPLE_ITEMSET_LIMIT = 1 << 20


def class_costs(offsets, items, N: int, prefilter_minsup: int, sample_rate: float, rel_minsup: float, seed: int,
                kind: int = 0, limit: int = SAMPLE_ITEMSET_LIMIT, return_minsup: bool = False):
    """Sample-based relative class sizes and their LPT order; returns (cost f64[N_f], order u32[N_f], |F_s|)
    (plus the sample minsup used when ``return_minsup``).

    kind 0: share of the sample's frequent itemsets; kind 1: share of the bitmap intersections.
    While the sample has more than ``limit`` frequent itemsets (0: no limit) its minsup doubles."""
    lib = _load()
    offsets, items = _csr(offsets, items)
    cost = np.zeros(max(N, 1), dtype=np.float64)
    order = np.zeros(max(N, 1), dtype=np.uint32)
    nk = ctypes.c_uint32(0)
    nfs = ctypes.c_uint64(0)
    ms = ctypes.c_uint32(0)
    rc = lib.oracle_class_costs_limit(offsets.ctypes.data, items.ctypes.data, offsets.size - 1, N, prefilter_minsup,
                                      sample_rate, rel_minsup, seed, kind, limit, cost.ctypes.data, order.ctypes.data,
                                      ctypes.byref(nk), ctypes.byref(nfs), ctypes.byref(ms))
    if rc != 0:
        raise ValueError(f"class_costs failed {rc}")
    if return_minsup:
        return cost[: nk.value], order[: nk.value], nfs.value, ms.value
    return cost[: nk.value], order[: nk.value], nfs.value


def splitmix64_at(seed: int, k: int) -> int:
    """k-th output (0-based) of SplitMix64 started at state ``seed``."""
    return _load().oracle_splitmix64_at(seed, k)


def extension_supports(offsets, items, N: int, prefix, candidates):
    """supp(P u {c}) for every candidate c (Def. "Itemset cover and support", Ch. 2: the number of
    transactions that contain every item of the set), counted by one scan of the transactions: a
    transaction covers P u {c} iff it holds all distinct items of P and also c.  Repeated items in a
    transaction or in P count once; a candidate inside P gives supp(P).  Returns u64[len(candidates)]."""
    offsets, items = _csr(offsets, items)
    D = offsets.size - 1
    prefix = np.unique(np.asarray(prefix, dtype=np.int64))
    cand = np.asarray(candidates, dtype=np.int64)
    if prefix.size == 0 or (prefix.size and (prefix.min() < 0 or prefix.max() >= N)) or \
            (cand.size and (cand.min() < 0 or cand.max() >= N)):
        raise ValueError("prefix must be non-empty and every id < N")
    tx = np.repeat(np.arange(D, dtype=np.int64), np.diff(offsets.astype(np.int64)))
    body = items[int(offsets[0]): int(offsets[-1])].astype(np.int64)
    pairs = np.unique(tx * N + body)  # distinct (transaction, item)
    ptx, pit = pairs // N, pairs % N
    in_p = np.isin(pit, prefix)
    covers_p = np.bincount(ptx[in_p], minlength=D) == prefix.size
    per_item = np.bincount(pit[covers_p[ptx]], minlength=N)
    return per_item[cand].astype(np.uint64)


def closed_maximal(offsets, items, N: int, minsup: int):
    """Flags of every frequent itemset (Ch. 2): bit 0 = closed (Def. "Closed itemset": the itemset equals
    its closure, the set of items contained in every transaction that contains it), bit 1 = maximal
    (Def. "Maximal Frequent Itemset": no proper superset is frequent).  Both follow from the counts of
    every item over the transactions containing the itemset: closed iff no item outside it is counted
    supp times, maximal iff no item outside it is counted at least minsup times.  Returns the O1 result
    (canonical order) and the flags, u8 per itemset."""
    so, si, sp = eclat(offsets, items, N, minsup)
    offsets, items = _csr(offsets, items)
    D = offsets.size - 1
    tx = np.repeat(np.arange(D, dtype=np.int64), np.diff(offsets.astype(np.int64)))
    body = items[int(offsets[0]): int(offsets[-1])].astype(np.int64)
    pairs = np.unique(tx * N + body)  # distinct (transaction, item)
    ptx, pit = pairs // N, pairs % N
    tids = [ptx[pit == i] for i in range(N)]  # tidlist of every item (ascending)
    flags = np.zeros(len(sp), dtype=np.uint8)
    for k in range(len(sp)):
        s = [int(v) for v in si[so[k]:so[k + 1]]]
        t = tids[s[0]]
        for v in s[1:]:
            t = np.intersect1d(t, tids[v], assume_unique=True)
        assert len(t) == int(sp[k])
        cnt = np.bincount(pit[np.isin(ptx, t)], minlength=N)
        cnt[s] = 0
        closed = not np.any(cnt == len(t))
        maximal = not np.any(cnt >= minsup)
        flags[k] = (1 if closed else 0) | (2 if maximal else 0)
    return so, si, sp, flags
