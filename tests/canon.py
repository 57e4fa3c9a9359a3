"""Canonical form and digest of a frequent-itemset result (test infrastructure).

Canonical order: items ascending inside a set, sets in the thesis's
lexicographic order (Ch. 9: item by item, a proper prefix first).  The digest
hashes, for every set in that order, its length, its items and its support as
little-endian u32 words."""
import hashlib

import numpy as np


def canonical_order(set_offsets, set_items):
    so = np.asarray(set_offsets, dtype=np.int64)
    n = len(so) - 1
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    lens = np.diff(so)
    width = int(lens.max())
    mat = np.full((n, width), -1, dtype=np.int64)
    rows = np.repeat(np.arange(n), lens)
    cols = np.arange(len(set_items)) - np.repeat(so[:-1], lens)
    mat[rows, cols] = np.asarray(set_items, dtype=np.int64)
    # items inside a set are ascending already (both producers guarantee it); check
    if width > 1:
        inner = mat[:, 1:] - mat[:, :-1]
        ok = (inner > 0) | (mat[:, 1:] == -1)
        if not np.all(ok):
            raise ValueError("items not ascending inside a set")
    return np.lexsort(tuple(mat[:, c] for c in range(width - 1, -1, -1)))


def digest(set_offsets, set_items, supports):
    """(n_sets, n_items, sum of supports, max length, sha256 hex) of the canonical result."""
    so = np.asarray(set_offsets, dtype=np.int64)
    si = np.asarray(set_items, dtype=np.uint32)
    sp = np.asarray(supports, dtype=np.uint32)
    order = canonical_order(so, si)
    lens = np.diff(so)
    h = hashlib.sha256()
    # serialise in canonical order: [len, items..., support] per set
    rec_len = lens[order] + 2
    out = np.empty(int(rec_len.sum()), dtype="<u4")
    pos = np.concatenate([[0], np.cumsum(rec_len)[:-1]]) if len(order) else np.zeros(0, dtype=np.int64)
    out[pos] = lens[order]
    out[pos + rec_len - 1] = sp[order]
    starts = so[:-1][order]
    if len(order):
        lo = lens[order]
        within = np.arange(int(lens.sum())) - np.repeat(np.cumsum(lo) - lo, lo)  # position inside each set
        out[np.repeat(pos + 1, lo) + within] = si[np.repeat(starts, lo) + within]
    h.update(out.tobytes())
    return {"n_sets": int(len(sp)), "n_items": int(lens.sum()), "sum_supports": int(sp.astype(np.int64).sum()),
            "max_len": int(lens.max()) if len(lens) else 0, "sha256": h.hexdigest()}
