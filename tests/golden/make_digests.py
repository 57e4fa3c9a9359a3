"""Writes tests/golden/digests.json: for every named workload, the SHA-256 of
its generated CSR database and the digest of the CPU oracle's frequent
itemsets (count, items, support sum, longest set, SHA-256 of the canonical
output).  Calls only the seeded generator and oracle/ (O1 Eclat); the GPU path
is never involved.  The large workload takes about 15 minutes single-threaded.

    python tests/golden/make_digests.py [name ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import canon  # noqa: E402
import oracle  # noqa: E402
from paper_2108_05038_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "digests.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        w = synth.make_workload(name)
        t0 = time.time()
        so, si, sp = oracle.eclat(w["offsets"], w["items"], w["N"], w["minsup"])
        dt = time.time() - t0
        data[name] = {"csr_sha256": synth.csr_digest(w["offsets"], w["items"]), "D": w["D"], "N": w["N"],
                      "nnz": int(len(w["items"])), "minsup": w["minsup"], "oracle": canon.digest(so, si, sp),
                      "oracle_seconds": round(dt, 1)}
        print(name, data[name], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "sparse_mid", "dense_deep", "dense_exact37", "large_sparse"])
