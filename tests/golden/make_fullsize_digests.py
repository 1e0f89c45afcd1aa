#!/usr/bin/env python
"""Write the oracle's digests of the full-size single-text workloads.

For each workload this builds the block tree with the CPU oracle (plain,
single-threaded; section 3 of the paper for the tree, section 3.1 for the
leftmost occurrences, every fingerprint match verified) and stores, in
``tests/golden/fullsize_<workload>.json``:

* the SHA-256 and length of the generated text (so that a different input,
  e.g. from another numpy release, is told apart from a wrong build);
* the SHA-256 and length of the canonical serialization of the tree (marks,
  pointers, offsets and leaf text of every level);
* per level: block count and block size after pruning (read back from the
  serialization), and the block count and covered bytes of the unpruned
  construction (the oracle's statistics);
* seeded access / rank / select queries with the oracle's answers.

Only ``oracle/`` and the seeded input generators are used; nothing here comes
from the CUDA library.  Runtime: minutes for the 256 MiB text, most of an hour
for the 2 GiB genome (one core each).

    python tests/golden/make_fullsize_digests.py text_versions_256MiB
    python tests/golden/make_fullsize_digests.py dna_genome_2GiB
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_23314_gb300 import workloads  # noqa: E402

WORKLOADS = {
    # name: (generator, sigma, tau, leaf_len)
    "text_versions_256MiB": (lambda: workloads.text_versions(), 96, 4, 32),
    "dna_genome_2GiB": (lambda: workloads.dna_genome(), 5, 4, 64),
}
NQ = 1000  # queries of each kind


def sha(b) -> str:
    return hashlib.sha256(b).hexdigest()


def queries(tree: "oracle.Tree", T: np.ndarray, seed: int) -> dict:
    """NQ seeded queries of each kind (access i ~ U[0, n); rank: a present
    symbol, i ~ U[0, n]; select: a present symbol, j ~ U[1, count]) and the
    oracle's answers."""
    rng = np.random.default_rng(seed)
    n = len(T)
    counts = np.bincount(T, minlength=256)
    syms = np.flatnonzero(counts)
    acc_i = rng.integers(0, n, NQ)
    rc = syms[rng.integers(0, len(syms), NQ)]
    ri = rng.integers(0, n + 1, NQ)
    sc = syms[rng.integers(0, len(syms), NQ)]
    sj = (rng.random(NQ) * counts[sc]).astype(np.int64) + 1
    return {
        "access": [[int(i), tree.access(int(i))] for i in acc_i],
        "rank": [[int(c), int(i), tree.rank(int(c), int(i))] for c, i in zip(rc, ri)],
        "select": [[int(c), int(j), tree.select(int(c), int(j))] for c, j in zip(sc, sj)],
    }


def digest(name: str) -> dict:
    gen, sigma, tau, leaf = WORKLOADS[name]
    t0 = time.time()
    T = gen()
    rec = {"workload": name, "sigma": sigma, "tau": tau, "leaf_len": leaf, "prune": True,
           "n": int(len(T)), "text_sha256": sha(T.tobytes())}
    t1 = time.time()
    tree = oracle.build(T, tau, leaf, prune=True)
    t2 = time.time()
    blob = tree.export()
    p = oracle.parse(blob, as_numpy=True)
    st = tree.stats()
    rec["export_sha256"] = sha(blob)
    rec["export_len"] = len(blob)
    rec["levels"] = [{"b": lv.b, "nblocks_pruned": int(len(lv.marks)),
                      "nmarked_pruned": int(np.count_nonzero(lv.marks)),
                      "nblocks": int(s["nblocks"]), "cov": int(s["cov"])}
                     for lv, s in zip(p.levels, st)]
    rec["leaf_bytes"] = len(p.leaf_text)
    rec["queries"] = queries(tree, T, seed=0xB7EE0100)
    rec["oracle_build_s"] = round(t2 - t1, 1)
    rec["generate_s"] = round(t1 - t0, 1)
    return rec


def main():
    names = sys.argv[1:] or sorted(WORKLOADS)
    for name in names:
        rec = digest(name)
        path = os.path.join(HERE, f"fullsize_{name}.json")
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")
        print(f"{name}: oracle build {rec['oracle_build_s']} s -> {path}", flush=True)


if __name__ == "__main__":
    main()
