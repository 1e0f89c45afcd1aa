"""Full-size workloads on the GPU, in the launch configuration bench.py times.

Bit-exact against the oracle at full size: tests/golden/fullsize_*.json holds,
for the 256 MiB versioned text and the 2 GiB DNA copies, the SHA-256 of the
oracle's canonical serialization of the pruned tree, its per-level block and
mark counts, and 1000 seeded access / rank / select answers, written by
tests/golden/make_fullsize_digests.py from oracle/ alone (minutes and most of
an hour of CPU).  The GPU build must reproduce the digest exactly; a
mismatch is reported by the first level whose counts differ.

Beyond the digest: sampled outputs against the definition (bytes.find gives
the leftmost occurrence of a sampled block or pair string), properties that
hold at any size (every pointer copies its source, lies strictly left,
targets marked blocks; the leaf text is the marked last-level blocks), naive
query counts for sampled symbols, equality of the two window-scan strategies
(anchored and dense), of the one- and two-phase window tests, and of the
parallel pruning rounds with the sequential right-to-left finish.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

from paper_2512_23314_gb300 import bt, workloads
from tests.helpers import check_leftmost_sampled, check_pointers
from tests.test_gpu_parity import run_queries

pytestmark = pytest.mark.gpu


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def check_digest(name, T, tree, blob):
    """The GPU tree of a full-size workload against the oracle's stored digest."""
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        g = json.load(f)
    assert hashlib.sha256(T.tobytes()).hexdigest() == g["text_sha256"], "generated text differs"
    if hashlib.sha256(blob).hexdigest() != g["export_sha256"] or len(blob) != g["export_len"]:
        import oracle
        p = oracle.parse(blob, as_numpy=True)
        for l, (lv, want) in enumerate(zip(p.levels, g["levels"])):
            got = (lv.b, len(lv.marks), int(np.count_nonzero(lv.marks)))
            exp = (want["b"], want["nblocks_pruned"], want["nmarked_pruned"])
            assert got == exp, f"level {l}: (b, blocks, marked) {got} != oracle {exp}"
        assert len(p.levels) == len(g["levels"]), "level count differs"
        raise AssertionError("export differs from the oracle's (same per-level counts)")
    q = g["queries"]
    for kind, key in ((bt.BT_Q_ACCESS, "access"), (bt.BT_Q_RANK, "rank"), (bt.BT_Q_SELECT, "select")):
        rows = np.array(q[key], dtype=np.int64)
        args = rows[:, 0] if kind == bt.BT_Q_ACCESS else rows[:, :2].ravel()
        out = torch.empty(len(rows), dtype=torch.int64, device="cuda")
        tree.query_batch(kind, torch.from_numpy(np.ascontiguousarray(args)).cuda(), out)
        assert np.array_equal(out.cpu().numpy(), rows[:, -1]), key


def _build(d_text, sigma, tau, leaf, **kw):
    t = bt.Tree(d_text, sigma, tau, leaf, bt.BuildOptions(**kw))
    return t, t.export()


@pytest.mark.parametrize("name", ["text_versions_256MiB", "dna_genome_2GiB"])
def test_full_size_workload(name):
    if name == "text_versions_256MiB":
        T, sigma, tau, leaf, per_level = workloads.text_versions(), 96, 4, 32, 8
    else:
        T, sigma, tau, leaf, per_level = workloads.dna_genome(), 5, 4, 64, 2
    d = torch.from_numpy(T).cuda()
    t, blob = _build(d, sigma, tau, leaf)
    check_digest(name, T, t, blob)
    _, blob_dense = _build(d, sigma, tau, leaf, dense_scan=True)
    assert blob == blob_dense
    if name == "text_versions_256MiB":
        # Pruning by parallel frontier rounds (wide ones on many CTAs, narrow
        # ones on one) against the sequential right-to-left rule alone.
        _, blob_seq = _build(d, sigma, tau, leaf, max_rounds=1)
        assert blob == blob_seq
    else:
        # The two-phase window tests the bench uses on this workload.
        _, blob_two = _build(d, sigma, tau, leaf, two_phase=True)
        assert blob == blob_two
    p, blocks = check_pointers(T, blob, sample=300)
    check_leftmost_sampled(T, p, blocks, per_level=per_level)
    syms = np.unique(T)[:3]
    run_queries(t, T, 30_000, 17, symbols=syms)
    t.close()
    tu, blob_u = _build(d, sigma, tau, leaf, prune=False)
    pu, blocks_u = check_pointers(T, blob_u, sample=300)
    check_leftmost_sampled(T, pu, blocks_u, per_level=per_level, seed=3)
    st = tu.stats()
    assert st[0]["cov"] == len(T)
    assert all(s["collisions"] == 0 for s in st)
