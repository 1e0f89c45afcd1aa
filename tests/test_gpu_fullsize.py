"""Full-size workloads on the GPU, in the launch configuration bench.py times.

The oracle cannot build 256 MiB or 2 GiB texts in seconds, so these check
sampled outputs against the definition (bytes.find gives the leftmost
occurrence of a sampled block or pair string), properties that hold at any
size (every pointer copies its source, lies strictly left, targets marked
blocks; the leaf text is the marked last-level blocks), naive query counts
for sampled symbols, equality of the two independent window-scan strategies
(anchored and dense), of the one- and two-phase window tests, and of the
parallel pruning rounds with the sequential right-to-left finish.
"""
import numpy as np
import pytest
import torch

from paper_2512_23314_gb300 import bt, workloads
from tests.helpers import check_leftmost_sampled, check_pointers
from tests.test_gpu_parity import run_queries

pytestmark = pytest.mark.gpu


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
