"""Space-efficient rank/select support (BT_FLAG_LEAF_COUNTS).

The last level stores no symbol counters; rank and select count the leaf
text when they need one.  The tree must be byte-identical to the default
build, every query must equal naive counts on T, and the tree must hold
fewer device bytes.
"""
import numpy as np
import pytest
import torch

from paper_2512_23314_gb300 import bt, workloads
from tests.test_gpu_parity import gpu_export, run_queries

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,tau,leaf,sigma,seed", [
    (5000, 2, 4, 30, 1),           # tiny blocks: leaf text windows cross aligned words
    (200_001, 4, 16, 30, 2),
    (1 << 20, 2, 16, 96, 3),
    (777_777, 3, 7, 5, 4),         # odd leaf length and arity, unaligned leaf rows
    (3000, 4, 64, 200, 5),         # a two-level tree
])
def test_leaf_counts_tree_and_queries(n, tau, leaf, sigma, seed):
    T = workloads.text_versions(n=n, base_len=max(512, n // 20), sigma=sigma, seed=seed)
    sigma_eff = max(sigma, len(np.unique(T)))
    for prune in (True, False):
        td, blob = gpu_export(T, sigma_eff, tau, leaf, prune=prune)
        tc, blob_c = gpu_export(T, sigma_eff, tau, leaf, prune=prune, leaf_counts=True)
        assert blob_c == blob
        run_queries(tc, T, 20000, seed)
        if td.stats()[-1]["nblocks"] > 0 and len(td.stats()) >= 2:
            assert bt.bt_device_bytes(tc.handle) < bt.bt_device_bytes(td.handle)
        td.close()
        tc.close()


def test_leaf_counts_full_size_queries_sampled():
    T = workloads.text_versions(n=64 << 20)
    d = torch.from_numpy(T).cuda()
    t = bt.Tree(d, 96, 4, 32, bt.BuildOptions(leaf_counts=True))
    run_queries(t, T, 30000, 9, symbols=np.unique(T)[:4])
    t.close()
