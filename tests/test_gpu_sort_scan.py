"""The sort-based level pass (BT_FLAG_SORT_SCAN) against the oracle.

The leftmost window of every block and pair comes from radix-sorted
(fingerprint, position) tuples of all windows of the level instead of table
probes.  The tree must be byte-identical to the oracle's: on seeded tiny
texts (every shape of level), with explicit level sizes (Figure 1), with a
weak modulus that forces fingerprint collisions (verification and the exact
rescan still decide), and against the default path on larger texts.
"""
import random

import numpy as np
import pytest
import torch

import oracle
from paper_2512_23314_gb300 import bt, workloads
from tests.test_gpu_parity import gpu_export
from tests.test_oracle import _random_text, load_fig1

pytestmark = pytest.mark.gpu


def test_sort_scan_random_tiny():
    rng = random.Random(777)
    for it in range(200):
        n = rng.randrange(1, 400)
        text = _random_text(rng, n, rng.choice([1, 2, 3, 4, 26]))
        tau, leaf = rng.choice([2, 3, 4, 5, 8]), rng.choice([1, 2, 3, 4, 8, 16])
        prune = rng.random() < 0.6
        ref = oracle.build(text, tau, leaf, prune=prune).export()
        _, blob = gpu_export(text, 256, tau, leaf, prune=prune, sort_scan=True)
        assert blob == ref, (text, tau, leaf, prune)


def test_sort_scan_figure1_and_weak_modulus():
    text, tau, sizes, _ = load_fig1()
    for prune in (True, False):
        ref = oracle.build(text, tau, 1, prune=prune, level_sizes=sizes).export()
        _, blob = gpu_export(text, 6, tau, 1, prune=prune, level_sizes=tuple(sizes), sort_scan=True)
        assert blob == ref
    rng = random.Random(5)
    total = 0
    for it in range(30):
        text = _random_text(rng, rng.randrange(100, 3000), rng.choice([2, 3]))
        tau, leaf = rng.choice([2, 4]), rng.choice([1, 2, 4])
        ref = oracle.build(text, tau, leaf, prune=bool(it % 2)).export()
        t, blob = gpu_export(text, 8, tau, leaf, prune=bool(it % 2), modulus=331, seed=it, sort_scan=True)
        assert blob == ref
        total += sum(s["collisions"] for s in t.stats())
    assert total > 0


@pytest.mark.parametrize("n,tau,leaf", [(1 << 20, 2, 16), (5_000_003, 4, 32), (16 << 20, 4, 32)])
def test_sort_scan_equals_default_and_oracle(n, tau, leaf):
    T = workloads.text_versions(n=n, base_len=max(4096, n // 16), sigma=40, seed=n)
    d = torch.from_numpy(T).cuda()
    a = bt.Tree(d, 40, tau, leaf).export()
    b = bt.Tree(d, 40, tau, leaf, bt.BuildOptions(sort_scan=True)).export()
    assert a == b
    if n <= 1 << 20:
        assert b == oracle.build(T, tau, leaf, prune=True).export()


# Domain decomposition (section 4.2): the windows in K parts, each keeping
# only the first window of each key fingerprint; the same tree for every K.

def test_partitions_random_tiny():
    rng = random.Random(4242)
    for it in range(160):
        n = rng.randrange(1, 500)
        text = _random_text(rng, n, rng.choice([1, 2, 3, 4, 26]))
        tau, leaf = rng.choice([2, 3, 4, 5, 8]), rng.choice([1, 2, 3, 4, 8, 16])
        prune = rng.random() < 0.6
        k = rng.choice([2, 3, 7, 64, 1000])
        ref = oracle.build(text, tau, leaf, prune=prune).export()
        _, blob = gpu_export(text, 256, tau, leaf, prune=prune, sort_scan=True, partitions=k)
        assert blob == ref, (text, tau, leaf, prune, k)


def test_partitions_figure1_and_weak_modulus():
    text, tau, sizes, _ = load_fig1()
    for k in (2, 5):
        ref = oracle.build(text, tau, 1, prune=True, level_sizes=sizes).export()
        _, blob = gpu_export(text, 6, tau, 1, prune=True, level_sizes=tuple(sizes), sort_scan=True, partitions=k)
        assert blob == ref
    rng = random.Random(15)
    total = 0
    for it in range(20):
        text = _random_text(rng, rng.randrange(100, 3000), rng.choice([2, 3]))
        tau, leaf = rng.choice([2, 4]), rng.choice([1, 2, 4])
        ref = oracle.build(text, tau, leaf, prune=bool(it % 2)).export()
        t, blob = gpu_export(text, 8, tau, leaf, prune=bool(it % 2), modulus=331, seed=it, sort_scan=True,
                             partitions=rng.choice([2, 9]))
        assert blob == ref
        total += sum(s["collisions"] for s in t.stats())
    assert total > 0


def test_partitions_oracle_1MiB_and_default_16MiB():
    T = workloads.dna_copies(n=1 << 20, seed=0xB7EE0001)
    ref = oracle.build(T, 2, 16, prune=True).export()
    d = torch.from_numpy(T).cuda()
    for k in (4, 33):
        assert bt.Tree(d, 4, 2, 16, bt.BuildOptions(sort_scan=True, partitions=k)).export() == ref
    n = 16 << 20
    T = workloads.text_versions(n=n, base_len=n // 16, sigma=96, seed=0xB7EE0002)
    d = torch.from_numpy(T).cuda()
    a = bt.Tree(d, 96, 4, 32).export()
    assert bt.Tree(d, 96, 4, 32, bt.BuildOptions(sort_scan=True, partitions=16)).export() == a


def test_partitions_bound_working_memory():
    # The peak of the stream-ordered pool during a build: the one-part sort
    # holds about 24 bytes per window of a level, 16 parts a sixteenth of that
    # plus the kept tuples.
    n = 16 << 20
    T = workloads.text_versions(n=n, base_len=n // 16, sigma=96, seed=0xB7EE0002)
    d = torch.from_numpy(T).cuda()
    torch.cuda.synchronize()
    peaks = {}
    for k in (1, 16):
        bt.bt_device_pool_peak(reset=True)
        t = bt.Tree(d, 96, 4, 32, bt.BuildOptions(sort_scan=True, partitions=k))
        torch.cuda.synchronize()
        peaks[k] = bt.bt_device_pool_peak()
        del t
        torch.cuda.synchronize()
    assert peaks[16] < 0.6 * peaks[1], peaks
