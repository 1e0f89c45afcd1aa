"""The multithreaded CPU baseline builds the same tree as the oracle
(byte-equal canonical serializations), for any thread count (no GPU needed)."""
import numpy as np
import pytest

import cpu_mt
import oracle
from paper_2512_23314_gb300 import workloads


def _cases(count: int, seed: int):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, 2500))
        sigma = int(rng.choice([1, 2, 4, 26, 256]))
        tau = int(rng.choice([2, 3, 4, 8]))
        leaf = int(rng.choice([1, 2, 3, 8, 16]))
        if rng.integers(2):
            base = rng.integers(0, sigma, int(rng.integers(1, 40)), dtype=np.uint8)
            T = np.resize(base, n)
            k = rng.integers(0, n, max(1, n // 100))
            T[k] = rng.integers(0, sigma, len(k))
        else:
            T = rng.integers(0, sigma, n, dtype=np.uint8)
        yield T.astype(np.uint8), tau, leaf


@pytest.mark.parametrize("prune", [False, True])
def test_cpu_mt_equals_oracle_random(prune):
    for T, tau, leaf in _cases(150, 11 + prune):
        want = oracle.build(T, tau, leaf, prune=prune).export()
        assert cpu_mt.build_tree(T, tau, leaf, prune=prune) == want, (len(T), tau, leaf)


@pytest.mark.parametrize("gen,tau,leaf", [
    (lambda: workloads.text_versions(n=1 << 20, base_len=64 << 10), 4, 32),
    (lambda: workloads.dna_copies(n=1 << 20), 2, 16),
])
def test_cpu_mt_equals_oracle_workloads(gen, tau, leaf):
    T = gen()
    want = oracle.build(T, tau, leaf, prune=True).export()
    for th in (1, 3, 0):
        assert cpu_mt.build_tree(T, tau, leaf, prune=True, nthreads=th) == want


def test_cpu_mt_rejects_bad_arguments():
    with pytest.raises(RuntimeError):
        cpu_mt.build_tree(np.zeros(0, np.uint8), 4, 8)
    with pytest.raises(RuntimeError):
        cpu_mt.build_tree(np.zeros(10, np.uint8), 1, 8)
    with pytest.raises(RuntimeError):
        cpu_mt.build_tree(np.zeros(10, np.uint8), 4, 0)


def test_cpu_mt_seed_independent():
    T = workloads.text_versions(n=100_000, base_len=10_000, sigma=8, seed=3)
    a = cpu_mt.build_tree(T, 4, 8, seed=1)
    assert a == cpu_mt.build_tree(T, 4, 8, seed=12345)
