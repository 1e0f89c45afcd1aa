"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer and byte work, so the bar is bit-exact: the canonical serializations
(level bit vectors, pointers, offsets, leaf text) must be identical, and
query answers must equal naive counts on T.
"""
import random

import numpy as np
import pytest
import torch

import oracle
import oracle.brute as brute
from paper_2512_23314_gb300 import bt, workloads
from tests.helpers import check_leftmost_sampled, check_pointers
from tests.test_oracle import _random_text, load_fig1

pytestmark = pytest.mark.gpu


def gpu_export(text, sigma, tau, leaf, on_device=True, **kw):
    a = np.frombuffer(bytes(text), np.uint8) if isinstance(text, (bytes, bytearray)) else text
    src = torch.from_numpy(np.ascontiguousarray(a)).cuda() if on_device else a
    t = bt.Tree(src, sigma, tau, leaf, bt.BuildOptions(**kw))
    blob = t.export()
    return t, blob


def test_base_matches_oracle():
    for seed in (0, 1, 12345, 2**40 + 7):
        for q in (0, 331, 65521):
            assert bt.bt_fingerprint_base(seed, q) == oracle.base(seed, q)


def test_prefix_fingerprint_kernel():
    for n, seed, q in [(1, 0, 0), (31, 1, 0), (32, 2, 0), (33, 3, 0), (100_000, 4, 0),
                       (1 << 20, 5, 0), (32 * 1024 * 1024 + 77, 6, 0), (5000, 7, 331)]:
        text = workloads.random_bytes(n, 256, seed)
        d = torch.from_numpy(text).cuda()
        m = n // 32 + 1
        out = torch.empty(m, dtype=torch.int64, device="cuda")
        bt.bt_prefix_fingerprints(d, n, seed, q, 32, out)
        got = out.cpu().numpy().view(np.uint64)
        B = oracle.base(seed, q)
        js = sorted(set([0, 1, m - 1, m // 2] + list(np.random.default_rng(seed).integers(0, m, 20))))
        for j in js:
            if 32 * j > n:
                continue
            assert int(got[j]) == oracle.fingerprint(text, 0, 32 * j, B, q), (n, j)


@pytest.mark.parametrize("variant", ["pruned", "unpruned"])
def test_figure1(variant):
    text, tau, sizes, _ = load_fig1()
    ref = oracle.build(text, tau, 1, prune=variant == "pruned", level_sizes=sizes).export()
    _, blob = gpu_export(text, 6, tau, 1, prune=variant == "pruned", level_sizes=tuple(sizes))
    assert blob == ref


def test_parity_random_tiny():
    rng = random.Random(31337)
    for it in range(400):
        n = rng.randrange(1, 300)
        text = _random_text(rng, n, rng.choice([1, 2, 3, 4, 26]))
        tau, leaf = rng.choice([2, 3, 4, 5, 8]), rng.choice([1, 2, 3, 4, 8, 16])
        prune = rng.random() < 0.6
        root = rng.choice([0, 0, 2, 3])
        ref = oracle.build(text, tau, leaf, prune=prune, root_arity=root).export()
        _, blob = gpu_export(text, 256, tau, leaf, on_device=bool(it % 2), prune=prune,
                             root_arity=root, seed=rng.randrange(1 << 30))
        assert blob == ref, (text, tau, leaf, prune, root)


def test_parity_explicit_sizes():
    rng = random.Random(4242)
    for _ in range(100):
        L = rng.randrange(1, 5)
        sizes = [rng.randrange(1, 4)]
        for _ in range(L - 1):
            sizes.insert(0, sizes[0] * rng.randrange(2, 5))
        n = rng.randrange(1, sizes[0] * rng.randrange(1, 6) + 1)
        text = _random_text(rng, n, rng.choice([2, 3, 4]))
        prune = rng.random() < 0.5
        ref = brute.serialize(brute.build(text, 3, 1, prune=prune, explicit=sizes))
        _, blob = gpu_export(text, 8, 3, 1, prune=prune, level_sizes=tuple(sizes))
        assert blob == ref, (text, sizes, prune)


@pytest.mark.parametrize("n,tau,leaf,kind", [
    (4096, 2, 16, "dna"), (4096 + 1, 2, 16, "dna"), (65536 - 7, 4, 32, "text"),
    (100_003, 4, 8, "text"), (262_144, 8, 4, "dna"), (300_001, 3, 5, "text"),
    (1 << 20, 2, 16, "dna"), (2_000_000 + 13, 4, 32, "text"), (777_777, 2, 64, "unary"),
    (500_000, 4, 32, "random"),
])
def test_parity_sizes_and_tails(n, tau, leaf, kind):
    if kind == "dna":
        text = workloads.dna_copies(n=n, seed_len=max(256, n // 16), seed=n)
    elif kind == "text":
        text = workloads.text_versions(n=n, base_len=max(1024, n // 16), sigma=40, seed=n)
    elif kind == "unary":
        text = np.full(n, ord("a"), np.uint8)
    else:
        text = workloads.random_bytes(n, 256, n)
    for prune in (True, False):
        ref = oracle.build(text, tau, leaf, prune=prune).export()
        t, blob = gpu_export(text, 256, tau, leaf, prune=prune)
        assert blob == ref
        st = t.stats()
        ost = oracle.build(text, tau, leaf, prune=False).stats()
        assert [s["cov"] for s in st] == [s["cov"] for s in ost]
        assert [s["nblocks"] for s in st] == [s["nblocks"] for s in ost]


def test_weak_modulus_forces_collisions():
    rng = random.Random(99)
    total = 0
    for it in range(60):
        n = rng.randrange(50, 3000)
        text = _random_text(rng, n, rng.choice([2, 3]))
        tau, leaf = rng.choice([2, 3, 4]), rng.choice([1, 2, 4])
        ref = oracle.build(text, tau, leaf, prune=bool(it % 2)).export()
        t, blob = gpu_export(text, 8, tau, leaf, prune=bool(it % 2), modulus=331, seed=it)
        assert blob == ref
        total += sum(s["collisions"] for s in t.stats())
    assert total > 0


def test_host_and_device_inputs_agree():
    text = workloads.text_versions(n=300_000, base_len=30_000, sigma=20, seed=5)
    _, a = gpu_export(text, 20, 4, 16, on_device=False)
    _, b = gpu_export(text, 20, 4, 16, on_device=True)
    assert a == b


def test_invalid_arguments():
    for args in [(b"abc", 0, 2, 4), (b"abc", 3, 1, 4), (b"abc", 3, 2, 0), (b"abcd", 3, 2, 1)]:
        with pytest.raises(bt.BTError) as e:
            bt.Tree(args[0], *args[1:])
        assert e.value.code == bt.BT_EINVAL


def _naive_queries(T, kinds, a0, a1):
    out = np.empty(len(kinds), dtype=np.uint64)
    for c in np.unique(a0[kinds != bt.BT_Q_ACCESS]):
        pos = np.flatnonzero(T == c)
        sel = (kinds == bt.BT_Q_RANK) & (a0 == c)
        out[sel] = np.searchsorted(pos, a1[sel], side="left")
        sel = (kinds == bt.BT_Q_SELECT) & (a0 == c)
        out[sel] = pos[a1[sel] - 1]
    sel = kinds == bt.BT_Q_ACCESS
    out[sel] = T[a0[sel]]
    return out


def run_queries(t, T, nq, seed, symbols=None):
    rng = np.random.default_rng(seed)
    n = len(T)
    syms = np.unique(T) if symbols is None else np.asarray(symbols, np.uint8)
    counts = {int(c): int((T == c).sum()) for c in syms}
    kinds = rng.integers(0, 3, nq)
    a0 = np.zeros(nq, np.int64)
    a1 = np.zeros(nq, np.int64)
    acc = kinds == bt.BT_Q_ACCESS
    a0[acc] = rng.integers(0, n, acc.sum())
    cs = rng.choice(syms, nq)
    a0[~acc] = cs[~acc]
    rk = kinds == bt.BT_Q_RANK
    a1[rk] = rng.integers(0, n + 1, rk.sum())
    sl = kinds == bt.BT_Q_SELECT
    a1[sl] = [rng.integers(1, counts[int(c)] + 1) for c in cs[sl]]
    want = _naive_queries(T, kinds, a0, a1)
    for kind in (bt.BT_Q_ACCESS, bt.BT_Q_RANK, bt.BT_Q_SELECT):
        sel = kinds == kind
        m = int(sel.sum())
        if kind == bt.BT_Q_ACCESS:
            args = torch.from_numpy(a0[sel].copy()).cuda()
        else:
            args = torch.from_numpy(np.stack([a0[sel], a1[sel]], 1).reshape(-1).copy()).cuda()
        out = torch.empty(m, dtype=torch.int64, device="cuda")
        t.query_batch(kind, args, out)
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want[sel]), kind


def test_queries_against_naive_counts():
    for n, tau, leaf, seed in [(5000, 2, 4, 1), (200_001, 4, 16, 2), (1 << 20, 2, 16, 3)]:
        T = workloads.text_versions(n=n, base_len=max(512, n // 20), sigma=30, seed=seed)
        for prune in (True, False):
            t, _ = gpu_export(T, 30, tau, leaf, prune=prune)
            run_queries(t, T, 20000, seed)
    t, _ = gpu_export(b"abcabcabd", 4, 2, 1)
    assert t.access(8) == ord("d") and t.rank(ord("c"), 9) == 2 and t.select(ord("c"), 2) == 5
    assert t.rank(ord("z"), 9) == 0
    for bad in (lambda: t.access(9), lambda: t.rank(97, 10), lambda: t.select(97, 0),
                lambda: t.select(97, 4), lambda: t.select(ord("z"), 1)):
        with pytest.raises(bt.BTError) as e:
            bad()
        assert e.value.code == bt.BT_ERANGE


def test_config_dna_copies_1mib_full():
    """1 MiB DNA copies, tau=2, leaf 16: bit-exact tree, 10^5 queries."""
    T = workloads.dna_copies()
    ref = oracle.build(T, 2, 16, prune=True)
    t, blob = gpu_export(T, 4, 2, 16)
    assert blob == ref.export()
    assert t.stats()[0]["b"] == 1 << 19 and len(t.stats()) == 16
    run_queries(t, T, 100_000, 11)


def _runs_text(n, seed, alphabet=b"ab", max_run=200):
    rng = np.random.default_rng(seed)
    out = bytearray()
    while len(out) < n:
        out += bytes([alphabet[rng.integers(len(alphabet))]]) * int(rng.integers(1, max_run))
    return np.frombuffer(bytes(out[:n]), np.uint8)


def _gram_selected(gram: bytes) -> bool:
    """Whether the anchored scan selects this 16-gram at density 1/8 (its
    polynomial hash times an odd constant, mod 2^32, below 2^29)."""
    h = 0
    for c in gram:
        h = (h * 0x01000193 + c) & 0xFFFFFFFF
    return ((h * 0x9E3779B1) & 0xFFFFFFFF) < (1 << 29)


def _far_anchor_text(n, seed):
    """Runs of one byte (whose 16-gram is not selected) of 70-150 bytes, each
    followed by one of three fixed strings: blocks that start in a run have
    their first selected gram beyond the 64 offsets of the anchor mask, and
    blocks with the same string after runs of different lengths anchor on the
    same gram at different far offsets."""
    rng = np.random.default_rng(seed)
    run = next(c for c in b"zyxwvutsrq" if not _gram_selected(bytes([c]) * 16))
    tails = [bytes(rng.integers(97, 123, 200, dtype=np.uint8)) for _ in range(3)]
    out = bytearray()
    while len(out) < n:
        out += bytes([run]) * int(rng.integers(70, 151)) + tails[int(rng.integers(3))]
    return np.frombuffer(bytes(out[:n]), np.uint8)


@pytest.mark.parametrize("scan", ["anchored", "dense", "tiny_queue", "gram_list", "two_phase"])
def test_anchored_and_dense_scans(scan):
    """Both window-scan strategies give the oracle's tree, including texts whose
    keys have no anchor (long runs) and short tails of every length; so does
    the anchored scan whose candidate queue overflows at every level, and the
    one that reads the selected-gram list, and the one that tests the windows of
    every level in two phases (the second against bounds the first tightened)."""
    kw = {"dense_scan": scan == "dense", "tiny_queue": scan == "tiny_queue",
          "gram_list": scan == "gram_list", "two_phase": scan == "two_phase"}
    cases = [
        (_runs_text(50_000, 1), 2, 8), (_runs_text(120_001, 2, b"abc", 500), 4, 16),
        (_runs_text(30_000, 3, b"a", 2), 2, 4), (np.full(100_003, 65, np.uint8), 4, 32),
        (workloads.dna_genome(n=600_000 + 37, genome_len=40_000, nrun_rate=1e-3, seed=9), 4, 64),
        (workloads.text_versions(n=333_333, base_len=20_000, sigma=96, seed=2), 4, 32),
        (workloads.text_versions(n=99_999, base_len=4096, sigma=4, seed=3), 2, 1),
        (workloads.random_bytes(70_001, 3, 4), 3, 2),
        (_far_anchor_text(200_000, 5), 2, 128), (_far_anchor_text(150_001, 6), 4, 96),
    ]
    for T, tau, leaf in cases:
        for prune in (True, False):
            ref = oracle.build(T, tau, leaf, prune=prune).export()
            _, blob = gpu_export(T, 256, tau, leaf, prune=prune, **kw)
            assert blob == ref, (len(T), tau, leaf, prune)
    rng = random.Random(7)
    for _ in range(150):
        n = rng.randrange(1, 3000)
        text = _random_text(rng, n, rng.choice([1, 2, 3, 26]))
        tau, leaf = rng.choice([2, 3, 4]), rng.choice([1, 3, 8, 40, 100])
        ref = oracle.build(text, tau, leaf).export()
        _, blob = gpu_export(text, 256, tau, leaf, **kw)
        assert blob == ref, (text, tau, leaf)


@pytest.mark.parametrize("max_rounds", [1, 2, 3, 7, 0])
def test_prune_round_bound(max_rounds):
    """Pruning decides the same blocks whatever the bound on the parallel
    frontier rounds (section 3.1's right-to-left rule): the rounds that do not
    finish leave the rest to the sequential finish; levels of more than 16 Ki
    blocks start with multi-CTA rounds and hand narrow frontiers to one CTA."""
    text = workloads.text_versions(n=4 << 20, base_len=64 << 10, sigma=26, seed=21)
    ref = _prune_ref(text)
    _, blob = gpu_export(text, 26, 4, 8, prune=True, max_rounds=max_rounds)
    assert blob == ref


_PRUNE_REF = {}


def _prune_ref(text):
    key = hash(text.tobytes())
    if key not in _PRUNE_REF:
        _PRUNE_REF[key] = oracle.build(text, 4, 8, prune=True).export()
    return _PRUNE_REF[key]


def test_mulmod_bench_values():
    """The integer-pipe microbenchmark runs the fingerprint multiply: every
    chain ends at a0 * B^iters mod 2^61 - 1 (B the base of the seed)."""
    blocks, iters, seed = 2, 100, 5
    out = torch.empty(blocks * 256, dtype=torch.int64, device="cuda")
    n = bt.bt_mulmod_bench(blocks, iters, out, None, seed=seed)
    torch.cuda.synchronize()
    assert n == blocks * 256 * iters * 8
    q = (1 << 61) - 1
    bi = pow(oracle.base(seed), iters, q)
    vals = out.cpu().numpy().view(np.uint64)
    for t in (0, 1, 255, 256, 511):
        x = 0
        for u in range(8):
            x ^= ((t * 8 + u) % (q - 1) + 1) * bi % q
        assert int(vals[t]) == x
