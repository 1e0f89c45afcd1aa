"""The persistent batched kernel (bt_build_batch) against the oracle.

Every document of a batch is built by one CTA of the batched kernel, which
takes documents from a device work queue and runs all levels, pruning and
the counters without the host.  Each tree must be byte-identical to the
oracle's (and so to a standalone bt_build_ex), whatever the batch around it,
and must answer queries like naive counts on its text.
"""
import random

import numpy as np
import pytest
import torch

import oracle
from paper_2512_23314_gb300 import bt, workloads
from tests.test_oracle import _random_text, load_fig1

pytestmark = pytest.mark.gpu


def batch(docs, **kw):
    o, keep = bt.BuildOptions(**kw).to_c()
    hs = bt.bt_build_batch([d.text for d in docs], [len(d.text) for d in docs], [d.sigma for d in docs],
                           [d.tau for d in docs], [d.leaf_len for d in docs], o, nworkers=4)
    del keep
    try:
        return [bt.bt_export(h) for h in hs], hs
    except Exception:
        for h in hs:
            bt.bt_free(h)
        raise


def free_all(hs):
    for h in hs:
        bt.bt_free(h)


def test_batch_kernel_equals_oracle_on_220_documents():
    # Versioned-text documents of 1 KiB - 1 MiB, sigma 4-128, tau 2/4/8,
    # leaf 32: the batched workload's recipe at sizes the oracle builds in
    # seconds.  Every document is checked against the oracle.
    docs = workloads.doc_mix(220, min_len=1 << 10, max_len=1 << 20, seed=0xB7EE0044)
    blobs, hs = batch(docs)
    try:
        for d, blob in zip(docs, blobs):
            assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=True).export()
        # The host-worker arm of the same call gives the same trees.
        wb, wh = batch(docs[::7], batch_workers=True)
        free_all(wh)
        assert wb == blobs[::7]
    finally:
        free_all(hs)


def test_batch_kernel_unpruned_and_weak_modulus():
    # A modulus of 331 makes fingerprint collisions frequent: verification
    # finds them and the exact rescan keeps the tree unchanged.
    docs = workloads.doc_mix(30, min_len=200, max_len=48 << 10, taus=(2, 3, 4), leaf_len=8, seed=91)
    for prune in (False, True):
        for q in (0, 331):
            blobs, hs = batch(docs, prune=prune, modulus=q)
            free_all(hs)
            for d, blob in zip(docs, blobs):
                assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=prune).export(), (prune, q)


def test_batch_kernel_shapes_and_edge_cases():
    # tau not a power of two, odd leaf lengths, texts shorter than a leaf, a
    # single byte, periodic texts, random bytes (no repeats to find).
    rng = np.random.default_rng(5)
    docs = []
    for i in range(60):
        tau = int(rng.choice([2, 3, 5, 7]))
        leaf = int(rng.choice([1, 3, 7, 16, 33]))
        kind = i % 4
        if kind == 0:
            t = _random_text(random.Random(i), int(rng.integers(1, 3000)), int(rng.integers(1, 5)))
        elif kind == 1:
            t = np.frombuffer(b"ab" * int(rng.integers(1, 2000)), np.uint8)
        elif kind == 2:
            t = workloads.random_bytes(int(rng.integers(1, 5000)), 256, i)
        else:
            t = workloads.text_versions(n=int(rng.integers(100, 20000)), base_len=512, sigma=20, seed=i)
        t = np.ascontiguousarray(np.frombuffer(bytes(t), np.uint8))
        docs.append(workloads.Doc(t, 256, tau, leaf))
    docs.append(workloads.Doc(np.frombuffer(b"x", np.uint8).copy(), 1, 2, 4))
    blobs, hs = batch(docs)
    free_all(hs)
    for d, blob in zip(docs, blobs):
        assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=True).export()


def test_batch_kernel_figure1_sizes():
    text, tau, sizes, _ = load_fig1()
    t = np.frombuffer(bytes(text), np.uint8).copy()
    docs = [workloads.Doc(t, 6, tau, 1)] * 3
    for prune in (True, False):
        blobs, hs = batch(docs, prune=prune, level_sizes=tuple(sizes))
        free_all(hs)
        ref = oracle.build(text, tau, 1, prune=prune, level_sizes=sizes).export()
        assert blobs == [ref] * 3


def test_batched_trees_answer_queries():
    docs = workloads.doc_mix(12, min_len=4 << 10, max_len=256 << 10, seed=17)
    _, hs = batch(docs)
    rng = np.random.default_rng(3)
    try:
        for d, h in zip(docs, hs):
            T = d.text
            n = len(T)
            q = 300
            out = torch.empty(q, dtype=torch.int64, device="cuda")
            i = rng.integers(0, n, q)
            bt.bt_query_batch(h, bt.BT_Q_ACCESS, torch.from_numpy(i.astype(np.int64)).cuda(), q, out)
            assert np.array_equal(out.cpu().numpy(), T[i].astype(np.int64))
            syms = np.unique(T)
            c = syms[rng.integers(0, len(syms), q)].astype(np.int64)
            i = rng.integers(0, n + 1, q)
            args = np.stack([c, i], 1).ravel()
            bt.bt_query_batch(h, bt.BT_Q_RANK, torch.from_numpy(args).cuda(), q, out)
            got = out.cpu().numpy()
            for k in range(q):
                assert got[k] == np.count_nonzero(T[:i[k]] == c[k])
            counts = np.bincount(T, minlength=256)
            j = (rng.random(q) * counts[c]).astype(np.int64) + 1
            args = np.stack([c, j], 1).ravel()
            bt.bt_query_batch(h, bt.BT_Q_SELECT, torch.from_numpy(args).cuda(), q, out)
            got = out.cpu().numpy()
            for k in range(q):
                assert got[k] == np.flatnonzero(T == c[k])[j[k] - 1]
    finally:
        free_all(hs)


def test_batch_kernel_trees_freed_in_any_order():
    docs = workloads.doc_mix(40, min_len=1 << 10, max_len=64 << 10, seed=23)
    blobs, hs = batch(docs)
    order = np.random.default_rng(0).permutation(len(hs))
    for k in order[:20]:
        bt.bt_free(hs[k])
    # The trees still held keep their arrays (the shared pool lives on).
    for k in order[20:]:
        assert bt.bt_export(hs[k]) == blobs[k]
    for k in order[20:]:
        bt.bt_free(hs[k])
    torch.cuda.synchronize()


def test_batch_kernel_rejects_bad_alphabet_and_frees():
    docs = workloads.doc_mix(8, min_len=1 << 10, max_len=8 << 10, seed=3)
    sig = [d.sigma for d in docs]
    sig[5] = 1
    o = bt.bt_opts_default()
    with pytest.raises(bt.BTError) as e:
        bt.bt_build_batch([d.text for d in docs], [len(d.text) for d in docs], sig,
                          [d.tau for d in docs], [d.leaf_len for d in docs], o)
    assert e.value.code == bt.BT_EINVAL


def test_batch_kernel_anchored_scan_on_every_level():
    # BT_FLAG_ANCHOR_ALL: every level of 32-byte blocks or more scans by
    # anchors, so short blocks (most without a selected gram) take the 8-byte
    # prefix filter, and the short tail is anchored or prefiltered.  The same
    # trees as the oracle's, also under frequent fingerprint collisions.
    docs = workloads.doc_mix(60, min_len=1 << 10, max_len=256 << 10, seed=0xA7C40001)
    blobs, hs = batch(docs, anchor_all=True)
    free_all(hs)
    for d, blob in zip(docs, blobs):
        assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=True).export()
    weak = workloads.doc_mix(24, min_len=200, max_len=48 << 10, taus=(2, 3, 4), leaf_len=8, seed=93)
    for prune in (False, True):
        blobs, hs = batch(weak, prune=prune, modulus=331, anchor_all=True)
        free_all(hs)
        for d, blob in zip(weak, blobs):
            assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=prune).export(), prune
    rng = np.random.default_rng(11)
    odd = []
    for i in range(24):
        tau = int(rng.choice([2, 3, 5, 7]))
        leaf = int(rng.choice([3, 16, 33]))
        if i % 3 == 0:
            t = np.frombuffer(b"abcd" * int(rng.integers(10, 3000)), np.uint8)
        elif i % 3 == 1:
            t = workloads.random_bytes(int(rng.integers(100, 20000)), 256, i)
        else:
            t = workloads.text_versions(n=int(rng.integers(1000, 60000)), base_len=700, sigma=12, seed=i)
        odd.append(workloads.Doc(np.ascontiguousarray(np.frombuffer(bytes(t), np.uint8)), 256, tau, leaf))
    blobs, hs = batch(odd, anchor_all=True)
    free_all(hs)
    for d, blob in zip(odd, blobs):
        assert blob == oracle.build(d.text, d.tau, d.leaf_len, prune=True).export()
