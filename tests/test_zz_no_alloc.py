"""The allocation-free prefix-fingerprint entry point agrees with the regular one.

bt_prefix_fingerprints_noalloc serves callers that cannot allocate device
memory.  For example, a runtime that owns all device memory through its own
allocator and forbids the libraries it loads to call cudaMalloc, or a code
path that must not risk an allocation's implicit synchronisation or failure.
Its scratch is a fixed array in device memory, shared by every call.  This
file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2512_23314_gb300 import bt, workloads


def _both(text_dev, n, seed, modulus):
    m = n // 32 + 1
    ref = torch.empty(m, dtype=torch.int64, device="cuda")
    out = torch.full((m,), -1, dtype=torch.int64, device="cuda")
    bt.bt_prefix_fingerprints(text_dev, n, seed, modulus, 32, ref)
    bt.bt_prefix_fingerprints_noalloc(text_dev, n, seed, modulus, 32, out)
    torch.cuda.synchronize()
    return ref, out


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    # Two calls in a row (different sizes, so the shared scratch holds the
    # previous call's contents when the second one starts), then two with
    # the test modulus.  Integer results: they must be identical.
    for n, seed, modulus in [(3_000_017, 11, 0), (100_000, 12, 0), (50_001, 13, 331), (4096, 14, 331)]:
        text = workloads.random_bytes(n, 256, seed)
        d = torch.from_numpy(text).cuda()
        ref, out = _both(d, n, seed, modulus)
        assert torch.equal(ref, out), (n, seed, modulus)


@pytest.mark.gpu
def test_noalloc_multi_tile_aggregates_against_the_oracle():
    # 32 MiB + 77 bytes: 1 Mi + 2 chunks of 32 bytes, so 1025 per-CTA
    # aggregates and the single-CTA aggregate scan runs a second tile.  Two
    # calls in a row, compared with the allocating entry point and, at
    # sampled strides, with the oracle's Horner fingerprint of the prefix.
    n = (32 << 20) + 77
    text = workloads.random_bytes(n, 256, 21)
    d = torch.from_numpy(text).cuda()
    for seed in (5, 6):
        ref, out = _both(d, n, seed, 0)
        assert torch.equal(ref, out)
        got = out.cpu().numpy().view(np.uint64)
        B = oracle.base(seed)
        rng = np.random.default_rng(seed)
        js = np.concatenate([[0, 1, 1023, 1024, 1025, 32767, 32768, n // 32],
                             rng.integers(0, n // 32 + 1, 40)])
        for j in js:
            j = int(j)
            assert int(got[j]) == oracle.fingerprint(text, 0, 32 * j, B), j


@pytest.mark.gpu
def test_noalloc_rejects_texts_beyond_its_scratch():
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(bt.BTError) as e:
        # The size check runs on the host before any kernel: nothing is read.
        bt.bt_prefix_fingerprints_noalloc(d, (1 << 31) + 1, 0, 0, 32, out)
    assert e.value.code == bt.BT_ERANGE


def _raw_call(n):
    lib = bt.lib()
    f = lib.bt_prefix_fingerprints_noalloc
    return f(ctypes.c_void_p(0), ctypes.c_uint64(n), ctypes.c_uint64(0), ctypes.c_uint64(0),
             ctypes.c_uint32(32), ctypes.c_void_p(0), ctypes.c_void_p(0))


def test_noalloc_size_limit_boundary_on_the_host():
    # No GPU needed: the size check comes first, so 2^31 + 1 bytes is refused
    # as out of range, while 2^31 bytes passes it and only then fails on the
    # null pointers (nothing is launched in either case).
    assert _raw_call((1 << 31) + 1) == bt.BT_ERANGE
    assert _raw_call(1 << 31) == bt.BT_EINVAL
