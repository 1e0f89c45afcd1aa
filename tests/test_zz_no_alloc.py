"""The allocation-free prefix-fingerprint entry point agrees with the regular one.

bt_prefix_fingerprints_noalloc serves callers that cannot allocate device
memory.  For example, a runtime that owns all device memory through its own
allocator and forbids the libraries it loads to call cudaMalloc, or a code
path that must not risk an allocation's implicit synchronisation or failure.
Its scratch is a fixed array in device memory, shared by every call.  This
file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2512_23314_gb300 import bt, workloads

pytestmark = pytest.mark.gpu


def _both(text_dev, n, seed, modulus):
    m = n // 32 + 1
    ref = torch.empty(m, dtype=torch.int64, device="cuda")
    out = torch.full((m,), -1, dtype=torch.int64, device="cuda")
    bt.bt_prefix_fingerprints(text_dev, n, seed, modulus, 32, ref)
    bt.bt_prefix_fingerprints_noalloc(text_dev, n, seed, modulus, 32, out)
    torch.cuda.synchronize()
    return ref, out


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    # Two calls in a row (different sizes, so the shared scratch holds the
    # previous call's contents when the second one starts), then two with
    # the test modulus.  Integer results: they must be identical.
    for n, seed, modulus in [(3_000_017, 11, 0), (100_000, 12, 0), (50_001, 13, 331), (4096, 14, 331)]:
        text = workloads.random_bytes(n, 256, seed)
        d = torch.from_numpy(text).cuda()
        ref, out = _both(d, n, seed, modulus)
        assert torch.equal(ref, out), (n, seed, modulus)


def test_noalloc_rejects_texts_beyond_its_scratch():
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(bt.BTError) as e:
        # The size check runs on the host before any kernel: nothing is read.
        bt.bt_prefix_fingerprints_noalloc(d, (1 << 31) + 1, 0, 0, 32, out)
    assert e.value.code == bt.BT_ERANGE
