"""Builds that cannot get device memory fail cleanly.

A test hook caps the size of any single device allocation a build makes;
above the cap the allocation fails as if the device were out of memory.  The
build must return BT_ENOMEM, hand back every byte it took from the device's
stream-ordered pool, and leave the library usable: the next build, without
the cap, gives the same tree as before.
"""
import pytest
import torch

from paper_2512_23314_gb300 import bt, workloads

pytestmark = pytest.mark.gpu


def _capped(limit, fn):
    bt.bt_test_alloc_limit(limit)
    try:
        with pytest.raises(bt.BTError) as e:
            fn()
        return e.value.code
    finally:
        bt.bt_test_alloc_limit(0)


def test_single_build_fails_with_enomem_and_frees_everything():
    T = workloads.text_versions(n=4 << 20, base_len=256 << 10, seed=3)
    d = torch.from_numpy(T).cuda()
    ref = bt.Tree(d, 96, 4, 32).export()
    torch.cuda.synchronize()
    used0 = bt.bt_device_pool_used()
    # 1 MiB stops the stride-32 prefix values, 16 MiB the prefix array of
    # every position (32 MiB for this text); host input also needs a copy.
    for limit in (1 << 20, 16 << 20):
        for src in (d, T):
            assert _capped(limit, lambda: bt.Tree(src, 96, 4, 32)) == bt.BT_ENOMEM
            torch.cuda.synchronize()
            assert bt.bt_device_pool_used() == used0
    assert bt.Tree(d, 96, 4, 32).export() == ref


def test_batch_build_fails_with_enomem_and_frees_everything():
    docs = workloads.doc_mix(24, min_len=16 << 10, max_len=512 << 10, seed=41)
    args = ([x.text for x in docs], [len(x.text) for x in docs], [x.sigma for x in docs],
            [x.tau for x in docs], [x.leaf_len for x in docs])
    ref = bt.bt_build_batch(*args)
    ref_blobs = [bt.bt_export(h) for h in ref]
    for h in ref:
        bt.bt_free(h)
    torch.cuda.synchronize()
    used0 = bt.bt_device_pool_used()
    for workers in (False, True):
        o, _ = bt.BuildOptions(batch_workers=workers).to_c()
        assert _capped(256 << 10, lambda: bt.bt_build_batch(*args, o)) == bt.BT_ENOMEM
        torch.cuda.synchronize()
        assert bt.bt_device_pool_used() == used0
    hs = bt.bt_build_batch(*args)
    assert [bt.bt_export(h) for h in hs] == ref_blobs
    for h in hs:
        bt.bt_free(h)
