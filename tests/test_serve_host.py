"""Host logic of the serving loop (no GPU): admission under the HBM budget,
eviction of the oldest resident trees, and the switch from the admission
estimate to a built tree's real device bytes.  The library calls it makes
(freeing a tree, reading its device bytes) are replaced by fakes."""
import threading
import time

import pytest

from paper_2512_23314_gb300 import serve


@pytest.fixture
def fake_lib(monkeypatch):
    freed = []
    monkeypatch.setattr(serve.bt, "bt_free", lambda h: freed.append(h))
    monkeypatch.setattr(serve.bt, "bt_device_bytes", lambda h: 10)
    return freed


def test_admission_evicts_oldest_and_charges_real_bytes(fake_lib):
    s = serve.Server(hbm_budget=100, lanes=1)
    s._admit(40)
    s._retire(0, "h0", 40)  # the estimate 40 becomes the real 10
    s._admit(40)
    s._retire(1, "h1", 40)
    assert s._charged == 20 and s._evictions == 0
    s._admit(85)  # 20 + 85 > 100: the oldest tree goes, 10 + 85 fits
    assert fake_lib == ["h0"] and s._evictions == 1 and s._charged == 95
    s._retire(2, "h2", 85)
    assert s._charged == 20
    assert list(s._resident) == [1, 2]


def test_document_larger_than_budget_runs_alone(fake_lib):
    s = serve.Server(hbm_budget=100, lanes=1)
    s._admit(40)
    s._retire(0, "h0", 40)
    s._admit(500)  # evicts everything resident, then runs alone over the budget
    assert fake_lib == ["h0"] and s._charged == 500 and s._inflight == 1


def test_admission_waits_for_builds_in_flight(fake_lib):
    s = serve.Server(hbm_budget=100, lanes=2)
    s._admit(80)  # in flight, nothing resident to evict
    done = threading.Event()

    def second():
        s._admit(50)
        done.set()

    th = threading.Thread(target=second)
    th.start()
    time.sleep(0.2)
    assert not done.is_set()  # 80 + 50 > 100 with a build in flight: it waits
    s._retire(0, "h0", 80)  # the first build is charged its real 10 bytes
    th.join(timeout=5)
    assert done.is_set() and s._charged == 60 and s._max_inflight == 1


class _FakeStream:
    cuda_stream = 0


def _arrivals(k):
    from paper_2512_23314_gb300.workloads import Arrival, Doc
    import numpy as np
    return [Arrival(0.0, Doc(np.zeros(64 + i, np.uint8), 4, 2, 16)) for i in range(k)]


def test_worker_error_is_raised_and_releases_its_charge(fake_lib, monkeypatch):
    """A build that fails in a worker thread ends run() with that error (no
    hang), and the failed document's admission charge is given back."""
    monkeypatch.setattr(serve.torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(serve.torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(serve.bt, "bt_opts_default", lambda: None)
    built = []

    def fake_build(text, n, sigma, tau, leaf, opts, stream):
        if n == 66:
            raise serve.bt.BTError(serve.bt.BT_EINVAL, "bt_build_ex")
        built.append(n)
        return f"h{n}"

    monkeypatch.setattr(serve.bt, "bt_build_ex", fake_build)
    monkeypatch.setattr(serve.Server, "_queries", lambda self, h, n, rng, stream, keep=0: (0.0, None))
    # small_max=0: every document is built alone with bt_build_ex.
    s = serve.Server(hbm_budget=1 << 40, lanes=3, small_max=0)
    t0 = time.perf_counter()
    with pytest.raises(serve.bt.BTError):
        s.run(_arrivals(6))
    assert time.perf_counter() - t0 < 10
    assert sorted(built) == [64, 65, 67, 68, 69]
    assert s._inflight == 0
    # Only the five built trees stay charged (10 bytes each from the fake).
    assert s._charged == 50 and len(s._resident) == 5


def test_every_worker_failing_still_returns(fake_lib, monkeypatch):
    monkeypatch.setattr(serve.torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(serve.torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(serve.bt, "bt_opts_default", lambda: None)

    def fail(*a):
        raise RuntimeError("device lost")

    monkeypatch.setattr(serve.bt, "bt_build_ex", fail)
    s = serve.Server(hbm_budget=1 << 40, lanes=2, small_max=0)
    with pytest.raises(RuntimeError, match="device lost"):
        s.run(_arrivals(5))
    assert s._inflight == 0 and s._charged == 0


def test_small_documents_go_out_in_micro_batches(fake_lib, monkeypatch):
    """Small documents waiting together are built by one bt_build_batch call
    on 1/lanes of the SMs; a failing micro-batch releases every charge."""
    monkeypatch.setattr(serve.torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(serve.torch.cuda, "synchronize", lambda *a: None)
    calls = []

    def fake_batch(texts, ns, sigmas, taus, leafs, opts, nworkers=0):
        calls.append((list(ns), opts.batch_ctas))
        return [f"b{n}" for n in ns]

    monkeypatch.setattr(serve.bt, "bt_build_batch", fake_batch)
    monkeypatch.setattr(serve.Server, "_queries", lambda self, h, n, rng, stream, keep=0: (0.0, None))
    s = serve.Server(hbm_budget=1 << 40, lanes=2, small_max=1 << 20, sm_count=152)
    rep = s.run(_arrivals(40))  # all arrive at t = 0
    assert rep.docs == 40 and rep.batches == len(calls) >= 1
    assert sorted(n for ns, _ in calls for n in ns) == list(range(64, 104))
    assert all(ctas == 76 for _, ctas in calls)
    assert rep.mean_batch_docs > 1 and s._inflight == 0 and len(s._resident) == 40

    def failing(*a, **k):
        raise RuntimeError("batch failed")

    monkeypatch.setattr(serve.bt, "bt_build_batch", failing)
    s2 = serve.Server(hbm_budget=1 << 40, lanes=2, sm_count=152)
    with pytest.raises(RuntimeError, match="batch failed"):
        s2.run(_arrivals(10))
    assert s2._inflight == 0 and s2._charged == 0


def test_lane_that_cannot_start_ends_run(fake_lib, monkeypatch):
    """A lane whose stream cannot be made is recorded like a failed unit:
    run() raises that error instead of waiting for documents nobody serves."""
    def no_stream():
        raise RuntimeError("no stream")

    monkeypatch.setattr(serve.torch.cuda, "Stream", no_stream)
    monkeypatch.setattr(serve.torch.cuda, "synchronize", lambda *a: None)
    s = serve.Server(hbm_budget=1 << 40, lanes=2, small_max=0)
    t0 = time.perf_counter()
    with pytest.raises(RuntimeError, match="no stream"):
        s.run(_arrivals(4))
    assert time.perf_counter() - t0 < 10


def test_small_documents_behind_a_large_one_share_a_batch(fake_lib, monkeypatch):
    """Small documents waiting behind large ones are gathered into one
    micro-batch; the large ones keep their places and are built alone."""
    monkeypatch.setattr(serve.torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(serve.torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(serve.bt, "bt_opts_default", lambda: serve.bt.bt_opts())
    batches, alone = [], []

    def fake_batch(texts, ns, sigmas, taus, leafs, opts, nworkers=0):
        batches.append(list(ns))
        return [f"b{n}" for n in ns]

    def fake_build(text, n, sigma, tau, leaf, opts, stream):
        alone.append(n)
        return f"h{n}"

    monkeypatch.setattr(serve.bt, "bt_build_batch", fake_batch)
    monkeypatch.setattr(serve.bt, "bt_build_ex", fake_build)
    monkeypatch.setattr(serve.Server, "_queries", lambda self, h, n, rng, stream, keep=0: (0.0, None))
    from paper_2512_23314_gb300.workloads import Arrival, Doc
    import numpy as np
    sizes = [64, 2000, 65, 66, 2001, 67, 68]  # two large (> small_max = 1000) among small ones
    arr = [Arrival(0.0, Doc(np.zeros(k, np.uint8), 4, 2, 16)) for k in sizes]
    s = serve.Server(hbm_budget=1 << 40, lanes=1, small_max=1000, sm_count=152)
    rep = s.run(arr)
    assert rep.docs == len(sizes)
    assert sorted(alone) == [2000, 2001]
    assert sorted(n for b in batches for n in b) == [64, 65, 66, 67, 68]
    assert len(batches) <= 2
