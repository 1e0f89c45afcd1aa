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
    s = serve.Server(hbm_budget=100, nworkers=1)
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
    s = serve.Server(hbm_budget=100, nworkers=1)
    s._admit(40)
    s._retire(0, "h0", 40)
    s._admit(500)  # evicts everything resident, then runs alone over the budget
    assert fake_lib == ["h0"] and s._charged == 500 and s._inflight == 1


def test_admission_waits_for_builds_in_flight(fake_lib):
    s = serve.Server(hbm_budget=100, nworkers=2)
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
