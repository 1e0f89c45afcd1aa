"""Serving loop: continuous batching of block-tree builds under an HBM budget.

Documents arrive over time.  `lanes` host threads serve them; each lane owns
a CUDA stream and repeatedly takes work from the arrival queue:

* small documents (at most `small_max` bytes): every one waiting, in arrival
  order, up to `max_batch_docs` and as far as the HBM budget admits them, as
  one micro-batch built by bt_build_batch -- the persistent batched kernel,
  on 1/lanes of the SMs, so the micro-batches of different lanes run side by
  side on the device;
* a large document: alone, with bt_build_ex on the lane's stream (the whole
  GPU's level kernels for one text).

A document that arrives while others are on the GPU is taken by the next
lane that frees up, and its work overlaps theirs.  Admission charges an
estimate of each document's device footprint against the budget; the oldest
resident trees are evicted to make room.  After its build every document
answers a batch of mixed access / rank / select queries on its resident tree
(on the lane's stream).

Reported: p50 / p99 build latency (arrival -> tree ready) and query-batch
latency, admission wait (arrival -> build start), offered and sustained
documents per second, the largest backlog of waiting documents, the number
of micro-batches and their mean size, and the lanes' summed seconds in large
builds, micro-batches and queries.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import bt
from .workloads import Arrival


def estimate_bytes(n: int) -> int:
    """Device footprint charged at admission: the text, build scratch and the
    tree (a conservative multiple of the text, plus fixed overheads)."""
    return 56 * n + (64 << 20)


@dataclass
class DocResult:
    index: int
    n: int
    arrival: float
    start: float = 0.0
    built: float = 0.0
    queried: float = 0.0
    query_batch_s: float = 0.0
    batched: bool = False
    export: bytes | None = None
    queries: dict | None = None     # kept (arguments, answers) per query kind


@dataclass
class Report:
    docs: int
    wall_s: float
    offered_docs_per_s: float
    docs_per_s: float
    mb_per_s: float
    build_p50_ms: float
    build_p99_ms: float
    admission_wait_p50_ms: float
    admission_wait_p99_ms: float
    query_batch_p50_ms: float
    query_batch_p99_ms: float
    queries_per_doc: int
    max_backlog: int
    batches: int
    mean_batch_docs: float
    large_docs: int
    max_concurrent: int
    evictions: int
    lane_seconds: dict = field(default_factory=dict)  # summed over lanes: large builds, batches, queries
    results: list = field(default_factory=list, repr=False)

    def summary(self) -> dict:
        d = dict(self.__dict__)
        d.pop("results")
        return d


class Server:
    def __init__(self, hbm_budget: int = 120 << 30, lanes: int = 4, queries_per_doc: int = 10_000,
                 small_max: int = 1 << 20, max_batch_docs: int = 512, keep_exports: bool = False,
                 keep_queries: int = 0, seed: int = 0, sm_count: int | None = None):
        self.budget = hbm_budget
        self.lanes = lanes
        self.qpd = queries_per_doc
        self.small_max = small_max
        self.max_batch_docs = max_batch_docs
        self.keep_exports = keep_exports
        self.keep_queries = keep_queries
        self.seed = seed
        self.sm_count = sm_count
        self._lock = threading.Condition()
        self._charged = 0
        self._resident = collections.OrderedDict()  # index -> (tree handle, bytes)
        self._inflight = 0
        self._max_inflight = 0
        self._evictions = 0

    # -- memory accounting ---------------------------------------------------
    def _fits_locked(self, need: int) -> bool:
        """Evict the oldest resident trees until `need` fits; True if it does."""
        while self._charged + need > self.budget and self._resident:
            _, (h, b) = self._resident.popitem(last=False)
            bt.bt_free(h)
            self._charged -= b
            self._evictions += 1
        return self._charged + need <= self.budget

    def _charge_locked(self, need: int):
        self._charged += need
        self._inflight += 1
        self._max_inflight = max(self._max_inflight, self._inflight)

    def _admit(self, need: int):
        """Block until `need` bytes fit (a document larger than the budget
        still runs, alone, once nothing else is in flight)."""
        with self._lock:
            while not self._fits_locked(need):
                if self._inflight == 0:
                    break
                self._lock.wait()
            self._charge_locked(need)

    def _try_admit(self, need: int) -> bool:
        with self._lock:
            if not self._fits_locked(need):
                return False
            self._charge_locked(need)
            return True

    def _release(self, estimate: int):
        """A document whose build or queries failed: its admission charge and
        its place among the builds in flight are given back."""
        with self._lock:
            self._charged -= estimate
            self._inflight -= 1
            self._lock.notify_all()

    def _retire(self, index: int, handle: int, estimate: int):
        real = bt.bt_device_bytes(handle)
        with self._lock:
            self._charged += real - estimate
            self._resident[index] = (handle, real)
            self._inflight -= 1
            self._lock.notify_all()

    # -- queries -----------------------------------------------------------
    def _queries(self, handle: int, n: int, rng, stream, keep: int = 0) -> tuple[float, dict | None]:
        """One batch of mixed queries on a resident tree, all on `stream`:
        the symbol counts (rank at n), then access / rank / select arguments
        drawn on the device from the lane's generator `rng` (symbols among
        those present, select ranks within their counts), the three query
        launches and one synchronisation.  With keep > 0 the first `keep`
        arguments and answers of each kind are returned for checking."""
        t0 = time.perf_counter()
        q = self.qpd // 3
        with torch.cuda.stream(stream):
            dev = torch.device("cuda")
            syms = torch.arange(256, dtype=torch.int64, device=dev)
            cnt_args = torch.stack([syms, torch.full_like(syms, n)], 1).reshape(-1).contiguous()
            counts = torch.empty(256, dtype=torch.int64, device=dev)
            bt.bt_query_batch(handle, bt.BT_Q_RANK, cnt_args, 256, counts, stream)
            # The present symbols first, in byte order; np_ of them.
            present = torch.sort((counts == 0).to(torch.int8), stable=True).indices
            np_ = (counts > 0).sum()

            def pick():
                u = torch.randint(0, 1 << 30, (q,), generator=rng, device=dev)
                return present[u % np_]

            acc = torch.randint(0, n, (q,), generator=rng, device=dev)
            cs = pick()
            rk = torch.stack([cs, torch.randint(0, n + 1, (q,), generator=rng, device=dev)], 1).reshape(-1)
            cs2 = pick()
            cnt2 = counts[cs2]
            js = torch.minimum((torch.rand(q, generator=rng, device=dev, dtype=torch.float64) * cnt2)
                               .to(torch.int64) + 1, cnt2)
            sl = torch.stack([cs2, js], 1).reshape(-1)
            rk, sl = rk.contiguous(), sl.contiguous()
            out = torch.empty(3 * q, dtype=torch.int64, device=dev)
            bt.bt_query_batch(handle, bt.BT_Q_ACCESS, acc, q, out[:q], stream)
            bt.bt_query_batch(handle, bt.BT_Q_RANK, rk, q, out[q:2 * q], stream)
            bt.bt_query_batch(handle, bt.BT_Q_SELECT, sl, q, out[2 * q:], stream)
            kept = None
            if keep:
                k = min(keep, q)
                res = out.cpu().numpy()
                kept = {"access": (acc[:k].cpu().numpy(), res[:k].copy()),
                        "rank": (rk[:2 * k].reshape(-1, 2).cpu().numpy(), res[q:q + k].copy()),
                        "select": (sl[:2 * k].reshape(-1, 2).cpu().numpy(), res[2 * q:2 * q + k].copy())}
            stream.synchronize()
        return time.perf_counter() - t0, kept

    # -- main loop ---------------------------------------------------------
    def run(self, arrivals: list[Arrival]) -> Report:
        pending = collections.deque()
        results = [DocResult(i, len(a.doc.text), a.t) for i, a in enumerate(arrivals)]
        done = threading.Event()
        qlock = threading.Condition()
        t_start = time.perf_counter()
        n_total = len(arrivals)
        finished = [0]
        errors = []
        stats = {"backlog": 0, "batches": 0, "batch_docs": 0, "large": 0}
        lane_s = {"large_build": 0.0, "batch_build": 0.0, "queries": 0.0}
        if self.sm_count is None:
            try:
                self.sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            except Exception:  # no device: host tests with fake library calls
                self.sm_count = 152
        ctas = max(1, self.sm_count // max(1, self.lanes))

        def finish(k: int):
            with qlock:
                finished[0] += k
                if finished[0] >= n_total:
                    done.set()
                qlock.notify_all()

        def take():
            """The next unit of work: [one large document] or [small ones]."""
            with qlock:
                while not pending and not done.is_set():
                    qlock.wait()
                if not pending:
                    return None
                first = pending[0]
                if results[first].n > self.small_max:
                    pending.popleft()
                    return [first]
                # The small documents waiting, in arrival order, up to a batch;
                # the large ones among them keep their places.
                batch, rest = [], collections.deque()
                while pending and len(batch) < self.max_batch_docs:
                    i = pending.popleft()
                    (batch if results[i].n <= self.small_max else rest).append(i)
                rest.extend(pending)
                pending.clear()
                pending.extend(rest)
                return batch

        def serve_unit(unit, stream, rng):
            ests = [estimate_bytes(results[i].n) for i in unit]
            # The first document waits for room; the rest join the batch only
            # while they fit now, and go back to the queue otherwise.
            self._admit(ests[0])
            admitted = 1
            while admitted < len(unit) and self._try_admit(ests[admitted]):
                admitted += 1
            if admitted < len(unit):
                with qlock:
                    for i in reversed(unit[admitted:]):
                        pending.appendleft(i)
                    qlock.notify_all()
                unit, ests = unit[:admitted], ests[:admitted]
            handles = [None] * len(unit)
            try:
                t0 = time.perf_counter() - t_start
                for i in unit:
                    results[i].start = t0
                docs = [arrivals[i].doc for i in unit]
                if len(unit) == 1 and results[unit[0]].n > self.small_max:
                    d = docs[0]
                    handles[0] = bt.bt_build_ex(d.text, len(d.text), d.sigma, d.tau, d.leaf_len,
                                                bt.bt_opts_default(), stream.cuda_stream)
                    with qlock:
                        stats["large"] += 1
                else:
                    o, keep = bt.BuildOptions(batch_ctas=ctas).to_c()
                    handles = bt.bt_build_batch([d.text for d in docs], [len(d.text) for d in docs],
                                                [d.sigma for d in docs], [d.tau for d in docs],
                                                [d.leaf_len for d in docs], o)
                    del keep
                    for i in unit:
                        results[i].batched = True
                    with qlock:
                        stats["batches"] += 1
                        stats["batch_docs"] += len(unit)
                t1 = time.perf_counter() - t_start
                with qlock:
                    lane_s["large_build" if results[unit[0]].n > self.small_max else "batch_build"] += t1 - t0
                for i, h in zip(unit, handles):
                    r = results[i]
                    r.built = t1
                    if self.keep_exports:
                        r.export = bt.bt_export(h)
                    r.query_batch_s, r.queries = self._queries(h, r.n, rng, stream, self.keep_queries)
                    r.queried = time.perf_counter() - t_start
                with qlock:
                    lane_s["queries"] += time.perf_counter() - t_start - t1
            except BaseException:
                for h in handles:
                    if h is not None:
                        bt.bt_free(h)
                for e in ests:
                    self._release(e)
                raise
            for i, h, e in zip(unit, handles, ests):
                self._retire(i, h, e)
            return len(unit)

        def lane(widx: int):
            try:
                stream = torch.cuda.Stream()
                rng = None  # without a device (host tests) the queries take no generator
                if torch.cuda.is_available():
                    rng = torch.Generator(device="cuda")
                    rng.manual_seed(self.seed * 1000 + widx)
            except BaseException as e:  # a lane that cannot start: recorded like a failed unit
                with qlock:
                    errors.append(e)
                    qlock.notify_all()
                return
            while True:
                unit = take()
                if unit is None:
                    return
                try:
                    k = serve_unit(unit, stream, rng)
                except BaseException as e:  # recorded; run() re-raises the first one
                    with qlock:
                        errors.append(e)
                    k = len(unit)
                finish(k)

        threads = [threading.Thread(target=lane, args=(w,), daemon=True) for w in range(self.lanes)]
        for th in threads:
            th.start()
        for i, a in enumerate(arrivals):
            delay = a.t - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            with qlock:
                pending.append(i)
                stats["backlog"] = max(stats["backlog"], len(pending))
                qlock.notify()
        if n_total == 0:
            done.set()
        with qlock:
            while not done.is_set() and any(th.is_alive() for th in threads):
                qlock.wait(timeout=1.0)
            done.set()
            qlock.notify_all()
        for th in threads:
            th.join()
        wall = time.perf_counter() - t_start
        torch.cuda.synchronize()
        if not errors and finished[0] < n_total:
            raise RuntimeError(f"serving lanes ended with {n_total - finished[0]} documents unserved")
        if errors:
            raise errors[0]
        build_lat = np.array([r.built - r.arrival for r in results]) * 1e3
        wait = np.array([r.start - r.arrival for r in results]) * 1e3
        q_lat = np.array([r.query_batch_s for r in results]) * 1e3
        total_bytes = sum(r.n for r in results)
        span = arrivals[-1].t if n_total else 0.0
        pct = (lambda a, p: float(np.percentile(a, p)) if n_total else 0.0)
        return Report(
            docs=n_total, wall_s=wall, offered_docs_per_s=n_total / span if span > 0 else 0.0,
            docs_per_s=n_total / wall if wall > 0 else 0.0, mb_per_s=total_bytes / wall / 1e6 if wall > 0 else 0.0,
            build_p50_ms=pct(build_lat, 50), build_p99_ms=pct(build_lat, 99),
            admission_wait_p50_ms=pct(wait, 50), admission_wait_p99_ms=pct(wait, 99),
            query_batch_p50_ms=pct(q_lat, 50), query_batch_p99_ms=pct(q_lat, 99),
            queries_per_doc=3 * (self.qpd // 3), max_backlog=stats["backlog"], batches=stats["batches"],
            mean_batch_docs=stats["batch_docs"] / stats["batches"] if stats["batches"] else 0.0,
            large_docs=stats["large"], max_concurrent=self._max_inflight, evictions=self._evictions,
            lane_seconds=lane_s, results=results)

    def close(self):
        with self._lock:
            for h, _ in self._resident.values():
                bt.bt_free(h)
            self._resident.clear()
            self._charged = 0
