"""Serving loop: continuous batching of block-tree builds under an HBM budget.

Documents arrive over time.  A document is admitted when its estimated
device footprint fits in the budget next to the builds in flight and the
trees kept resident.  The oldest resident trees are evicted to make room.
Admitted documents go to `nworkers` worker threads, each issuing its builds
and queries on its own CUDA stream through the C ABI.  A document that
arrives while others are on the GPU therefore starts as soon as a worker and
memory are free, and its kernels overlap theirs.  After its build, every
document answers a batch of mixed access / rank / select queries on its
resident tree.

Latencies: build = arrival -> tree ready; query = one batch of queries
(submission -> answers on the host).  Reported as p50 / p99 with sustained
documents per second.
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
    export: bytes | None = None
    queries: dict | None = None     # kept (arguments, answers) per query kind


@dataclass
class Report:
    docs: int
    wall_s: float
    docs_per_s: float
    mb_per_s: float
    build_p50_ms: float
    build_p99_ms: float
    query_batch_p50_ms: float
    query_batch_p99_ms: float
    queries_per_doc: int
    max_concurrent: int
    evictions: int
    results: list = field(default_factory=list, repr=False)

    def summary(self) -> dict:
        d = dict(self.__dict__)
        d.pop("results")
        return d


class Server:
    def __init__(self, hbm_budget: int = 120 << 30, nworkers: int = 8, queries_per_doc: int = 10_000,
                 keep_exports: bool = False, keep_queries: int = 0, seed: int = 0):
        self.budget = hbm_budget
        self.nworkers = nworkers
        self.qpd = queries_per_doc
        self.keep_exports = keep_exports
        self.keep_queries = keep_queries
        self.seed = seed
        self._lock = threading.Condition()
        self._charged = 0
        self._resident = collections.OrderedDict()  # index -> (tree handle, bytes)
        self._inflight = 0
        self._max_inflight = 0
        self._evictions = 0

    # -- memory accounting ---------------------------------------------------
    def _admit(self, need: int):
        with self._lock:
            while self._charged + need > self.budget:
                if self._resident:
                    _, (h, b) = self._resident.popitem(last=False)
                    bt.bt_free(h)
                    self._charged -= b
                    self._evictions += 1
                    continue
                if self._inflight == 0:
                    break  # a single document larger than the budget still runs alone
                self._lock.wait()
            self._charged += need
            self._inflight += 1
            self._max_inflight = max(self._max_inflight, self._inflight)

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
    def _queries(self, handle: int, n: int, rng: np.random.Generator, stream,
                 keep: int = 0) -> tuple[float, dict | None]:
        """One batch of mixed queries on a resident tree, all on `stream` (the
        argument tensors are made inside the stream context, so no kernel of
        another stream writes them).  With keep > 0 the first `keep`
        arguments and answers of each kind are returned for checking."""
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            syms = torch.arange(256, dtype=torch.int64, device="cuda")
            cnt_args = torch.stack([syms, torch.full_like(syms, n)], 1).reshape(-1).contiguous()
            counts = torch.empty(256, dtype=torch.int64, device="cuda")
            bt.bt_query_batch(handle, bt.BT_Q_RANK, cnt_args, 256, counts, stream)
            c = counts.cpu().numpy()
            present = np.flatnonzero(c > 0)
            q = self.qpd // 3
            acc_h = rng.integers(0, n, q)
            cs = rng.choice(present, q)
            rk_h = np.stack([cs, rng.integers(0, n + 1, q)], 1).reshape(-1)
            cs2 = rng.choice(present, q)
            js = (rng.random(q) * c[cs2]).astype(np.int64) + 1
            sl_h = np.stack([cs2, js], 1).reshape(-1)
            acc = torch.from_numpy(acc_h).to("cuda", non_blocking=True)
            rk = torch.from_numpy(rk_h).cuda()
            sl = torch.from_numpy(sl_h).cuda()
            out = torch.empty(3 * q, dtype=torch.int64, device="cuda")
            bt.bt_query_batch(handle, bt.BT_Q_ACCESS, acc, q, out[:q], stream)
            bt.bt_query_batch(handle, bt.BT_Q_RANK, rk, q, out[q:2 * q], stream)
            bt.bt_query_batch(handle, bt.BT_Q_SELECT, sl, q, out[2 * q:], stream)
            res = out.cpu().numpy()
        dt = time.perf_counter() - t0
        kept = None
        if keep:
            k = min(keep, q)
            kept = {"access": (acc_h[:k].copy(), res[:k].copy()),
                    "rank": (rk_h[:2 * k].reshape(-1, 2).copy(), res[q:q + k].copy()),
                    "select": (sl_h[:2 * k].reshape(-1, 2).copy(), res[2 * q:2 * q + k].copy())}
        return dt, kept

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

        def finish_one():
            with qlock:
                finished[0] += 1
                if finished[0] == n_total:
                    done.set()
                qlock.notify_all()

        def serve_one(i, stream, rng, opts):
            a = arrivals[i]
            r = results[i]
            est = estimate_bytes(r.n)
            self._admit(est)
            h = None
            try:
                r.start = time.perf_counter() - t_start
                h = bt.bt_build_ex(a.doc.text, r.n, a.doc.sigma, a.doc.tau, a.doc.leaf_len, opts,
                                   stream.cuda_stream)
                r.built = time.perf_counter() - t_start
                if self.keep_exports:
                    r.export = bt.bt_export(h)
                r.query_batch_s, r.queries = self._queries(h, r.n, rng, stream, self.keep_queries)
                r.queried = time.perf_counter() - t_start
            except BaseException:
                if h is not None:
                    bt.bt_free(h)
                self._release(est)
                raise
            self._retire(i, h, est)

        def worker(widx: int):
            stream = torch.cuda.Stream()
            rng = np.random.default_rng(self.seed * 1000 + widx)
            opts = bt.bt_opts_default()
            while True:
                with qlock:
                    while not pending and not done.is_set():
                        qlock.wait()
                    if not pending:
                        return
                    i = pending.popleft()
                try:
                    serve_one(i, stream, rng, opts)
                except BaseException as e:  # recorded; run() re-raises the first one
                    with qlock:
                        errors.append(e)
                finally:
                    finish_one()

        threads = [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(self.nworkers)]
        for th in threads:
            th.start()
        for i, a in enumerate(arrivals):
            delay = a.t - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            with qlock:
                pending.append(i)
                qlock.notify()
        if n_total == 0:
            done.set()
        with qlock:
            while not done.is_set():
                qlock.wait(timeout=1.0)
            qlock.notify_all()
        for th in threads:
            th.join()
        wall = time.perf_counter() - t_start
        torch.cuda.synchronize()
        if errors:
            raise errors[0]
        build_lat = np.array([r.built - r.arrival for r in results]) * 1e3
        q_lat = np.array([r.query_batch_s for r in results]) * 1e3
        total_bytes = sum(r.n for r in results)
        rep = Report(
            docs=n_total, wall_s=wall, docs_per_s=n_total / wall, mb_per_s=total_bytes / wall / 1e6,
            build_p50_ms=float(np.percentile(build_lat, 50)) if n_total else 0.0,
            build_p99_ms=float(np.percentile(build_lat, 99)) if n_total else 0.0,
            query_batch_p50_ms=float(np.percentile(q_lat, 50)) if n_total else 0.0,
            query_batch_p99_ms=float(np.percentile(q_lat, 99)) if n_total else 0.0,
            queries_per_doc=3 * (self.qpd // 3), max_concurrent=self._max_inflight,
            evictions=self._evictions, results=results)
        return rep

    def close(self):
        with self._lock:
            for h, _ in self._resident.values():
                bt.bt_free(h)
            self._resident.clear()
            self._charged = 0
