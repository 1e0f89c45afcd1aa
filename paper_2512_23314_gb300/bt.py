"""ctypes binding of libbt.so -- argument marshalling only.

Every function has the name and argument order of its C entry point in
``include/bt.h``; non-zero status codes raise ``BTError``.  Texts may be
numpy uint8 arrays / bytes (host memory) or torch uint8 CUDA tensors (device
memory); query batches take device tensors.  There is no CPU fallback: if
the CUDA library is not built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libbt.so")

BT_OK, BT_EINVAL, BT_ERANGE, BT_ENOMEM, BT_ECUDA, BT_ETIMEOUT, BT_EINTERNAL = range(7)
BT_Q_ACCESS, BT_Q_RANK, BT_Q_SELECT = 0, 1, 2
BT_FLAG_DENSE_SCAN = 1
BT_FLAG_TINY_QUEUE = 2
BT_FLAG_GRAM_LIST = 4
BT_FLAG_TWO_PHASE = 8
BT_FLAG_BATCH_WORKERS = 16
BT_FLAG_LEAF_COUNTS = 32
BT_FLAG_SORT_SCAN = 64
BT_FLAG_ANCHOR_ALL = 128
ST_FIELDS = 10
ST_NAMES = ("nblocks", "b", "cov", "nmarked", "npairs", "verify_bytes", "collisions",
            "final_blocks", "candidates", "hits")


class BTError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class bt_opts(ctypes.Structure):
    _fields_ = [("prune", ctypes.c_int), ("root_arity", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("modulus", ctypes.c_uint64),
                ("level_sizes", ctypes.c_void_p), ("nlevels", ctypes.c_uint32),
                ("max_rounds", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("batch_ctas", ctypes.c_uint32), ("partitions", ctypes.c_uint32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"{LIBPATH} is missing: build it with "
                           "`python -m paper_2512_23314_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIBPATH)
    vp, u64, u32, u8 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint8
    P = ctypes.POINTER
    L.bt_opts_default.argtypes = [P(bt_opts)]
    L.bt_opts_default.restype = None
    L.bt_build.argtypes = [vp, u64, u32, u32, u32, P(vp)]
    L.bt_build_ex.argtypes = [vp, u64, u32, u32, u32, P(bt_opts), vp, P(vp)]
    L.bt_build_batch.argtypes = [vp, vp, vp, vp, vp, u64, P(bt_opts), u32, vp]
    L.bt_access.argtypes = [vp, u64, P(u8)]
    L.bt_rank.argtypes = [vp, u8, u64, P(u64)]
    L.bt_select.argtypes = [vp, u8, u64, P(u64)]
    L.bt_query_batch.argtypes = [vp, ctypes.c_int, vp, u64, vp, vp]
    L.bt_export.argtypes = [vp, vp, u64, P(u64)]
    L.bt_device_bytes.argtypes = [vp]
    L.bt_device_bytes.restype = u64
    L.bt_levels.argtypes = [vp]
    L.bt_levels.restype = u32
    L.bt_stats.argtypes = [vp, P(u64), u64]
    L.bt_prefix_fingerprints.argtypes = [vp, u64, u64, u64, u32, vp, vp]
    L.bt_prefix_fingerprints_noalloc.argtypes = [vp, u64, u64, u64, u32, vp, vp]
    L.bt_fingerprint_base.argtypes = [u64, u64]
    L.bt_fingerprint_base.restype = u64
    L.bt_free.argtypes = [vp]
    L.bt_free.restype = None
    L.bt_strerror.argtypes = [ctypes.c_int]
    L.bt_strerror.restype = ctypes.c_char_p
    L.bt_profile_enable.argtypes = [ctypes.c_int]
    L.bt_profile_enable.restype = None
    L.bt_profile_reset.argtypes = []
    L.bt_profile_reset.restype = None
    L.bt_profile_read.argtypes = [vp, u32, P(u32)]
    L.bt_launch_count.argtypes = []
    L.bt_launch_count.restype = u64
    L.bt_mulmod_bench.argtypes = [u32, u32, u64, vp, vp, P(u64)]
    L.bt_batch_report.argtypes = [vp, u32]
    L.bt_test_alloc_limit.argtypes = [u64]
    L.bt_test_alloc_limit.restype = None
    L.bt_device_pool_used.argtypes = [P(u64)]
    L.bt_device_pool_peak.argtypes = [P(u64), ctypes.c_int]
    L.bt_batch_cycles.argtypes = [vp, vp, u32]
    for name in ("bt_profile_read", "bt_build", "bt_build_ex", "bt_build_batch", "bt_access", "bt_rank", "bt_select",
                 "bt_query_batch", "bt_export", "bt_stats", "bt_prefix_fingerprints",
                 "bt_prefix_fingerprints_noalloc", "bt_mulmod_bench"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().bt_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def _check(rc: int, what: str):
    if rc != BT_OK:
        raise BTError(rc, what)


def _text_ptr(text):
    """(pointer, length, keepalive) for bytes / numpy (host) or a torch tensor."""
    if isinstance(text, (bytes, bytearray)):
        a = np.frombuffer(bytes(text), dtype=np.uint8)
        return a.ctypes.data, len(a), a
    if isinstance(text, np.ndarray):
        a = np.ascontiguousarray(text)
        if a.dtype != np.uint8:
            raise TypeError("text must be uint8")
        return a.ctypes.data, a.size, a
    if hasattr(text, "data_ptr"):  # torch tensor (host or device)
        if not text.is_contiguous() or text.element_size() != 1:
            raise TypeError("text tensor must be contiguous uint8")
        return text.data_ptr(), text.numel(), text
    raise TypeError(f"unsupported text type {type(text)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def bt_opts_default() -> bt_opts:
    o = bt_opts()
    lib().bt_opts_default(ctypes.byref(o))
    return o


def bt_build(text, n: int, sigma: int, tau: int, leaf_len: int) -> int:
    ptr, _, keep = _text_ptr(text)
    h = ctypes.c_void_p()
    _check(lib().bt_build(ptr, n, sigma, tau, leaf_len, ctypes.byref(h)), "bt_build")
    del keep
    return h.value


def bt_build_ex(text, n: int, sigma: int, tau: int, leaf_len: int, opts: bt_opts | None = None,
                stream=None) -> int:
    ptr, _, keep = _text_ptr(text)
    h = ctypes.c_void_p()
    o = opts if opts is not None else bt_opts_default()
    _check(lib().bt_build_ex(ptr, n, sigma, tau, leaf_len, ctypes.byref(o), _stream_ptr(stream),
                             ctypes.byref(h)), "bt_build_ex")
    del keep
    return h.value


def bt_build_batch(texts, ns, sigmas, taus, leaf_lens, opts: bt_opts | None = None,
                   nworkers: int = 0) -> list[int]:
    """Build many documents in one call; returns one tree handle per document."""
    nd = len(texts)
    keep = [_text_ptr(t) for t in texts]
    ptrs = (ctypes.c_void_p * max(1, nd))(*[k[0] for k in keep])
    a_ns = np.ascontiguousarray(ns, dtype=np.uint64)
    a_sg = np.ascontiguousarray(sigmas, dtype=np.uint32)
    a_tau = np.ascontiguousarray(taus, dtype=np.uint32)
    a_leaf = np.ascontiguousarray(leaf_lens, dtype=np.uint32)
    outs = (ctypes.c_void_p * max(1, nd))()
    o = opts if opts is not None else bt_opts_default()
    _check(lib().bt_build_batch(ptrs, a_ns.ctypes.data, a_sg.ctypes.data, a_tau.ctypes.data,
                                a_leaf.ctypes.data, nd, ctypes.byref(o), nworkers, outs),
           "bt_build_batch")
    del keep
    return [outs[i] for i in range(nd)]


def bt_batch_report() -> dict:
    """What the last bt_build_batch call did (measurement hook)."""
    a = (ctypes.c_uint64 * 13)()
    _check(lib().bt_batch_report(a, 13), "bt_batch_report")
    names = ("kernel_docs", "worker_docs", "launches", "retried", "threads", "ctas_per_sm", "pool_bytes",
             "scratch_bytes", "max_grid", "chunk", "tuning_trials", "upload_us", "kernel_us")
    return dict(zip(names, list(a)))


def bt_batch_cycles(t: int) -> list[int]:
    """SM cycles per phase of the CTA that built a batched tree."""
    a = (ctypes.c_uint64 * 6)()
    _check(lib().bt_batch_cycles(t, a, 6), "bt_batch_cycles")
    return list(a)


def bt_test_alloc_limit(nbytes: int) -> None:
    """Test hook: device allocations of a build larger than nbytes fail (0: off)."""
    lib().bt_test_alloc_limit(nbytes)


def bt_device_pool_peak(reset: bool = False) -> int:
    """High-water mark of the stream-ordered pool's bytes (reset: restart it)."""
    v = ctypes.c_uint64()
    _check(lib().bt_device_pool_peak(ctypes.byref(v), int(reset)), "bt_device_pool_peak")
    return v.value


def bt_device_pool_used() -> int:
    """Bytes allocated from the device's stream-ordered pool right now."""
    v = ctypes.c_uint64()
    _check(lib().bt_device_pool_used(ctypes.byref(v)), "bt_device_pool_used")
    return v.value


def bt_access(t: int, i: int) -> int:
    out = ctypes.c_uint8()
    _check(lib().bt_access(t, i, ctypes.byref(out)), "bt_access")
    return out.value


def bt_rank(t: int, c: int, i: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().bt_rank(t, c, i, ctypes.byref(out)), "bt_rank")
    return out.value


def bt_select(t: int, c: int, j: int) -> int:
    out = ctypes.c_uint64()
    _check(lib().bt_select(t, c, j, ctypes.byref(out)), "bt_select")
    return out.value


def bt_query_batch(t: int, kind: int, d_args, m: int, d_out, stream=None) -> None:
    _check(lib().bt_query_batch(t, kind, d_args.data_ptr(), m, d_out.data_ptr(),
                                _stream_ptr(stream)), "bt_query_batch")


def bt_export(t: int) -> bytearray:
    """The canonical serialization (a bytes-like bytearray, written in place)."""
    n = ctypes.c_uint64()
    _check(lib().bt_export(t, None, 0, ctypes.byref(n)), "bt_export")
    buf = bytearray(n.value)
    _check(lib().bt_export(t, (ctypes.c_uint8 * n.value).from_buffer(buf), n.value, ctypes.byref(n)),
           "bt_export")
    return buf


def bt_export_into(t: int, out) -> int:
    """Write the canonical serialization into `out` (a contiguous host uint8
    tensor, e.g. pinned, or a writable buffer); returns its length in bytes."""
    n = ctypes.c_uint64()
    if hasattr(out, "data_ptr"):
        if out.is_cuda or not out.is_contiguous() or out.element_size() != 1:
            raise TypeError("out must be a contiguous host uint8 tensor")
        ptr, cap = out.data_ptr(), out.numel()
    else:
        view = memoryview(out)
        cap = view.nbytes
        ptr = ctypes.addressof((ctypes.c_uint8 * cap).from_buffer(out))
    _check(lib().bt_export(t, ptr, cap, ctypes.byref(n)), "bt_export")
    return n.value


def bt_device_bytes(t: int) -> int:
    return int(lib().bt_device_bytes(t))


def bt_levels(t: int) -> int:
    return int(lib().bt_levels(t))


def bt_stats(t: int) -> list[dict]:
    L = bt_levels(t)
    a = (ctypes.c_uint64 * (L * ST_FIELDS))()
    _check(lib().bt_stats(t, a, L * ST_FIELDS), "bt_stats")
    return [dict(zip(ST_NAMES, a[l * ST_FIELDS:(l + 1) * ST_FIELDS])) for l in range(L)]


def bt_prefix_fingerprints(d_text, n: int, seed: int, modulus: int, stride: int, d_out,
                           stream=None) -> None:
    _check(lib().bt_prefix_fingerprints(d_text.data_ptr(), n, seed, modulus, stride,
                                        d_out.data_ptr(), _stream_ptr(stream)),
           "bt_prefix_fingerprints")


def bt_prefix_fingerprints_noalloc(d_text, n: int, seed: int, modulus: int, stride: int, d_out,
                                   stream=None) -> None:
    _check(lib().bt_prefix_fingerprints_noalloc(d_text.data_ptr(), n, seed, modulus, stride,
                                                d_out.data_ptr(), _stream_ptr(stream)),
           "bt_prefix_fingerprints_noalloc")


def bt_fingerprint_base(seed: int, modulus: int = 0) -> int:
    return int(lib().bt_fingerprint_base(seed, modulus))


def bt_free(t: int) -> None:
    if t:
        lib().bt_free(t)


def bt_strerror(code: int) -> str:
    return strerror(code)


class bt_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_uint64)]


def bt_profile_enable(on: bool) -> None:
    lib().bt_profile_enable(int(bool(on)))


def bt_profile_reset() -> None:
    lib().bt_profile_reset()


def bt_profile_read() -> dict:
    cnt = ctypes.c_uint32()
    _check(lib().bt_profile_read(None, 0, ctypes.byref(cnt)), "bt_profile_read")
    arr = (bt_profile_entry * max(1, cnt.value))()
    _check(lib().bt_profile_read(arr, cnt.value, ctypes.byref(cnt)), "bt_profile_read")
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms,
                                   "bytes": arr[i].bytes} for i in range(cnt.value)}


def bt_launch_count() -> int:
    return int(lib().bt_launch_count())


def bt_mulmod_bench(blocks: int, iters: int, d_out, stream=None, seed: int = 0) -> int:
    """Launch the modular-multiply microbenchmark on `stream` (a torch stream
    or None); d_out is a device tensor of blocks * 256 int64.  Returns the
    number of multiplies launched (time the launch with CUDA events)."""
    n = ctypes.c_uint64()
    _check(lib().bt_mulmod_bench(blocks, iters, seed, ctypes.c_void_p(d_out.data_ptr()), _stream_ptr(stream),
                                 ctypes.byref(n)), "bt_mulmod_bench")
    return int(n.value)


@dataclass
class BuildOptions:
    prune: bool = True
    root_arity: int = 0
    seed: int = 0
    modulus: int = 0
    level_sizes: tuple | None = None
    max_rounds: int = 0
    dense_scan: bool = False
    tiny_queue: bool = False  # test hook: forces the scan's queue-overflow path
    gram_list: bool = False  # test hook: selected-gram list whatever the text length
    two_phase: bool = False  # two-phase window tests on every anchored level (same tree)
    batch_workers: bool = False  # bt_build_batch: host workers instead of the batched kernel
    batch_ctas: int = 0  # bt_build_batch: CTAs of the batched kernel's launch (0: every SM)
    leaf_counts: bool = False  # no stored counters on the last level (space-efficient rank/select)
    sort_scan: bool = False  # leftmost windows by radix-sorting (fingerprint, position) tuples
    partitions: int = 0  # with sort_scan: parts of the domain decomposition (0 or 1: one)
    anchor_all: bool = False  # bt_build_batch test hook: anchored scan on every level of 32+ byte blocks

    def to_c(self):
        o = bt_opts_default()
        o.prune = int(self.prune)
        o.root_arity = self.root_arity
        o.seed = self.seed
        o.modulus = self.modulus
        o.max_rounds = self.max_rounds
        o.batch_ctas = self.batch_ctas
        o.partitions = self.partitions
        o.flags = ((BT_FLAG_DENSE_SCAN if self.dense_scan else 0)
                   | (BT_FLAG_TINY_QUEUE if self.tiny_queue else 0)
                   | (BT_FLAG_GRAM_LIST if self.gram_list else 0)
                   | (BT_FLAG_TWO_PHASE if self.two_phase else 0)
                   | (BT_FLAG_BATCH_WORKERS if self.batch_workers else 0)
                   | (BT_FLAG_LEAF_COUNTS if self.leaf_counts else 0)
                   | (BT_FLAG_SORT_SCAN if self.sort_scan else 0)
                   | (BT_FLAG_ANCHOR_ALL if self.anchor_all else 0))
        keep = None
        if self.level_sizes is not None:
            keep = np.ascontiguousarray(self.level_sizes, dtype=np.uint64)
            o.level_sizes = keep.ctypes.data
            o.nlevels = len(keep)
        return o, keep


class Tree:
    """Owning wrapper of a bt_tree handle."""

    def __init__(self, text, sigma: int, tau: int, leaf_len: int, options: BuildOptions | None = None,
                 stream=None):
        _, n, _ = _text_ptr(text)
        o, keep = (options or BuildOptions()).to_c()
        self.handle = bt_build_ex(text, n, sigma, tau, leaf_len, o, stream)
        del keep
        self.n = n

    def close(self):
        if getattr(self, "handle", None):
            bt_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def export(self) -> bytearray:
        return bt_export(self.handle)

    def stats(self) -> list[dict]:
        return bt_stats(self.handle)

    def access(self, i: int) -> int:
        return bt_access(self.handle, i)

    def rank(self, c: int, i: int) -> int:
        return bt_rank(self.handle, c, i)

    def select(self, c: int, j: int) -> int:
        return bt_select(self.handle, c, j)

    def query_batch(self, kind: int, d_args, d_out, stream=None):
        m = d_out.numel()
        bt_query_batch(self.handle, kind, d_args, m, d_out, stream)
