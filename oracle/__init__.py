"""CPU oracle for block-tree construction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

Two independent builders live here:

* ``build`` -- the plain single-threaded C builder (``bt_oracle.c``): Karp-Rabin
  fingerprints (section 2) in a hash table and one rolling scan over all of T
  per key length, every match verified byte by byte (section 3.1), then the
  optional pruning pass and access/rank/select on the finished tree;
* ``brute.build`` -- the definition written out in Python with ``bytes.find``
  as the leftmost-occurrence search, for tiny inputs only.

Parity: pinned.  The C builder is checked against the brute-force builder on
thousands of seeded tiny inputs, against the worked example of Figure 1,
against closed forms (a^n, texts without repeats, n <= leaf_len), against
naive access/rank/select counts, and against invariants that hold for any
block tree (pointers copy their target, targets lie strictly left, the
blocks-per-level bound of Lemma 5, independence of the fingerprint base and
modulus).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libbt_oracle.so")
_SRC = os.path.join(_HERE, "bt_oracle.c")

OK, EINVAL, ERANGE, ENOMEM, EINTERNAL = 0, 1, 2, 3, 4
ST_FIELDS = 7
ST_NAMES = ("nblocks", "b", "cov", "nmarked", "npairs", "verify_bytes", "collisions")


def build_library(force: bool = False) -> str:
    """Compile the C oracle with the host compiler (plain gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    fresh = os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bt_oracle.h")))
    if force or not fresh:
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_library())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        vp = ctypes.c_void_p
        L.bto_build.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                vp, ctypes.POINTER(vp)]
        L.bto_export.argtypes = [vp, vp, ctypes.c_uint64, u64p]
        L.bto_access.argtypes = [vp, ctypes.c_uint64, u8p]
        L.bto_rank.argtypes = [vp, ctypes.c_uint8, ctypes.c_uint64, u64p]
        L.bto_select.argtypes = [vp, ctypes.c_uint8, ctypes.c_uint64, u64p]
        L.bto_levels.argtypes = [vp]
        L.bto_levels.restype = ctypes.c_uint32
        L.bto_stats.argtypes = [vp, u64p, ctypes.c_uint64]
        L.bto_free.argtypes = [vp]
        L.bto_free.restype = None
        L.bto_base.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.bto_base.restype = ctypes.c_uint64
        L.bto_fingerprint.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64]
        L.bto_fingerprint.restype = ctypes.c_uint64
        _lib = L
    return _lib


class _Opts(ctypes.Structure):
    _fields_ = [("prune", ctypes.c_int), ("root_arity", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("modulus", ctypes.c_uint64),
                ("level_sizes", ctypes.c_void_p), ("nlevels", ctypes.c_uint32)]


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def _as_bytes(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        return np.frombuffer(bytes(text), dtype=np.uint8)
    a = np.ascontiguousarray(text)
    if a.dtype != np.uint8:
        raise TypeError("text must be uint8")
    return a


class Tree:
    """A block tree built by the C oracle; owns the native handle."""

    def __init__(self, text, tau: int, leaf_len: int, prune: bool = True, seed: int = 0,
                 modulus: int = 0, root_arity: int = 0, level_sizes=None):
        self._lib = lib()
        self.text = _as_bytes(text)
        sizes = None
        o = _Opts(int(bool(prune)), root_arity, seed, modulus, None, 0)
        if level_sizes is not None:
            sizes = np.ascontiguousarray(level_sizes, dtype=np.uint64)
            o.level_sizes = sizes.ctypes.data
            o.nlevels = len(sizes)
        h = ctypes.c_void_p()
        rc = self._lib.bto_build(self.text.ctypes.data, len(self.text), tau, leaf_len,
                                 ctypes.byref(o), ctypes.byref(h))
        if rc != OK:
            raise OracleError(rc, "bto_build")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.bto_free(h)
            self._h = None

    @property
    def levels(self) -> int:
        return int(self._lib.bto_levels(self._h))

    def export(self) -> bytes:
        n = ctypes.c_uint64()
        rc = self._lib.bto_export(self._h, None, 0, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "bto_export")
        buf = (ctypes.c_uint8 * n.value)()
        rc = self._lib.bto_export(self._h, buf, n.value, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "bto_export")
        return bytes(buf)

    def stats(self) -> list[dict]:
        L = self.levels
        a = (ctypes.c_uint64 * (L * ST_FIELDS))()
        rc = self._lib.bto_stats(self._h, a, L * ST_FIELDS)
        if rc != OK:
            raise OracleError(rc, "bto_stats")
        return [dict(zip(ST_NAMES, a[l * ST_FIELDS:(l + 1) * ST_FIELDS])) for l in range(L)]

    def access(self, i: int) -> int:
        out = ctypes.c_uint8()
        rc = self._lib.bto_access(self._h, i, ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "bto_access")
        return out.value

    def rank(self, c: int, i: int) -> int:
        out = ctypes.c_uint64()
        rc = self._lib.bto_rank(self._h, c, i, ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "bto_rank")
        return out.value

    def select(self, c: int, j: int) -> int:
        out = ctypes.c_uint64()
        rc = self._lib.bto_select(self._h, c, j, ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "bto_select")
        return out.value


def build(text, tau: int, leaf_len: int, **kw) -> Tree:
    return Tree(text, tau, leaf_len, **kw)


def base(seed: int, modulus: int = 0) -> int:
    return int(lib().bto_base(seed, modulus))


def fingerprint(text, s: int, length: int, b: int, modulus: int = 0) -> int:
    a = _as_bytes(text)
    return int(lib().bto_fingerprint(a.ctypes.data, s, length, b, modulus))


# ---------------------------------------------------------------------------
# Canonical serialization reader (shared by tests to compare and inspect).
# ---------------------------------------------------------------------------

@dataclass
class Level:
    b: int
    marks: list
    ptrs: list  # (ptr, off) of the unmarked blocks, in block order


@dataclass
class Parsed:
    n: int
    tau: int
    leaf_len: int
    prune: int
    levels: list
    leaf_text: bytes


def parse(blob: bytes, as_numpy: bool = False) -> Parsed:
    """Read the canonical serialization.  With as_numpy, marks are a numpy
    bool array and ptrs an (nptr, 2) int64 array (fast for large trees)."""
    a = np.frombuffer(blob, dtype="<u8")
    if int(a[0]) != 0x31454552544B4C42:
        raise ValueError("bad magic")
    n, tau, leaf, L, prune = (int(x) for x in a[1:6])
    i = 6
    levels = []
    for _ in range(L):
        c, b = int(a[i]), int(a[i + 1])
        i += 2
        nw = (c + 63) // 64
        words = np.ascontiguousarray(a[i:i + nw])
        i += nw
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:c].astype(bool)
        nptr = int(a[i])
        i += 1
        pa = a[i:i + 2 * nptr].reshape(-1, 2).astype(np.int64)
        i += 2 * nptr
        if as_numpy:
            levels.append(Level(b, bits, pa))
        else:
            levels.append(Level(b, [int(x) for x in bits], [(int(p), int(o)) for p, o in pa]))
    nleaf = int(a[i])
    i += 1
    leaf_text = blob[8 * i:8 * i + nleaf]
    return Parsed(n, tau, leaf, prune, levels, leaf_text)
