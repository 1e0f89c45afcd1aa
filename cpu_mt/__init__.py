"""The multithreaded CPU baseline (OpenMP): a straightforward parallel
block-tree builder timed beside the GPU build on the same host.

`build()` compiles `bt_cpu_mt.c` with gcc -fopenmp into `cpu_mt/_lib/`;
`build_tree()` returns the canonical serialization of the tree (the layout of
`bt_export`).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libbt_cpu_mt.so")
_SRC = os.path.join(_HERE, "bt_cpu_mt.c")
_HDR = os.path.join(_HERE, "bt_cpu_mt.h")


def build(force: bool = False) -> str:
    os.makedirs(_LIBDIR, exist_ok=True)
    fresh = os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not fresh:
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-Wall", "-Wextra", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.btmt_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_void_p), u64p]
        L.btmt_free.argtypes = [ctypes.c_void_p]
        L.btmt_free.restype = None
        L.btmt_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().btmt_threads())


def build_tree(text, tau: int, leaf_len: int, prune: bool = True, seed: int = 0, nthreads: int = 0) -> bytes:
    a = np.frombuffer(bytes(text), np.uint8) if isinstance(text, (bytes, bytearray)) else np.ascontiguousarray(text)
    out = ctypes.c_void_p()
    n = ctypes.c_uint64()
    rc = lib().btmt_build(a.ctypes.data, len(a), tau, leaf_len, int(bool(prune)), seed, nthreads,
                          ctypes.byref(out), ctypes.byref(n))
    if rc != 0:
        raise RuntimeError(f"btmt_build: error {rc}")
    try:
        return ctypes.string_at(out.value, n.value)
    finally:
        lib().btmt_free(out)
