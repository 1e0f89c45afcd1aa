"""The C ABI library builds, loads and exports every entry point of include/bt.h.

No compute call runs here: without a GPU the only call made is one that must
fail loudly (BT_ECUDA), never fall back to the CPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(bt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bt_build", "bt_build_ex", "bt_access", "bt_rank", "bt_select",
                     "bt_query_batch", "bt_export", "bt_free", "bt_strerror"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_2512_23314_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(bt_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2512_23314_gb300 import bt
    with pytest.raises(bt.BTError) as e:
        bt.Tree(b"abracadabra", 5, 2, 2)
    assert e.value.code == bt.BT_ECUDA


def test_export_into_checks_its_buffer_before_the_library():
    # The binding rejects a buffer it cannot hand to bt_export as plain host
    # bytes, before any library call.
    import torch

    from paper_2512_23314_gb300 import bt
    with pytest.raises(TypeError):
        bt.bt_export_into(1, torch.zeros(16, dtype=torch.int32))
    with pytest.raises(TypeError):
        bt.bt_export_into(1, torch.zeros(16, 2, dtype=torch.uint8).t())
