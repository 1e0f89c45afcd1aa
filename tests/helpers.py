"""Shared test helpers: tree structure rebuilt from the canonical serialization,
and properties every block tree must satisfy (checked at any size)."""
from __future__ import annotations

import numpy as np

import oracle


def level_blocks(p: "oracle.Parsed"):
    """Per level: (starts, lengths) numpy arrays, rebuilt from the marks."""
    out = []
    n = p.n
    b0 = p.levels[0].b
    st = np.arange(0, n, b0, dtype=np.int64)
    for l, lv in enumerate(p.levels):
        ln = np.minimum(lv.b, n - st)
        out.append((st, ln))
        if l + 1 < len(p.levels):
            bn = p.levels[l + 1].b
            m = np.asarray(lv.marks, dtype=bool)
            ps, pl = st[m], ln[m]
            nch = (pl + bn - 1) // bn
            par = np.repeat(np.arange(len(ps)), nch)
            first = np.repeat(np.cumsum(nch) - nch, nch)
            idx = np.arange(nch.sum()) - first
            st = ps[par] + idx * bn
    return out


def check_pointers(T: np.ndarray, blob: bytes, sample: int | None = None, seed: int = 0):
    """Every (or a sample of) pointer copies its source, lies strictly left,
    targets marked blocks; the leaf text equals the marked last-level blocks."""
    p = oracle.parse(blob, as_numpy=True)
    rng = np.random.default_rng(seed)
    blocks = level_blocks(p)
    for lv, (st, ln) in zip(p.levels, blocks):
        marks = np.asarray(lv.marks, dtype=bool)
        assert len(marks) == len(st)
        un = np.flatnonzero(~marks)
        assert len(un) == len(lv.ptrs)
        if len(un) == 0:
            continue
        pa = np.asarray(lv.ptrs, dtype=np.int64).reshape(-1, 2)
        pick = np.arange(len(un)) if sample is None or sample >= len(un) else \
            rng.choice(len(un), sample, replace=False)
        for i in pick:
            u = un[i]
            j, off = pa[i]
            s, L = st[u], ln[u]
            tgt = st[j] + off
            assert marks[j] and off < ln[j]
            assert tgt + L <= s
            if off + L > ln[j]:
                assert st[j + 1] == st[j] + ln[j] and marks[j + 1]
            assert np.array_equal(T[tgt:tgt + L], T[s:s + L])
    st, ln = blocks[-1]
    m = np.asarray(p.levels[-1].marks, dtype=bool)
    if sample is None:
        leaf = np.concatenate([T[a:a + b] for a, b in zip(st[m], ln[m])]) if m.any() else \
            np.zeros(0, np.uint8)
        assert bytes(leaf) == p.leaf_text
    return p, blocks


def check_leftmost_sampled(T: np.ndarray, p, blocks, per_level: int = 20, seed: int = 1):
    """The definition on samples: an unmarked block points to T.find(its
    string); a pair is leftmost iff T.find(pair string) is its start."""
    Tb = T.tobytes()
    rng = np.random.default_rng(seed)
    for lv, (st, ln) in zip(p.levels, blocks):
        marks = np.asarray(lv.marks, dtype=bool)
        un = np.flatnonzero(~marks)
        pa = np.asarray(lv.ptrs, dtype=np.int64).reshape(-1, 2)
        for i in (rng.choice(len(un), min(per_level, len(un)), replace=False) if len(un) else []):
            u = un[i]
            j, off = pa[i]
            s, L = int(st[u]), int(ln[u])
            assert Tb.find(Tb[s:s + L]) == st[j] + off
        c = len(st)
        if c < 2:
            continue
        for k in rng.choice(c - 1, min(per_level, c - 1), replace=False):
            if st[k + 1] != st[k] + ln[k]:
                continue
            s, L = int(st[k]), int(ln[k] + ln[k + 1])
            if Tb.find(Tb[s:s + L]) == s:
                assert marks[k] and marks[k + 1] or p.prune  # pruning may unmark
