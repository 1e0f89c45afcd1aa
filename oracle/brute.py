"""Brute-force block tree -- the definitions of section 3 written out, for tiny inputs.

TEST INFRASTRUCTURE ONLY.  No fingerprints, no hash tables: the leftmost
occurrence LO(x) of a string x is ``T.find(x)``, the lowest index at which x
occurs in T.  Everything else is a direct, quadratic restatement of:

* section 3: level 1 splits T into blocks of length b_1; a pair of blocks
  consecutive in T whose string occurs leftmost at the pair's own start marks
  both blocks; marked blocks get children of the next block size; an unmarked
  block points to the level block holding the leftmost occurrence of its
  string, with an offset;
* section 3.1, "Optional Pruning", under the reading stated in ``bt_oracle.c``;
* the canonical serialization described in ``bt_oracle.c``.

It shares no code with the C oracle: it is the independent builder the C
oracle is checked against.
"""
from __future__ import annotations

import struct


def level_sizes(n: int, tau: int, leaf: int, root_arity: int = 0, explicit=None) -> list[int]:
    if explicit is not None:
        return [int(x) for x in explicit]
    s0 = root_arity or tau
    h = 0
    while s0 * leaf * tau ** h < n:
        h += 1
    return [leaf * tau ** (h - l) for l in range(h + 1)]


def _containing(blocks, p):
    for j, (s, ln) in enumerate(blocks):
        if s <= p < s + ln:
            return j
    return None


def build(text: bytes, tau: int, leaf: int, prune: bool = True, root_arity: int = 0,
          explicit=None) -> dict:
    T = bytes(text)
    n = len(T)
    bs = level_sizes(n, tau, leaf, root_arity, explicit)
    L = len(bs)
    levels = []
    blocks = [(k * bs[0], min(bs[0], n - k * bs[0])) for k in range(-(-n // bs[0]))]
    for l in range(L):
        c = len(blocks)
        S = [T[s:s + ln] for s, ln in blocks]
        consecutive = [blocks[k][0] + blocks[k][1] == blocks[k + 1][0] for k in range(c - 1)]
        pair_leftmost = [consecutive[k] and T.find(S[k] + S[k + 1]) == blocks[k][0]
                         for k in range(c - 1)]
        marks = []
        for k in range(c):
            in_left = k > 0 and consecutive[k - 1]
            in_right = k < c - 1 and consecutive[k]
            marked = (k > 0 and pair_leftmost[k - 1]) or (k < c - 1 and pair_leftmost[k])
            marks.append(bool(marked or (not in_left and not in_right)))
        lo = [T.find(S[k]) for k in range(c)]
        ptrs = {}
        for u in range(c):
            if not marks[u]:
                j = _containing(blocks, lo[u])
                ptrs[u] = (j, lo[u] - blocks[j][0])
        levels.append({"b": bs[l], "blocks": list(blocks), "marks": marks, "ptrs": ptrs, "lo": lo})
        if l + 1 < L:
            bn = bs[l + 1]
            blocks = [(s + i, min(bn, ln - i)) for (s, ln), m in zip(blocks, marks) if m
                      for i in range(0, ln, bn)]
    if prune:
        _prune(levels)
    last = levels[-1]
    leaf_text = b"".join(T[s:s + ln] for (s, ln), m in zip(last["blocks"], last["marks"]) if m)
    return {"n": n, "tau": tau, "leaf": leaf, "prune": int(bool(prune)), "levels": levels,
            "leaf_text": leaf_text}


def _children(levels, l, k):
    """Indices on level l+1 of the children of block k of level l."""
    s, ln = levels[l]["blocks"][k]
    return [i for i, (cs, cl) in enumerate(levels[l + 1]["blocks"]) if s <= cs < s + ln]


def _window_blocks(blocks, p, length):
    return [j for j, (s, ln) in enumerate(blocks) if s < p + length and p < s + ln]


def _prune(levels):
    L = len(levels)
    for l in range(L - 2, -1, -1):
        v, w = levels[l], levels[l + 1]
        # Targets of the next level's pointers, as they stand before this
        # level's pass (a child deleted during the pass keeps protecting the
        # target of its pointer).
        next_targets = set()
        for u, (j, off) in w["ptrs"].items():
            p = w["blocks"][j][0] + off
            next_targets |= {w["blocks"][x][0]
                             for x in _window_blocks(w["blocks"], p, w["blocks"][u][1])}
        for k in range(len(v["blocks"]) - 1, -1, -1):
            if not v["marks"][k]:
                continue
            s, ln = v["blocks"][k]
            kids = _children(levels, l, k)
            # (i) no child has children
            if l + 1 < L - 1 and any(w["marks"][c] for c in kids):
                continue
            # (ii) no pointer of this level has a target window overlapping k
            hit = False
            for u, (j, off) in v["ptrs"].items():
                p = v["blocks"][j][0] + off
                if k in _window_blocks(v["blocks"], p, v["blocks"][u][1]):
                    hit = True
            if hit:
                continue
            # (iii) no pointer of the next level targets a child of k
            if any(w["blocks"][c][0] in next_targets for c in kids):
                continue
            # (iv) an earlier occurrence that does not overlap k
            if v["lo"][k] + ln > s:
                continue
            j = _containing(v["blocks"], v["lo"][k])
            v["marks"][k] = False
            v["ptrs"][k] = (j, v["lo"][k] - v["blocks"][j][0])
            keep = [i for i in range(len(w["blocks"])) if i not in set(kids)]
            new_index = {old: new for new, old in enumerate(keep)}
            w["blocks"] = [w["blocks"][i] for i in keep]
            w["marks"] = [w["marks"][i] for i in keep]
            w["lo"] = [w["lo"][i] for i in keep]
            w["ptrs"] = {new_index[u]: (new_index[j], off) for u, (j, off) in w["ptrs"].items()
                         if u in new_index}


def serialize(tree: dict) -> bytes:
    out = [struct.pack("<6Q", 0x31454552544B4C42, tree["n"], tree["tau"], tree["leaf"],
                       len(tree["levels"]), tree["prune"])]
    for v in tree["levels"]:
        c = len(v["blocks"])
        out.append(struct.pack("<2Q", c, v["b"]))
        for k0 in range(0, c, 64):
            word = sum(1 << (k - k0) for k in range(k0, min(c, k0 + 64)) if v["marks"][k])
            out.append(struct.pack("<Q", word))
        ptrs = sorted(v["ptrs"].items())
        out.append(struct.pack("<Q", len(ptrs)))
        for _, (j, off) in ptrs:
            out.append(struct.pack("<2Q", j, off))
    lt = tree["leaf_text"]
    out.append(struct.pack("<Q", len(lt)))
    out.append(lt + b"\0" * (-len(lt) % 8))
    return b"".join(out)


def access(tree: dict, i: int) -> int:
    """Follow the tree from the root to the leaf text (section 1, access)."""
    levels = tree["levels"]
    l = 0
    v = levels[0]
    k = _containing(v["blocks"], i)
    x = i
    for _ in range(4 * len(levels) + 4):
        v = levels[l]
        s, ln = v["blocks"][k]
        if v["marks"][k]:
            if l == len(levels) - 1:
                pos = 0
                for (bs_, bl), m in zip(v["blocks"][:k], v["marks"][:k]):
                    pos += bl if m else 0
                return tree["leaf_text"][pos + x - s]
            l += 1
            k = _containing(levels[l]["blocks"], x)
        else:
            j, off = v["ptrs"][k]
            x = v["blocks"][j][0] + off + (x - s)
            k = _containing(v["blocks"], x)
    raise RuntimeError("access did not terminate")
