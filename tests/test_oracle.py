"""Pins of the CPU oracle against things other than itself (no GPU needed).

* the worked example of Figure 1 (tests/golden/fig1_abrainadrain.txt);
* the brute-force builder (definitions of section 3 with bytes.find as the
  leftmost-occurrence search) on thousands of seeded tiny inputs;
* closed forms: a^n, texts without repeated windows, n <= leaf_len;
* access / rank / select against naive counts (section 1);
* invariants every block tree satisfies (pointer targets copy their source,
  lie strictly left, are marked; Lemma 5's bound of 3*z*tau blocks per level);
* independence of the result from the fingerprint base and modulus, including
  a weak modulus that forces fingerprint collisions through the verification;
* fingerprint values (section 2) against identities that fix them.
"""
import os
import random

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_2512_23314_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_fig1():
    text = tau = sizes = None
    trees, cur = {}, None
    for line in open(os.path.join(GOLDEN, "fig1_abrainadrain.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            trees[cur] = {"levels": [], "leaf": None}
            continue
        key, *rest = line.split()
        if key == "text":
            text = rest[0].encode()
        elif key == "tau":
            tau = int(rest[0])
        elif key == "sizes":
            sizes = [int(x) for x in rest]
        elif key == "level":
            b, marks, *ptrs = rest
            trees[cur]["levels"].append(
                (int(b), [int(c) for c in marks], [tuple(map(int, p.split(":"))) for p in ptrs]))
        elif key == "leaf":
            trees[cur]["leaf"] = rest[0].encode()
    return text, tau, sizes, trees


@pytest.mark.parametrize("variant", ["pruned", "unpruned"])
def test_figure1(variant):
    text, tau, sizes, trees = load_fig1()
    want = trees[variant]
    t = oracle.build(text, tau, 1, prune=(variant == "pruned"), level_sizes=sizes)
    got = oracle.parse(t.export())
    assert [(lv.b, lv.marks, lv.ptrs) for lv in got.levels] == want["levels"]
    assert got.leaf_text == want["leaf"]
    b = brute.build(text, tau, 1, prune=(variant == "pruned"), explicit=sizes)
    assert brute.serialize(b) == t.export()
    assert bytes(t.access(i) for i in range(len(text))) == text


def _random_text(rng, n, sigma):
    kind = rng.randrange(4)
    if kind == 0:
        return bytes(rng.randrange(sigma) + 65 for _ in range(n))
    if kind == 1:  # repeats of a short seed with point edits
        seed = [rng.randrange(sigma) + 65 for _ in range(rng.randrange(1, 12))]
        t = [seed[i % len(seed)] for i in range(n)]
        for _ in range(rng.randrange(0, 4)):
            t[rng.randrange(n)] = rng.randrange(sigma) + 65
        return bytes(t)
    if kind == 2:  # runs
        out = []
        while len(out) < n:
            out += [rng.randrange(sigma) + 65] * rng.randrange(1, 9)
        return bytes(out[:n])
    seed = bytes(rng.randrange(sigma) + 65 for _ in range(rng.randrange(4, 40)))
    out = bytearray()
    while len(out) < n:  # copies of a seed with edits
        s = bytearray(seed)
        for _ in range(rng.randrange(0, 3)):
            s[rng.randrange(len(s))] = rng.randrange(sigma) + 65
        out += s
    return bytes(out[:n])


def test_oracle_matches_brute_force_on_tiny_inputs():
    rng = random.Random(12345)
    cases = 0
    for _ in range(2500):
        n = rng.randrange(1, 200)
        sigma = rng.choice([1, 2, 3, 4, 26])
        text = _random_text(rng, n, sigma)
        tau = rng.choice([2, 2, 3, 4, 5])
        leaf = rng.choice([1, 2, 3, 4, 8])
        prune = rng.random() < 0.6
        root = rng.choice([0, 0, 0, 2, 3, 7])
        t = oracle.build(text, tau, leaf, prune=prune, root_arity=root, seed=rng.randrange(1 << 30))
        b = brute.build(text, tau, leaf, prune=prune, root_arity=root)
        assert brute.serialize(b) == t.export(), (text, tau, leaf, prune, root)
        cases += 1
    assert cases == 2500


def test_oracle_matches_brute_force_explicit_sizes():
    rng = random.Random(777)
    for _ in range(600):
        L = rng.randrange(1, 5)
        sizes = [rng.randrange(1, 4)]
        for _ in range(L - 1):
            sizes.insert(0, sizes[0] * rng.randrange(2, 5))
        n = rng.randrange(1, sizes[0] * rng.randrange(1, 6) + 1)
        text = _random_text(rng, n, rng.choice([2, 3, 4]))
        prune = rng.random() < 0.5
        t = oracle.build(text, 3, 1, prune=prune, level_sizes=sizes)
        b = brute.build(text, 3, 1, prune=prune, explicit=sizes)
        assert brute.serialize(b) == t.export(), (text, sizes, prune)


def test_closed_form_unary_text():
    # T = a^n with n = 2*leaf*tau^h: on every level the first pair is the only
    # leftmost pair, so marks are 1 1 0...0 and every pointer is (0, 0).
    for tau, leaf, h in [(2, 4, 5), (3, 2, 4), (4, 8, 3)]:
        n = 2 * leaf * tau ** h
        t = oracle.build(b"a" * n, tau, leaf, prune=False)
        p = oracle.parse(t.export())
        assert len(p.levels) == h + 1
        for l, lv in enumerate(p.levels):
            c = 2 if l == 0 else 2 * tau
            assert lv.marks == [1, 1] + [0] * (c - 2)
            assert lv.ptrs == [(0, 0)] * (c - 2)
        # Pruned: the second block of every non-root level (and of the root)
        # becomes a pointer to (0, 0); only the last level keeps 1 1 0...0.
        t = oracle.build(b"a" * n, tau, leaf, prune=True)
        p = oracle.parse(t.export())
        for l, lv in enumerate(p.levels):
            c = 2 if l == 0 else tau
            if l == len(p.levels) - 1:
                assert lv.marks == [1, 1] + [0] * (c - 2)
            else:
                assert lv.marks == [1] + [0] * (c - 1)
            assert all(x == (0, 0) for x in lv.ptrs)
        assert p.leaf_text == b"a" * (2 * leaf)


def test_closed_form_periodic_text():
    # T = w^m (truncated to n) with |w| dividing leaf_len: every block, pair
    # and tail starts at a multiple of |w|, so its string is a prefix of T and
    # its leftmost occurrence is 0 -- as for a^n.  Marks and pointers (pruned
    # or not) equal those of a^n of the same length; the leaf text is the
    # marked last-level blocks of T.
    rng = random.Random(5)
    for it in range(40):
        leaf = rng.choice([2, 4, 6, 8])
        period = rng.choice([d for d in range(1, leaf + 1) if leaf % d == 0])
        tau = rng.choice([2, 3, 4])
        n = rng.randrange(1, 4000)
        w = bytes(rng.randrange(256) for _ in range(period))
        text = (w * (n // period + 1))[:n]
        for prune in (False, True):
            got = oracle.parse(oracle.build(text, tau, leaf, prune=prune).export())
            unary = oracle.parse(oracle.build(b"a" * n, tau, leaf, prune=prune).export())
            assert [lv.marks for lv in got.levels] == [lv.marks for lv in unary.levels]
            assert [lv.ptrs for lv in got.levels] == [lv.ptrs for lv in unary.levels]
            check_invariants(text, oracle.build(text, tau, leaf, prune=prune).export())


def test_closed_form_no_repeats():
    # Without a repeated window of length leaf_len every block string occurs
    # once, every pair is leftmost and the tree is complete: s*tau^(l-1)
    # blocks on level l, all marked, no pointers, leaf text = T.
    for tau, leaf, h, seed in [(2, 8, 4, 1), (4, 6, 3, 2), (3, 5, 3, 3)]:
        n = 2 * leaf * tau ** h
        text = bytes(workloads.random_bytes(n, 256, seed))
        windows = {text[i:i + leaf] for i in range(n - leaf + 1)}
        assert len(windows) == n - leaf + 1
        for prune in (False, True):
            p = oracle.parse(oracle.build(text, tau, leaf, prune=prune).export())
            for l, lv in enumerate(p.levels):
                assert lv.marks == [1] * (2 * tau ** l)
                assert lv.ptrs == []
            assert p.leaf_text == text


@pytest.mark.parametrize("n", [1, 5, 16])
def test_closed_form_short_text(n):
    text = bytes(range(65, 65 + n))
    p = oracle.parse(oracle.build(text, 4, 16).export())
    assert len(p.levels) == 1
    assert p.levels[0].marks == [1] and p.levels[0].ptrs == [] and p.leaf_text == text


def _naive_select(text, c, j):
    cnt = 0
    for i, x in enumerate(text):
        if x == c:
            cnt += 1
            if cnt == j:
                return i
    return None


def test_queries_against_naive_counts():
    rng = random.Random(99)
    for it in range(60):
        n = rng.randrange(1, 600)
        text = _random_text(rng, n, rng.choice([2, 4, 7]))
        tau, leaf = rng.choice([2, 3, 4]), rng.choice([1, 2, 4, 8])
        t = oracle.build(text, tau, leaf, prune=bool(it % 2))
        assert bytes(t.access(i) for i in range(n)) == text
        for c in set(text) | {0}:
            pref = np.concatenate([[0], np.cumsum(np.frombuffer(text, np.uint8) == c)])
            for i in range(0, n + 1):
                assert t.rank(c, i) == pref[i]
            for j in range(1, int(pref[-1]) + 1):
                assert t.select(c, j) == _naive_select(text, c, j)
    t = oracle.build(b"abcabc", 2, 1)
    for bad in (lambda: t.access(6), lambda: t.rank(97, 7), lambda: t.select(97, 0),
                lambda: t.select(97, 3), lambda: t.select(120, 1)):
        with pytest.raises(oracle.OracleError) as e:
            bad()
        assert e.value.code == oracle.ERANGE
    assert t.rank(120, 6) == 0


def _blocks_of(p):
    """Block starts and lengths per level, rebuilt from the serialization."""
    out = []
    n = p.n
    b0 = p.levels[0].b
    blocks = [(k * b0, min(b0, n - k * b0)) for k in range(-(-n // b0))]
    for l, lv in enumerate(p.levels):
        out.append(blocks)
        if l + 1 < len(p.levels):
            bn = p.levels[l + 1].b
            blocks = [(s + i, min(bn, ln - i)) for (s, ln), m in zip(blocks, lv.marks) if m
                      for i in range(0, ln, bn)]
    return out


def check_invariants(text: bytes, blob: bytes):
    p = oracle.parse(blob)
    per_level = _blocks_of(p)
    for lv, blocks in zip(p.levels, per_level):
        assert len(blocks) == len(lv.marks)
        unmarked = [k for k, m in enumerate(lv.marks) if not m]
        assert len(unmarked) == len(lv.ptrs)
        for u, (j, off) in zip(unmarked, lv.ptrs):
            s, ln = blocks[u]
            ts = blocks[j][0] + off
            assert off < blocks[j][1]
            assert lv.marks[j] == 1
            assert text[ts:ts + ln] == text[s:s + ln]          # copy of the source
            assert ts + ln <= s                                  # strictly left
            if off + ln > blocks[j][1]:                          # crosses into j+1
                assert blocks[j + 1][0] == blocks[j][0] + blocks[j][1] and lv.marks[j + 1]
    last = per_level[-1]
    assert p.leaf_text == b"".join(text[s:s + ln] for (s, ln), m in zip(last, p.levels[-1].marks) if m)


def lz77_phrases(text: bytes) -> int:
    """Greedy LZ77 parse without self-reference (brute force, tiny inputs)."""
    i, z, n = 0, 0, len(text)
    while i < n:
        best = 0
        for j in range(i):
            ln = 0
            while i + ln < n and j + ln < i and text[j + ln] == text[i + ln]:
                ln += 1
            best = max(best, ln)
        i += max(best, 1)
        z += 1
    return z


def test_invariants_and_lemma5_bound():
    rng = random.Random(5)
    for it in range(40):
        n = rng.randrange(50, 400)
        text = _random_text(rng, n, rng.choice([2, 4]))
        tau, leaf = rng.choice([2, 3, 4]), rng.choice([1, 2, 4])
        unpruned = oracle.build(text, tau, leaf, prune=False)
        check_invariants(text, unpruned.export())
        check_invariants(text, oracle.build(text, tau, leaf, prune=True).export())
        z = lz77_phrases(text)
        for st in unpruned.stats()[1:]:
            assert st["nblocks"] <= 3 * z * tau          # Lemma 5


def test_invariants_on_versioned_text():
    text = bytes(workloads.text_versions(n=1 << 16, base_len=1 << 12, sigma=20, seed=3))
    for prune in (False, True):
        t = oracle.build(text, 4, 8, prune=prune)
        check_invariants(text, t.export())
        assert bytes(t.access(i) for i in range(0, len(text), 97)) == text[::97]


def test_independent_of_base_and_modulus():
    rng = random.Random(2024)
    collided = 0
    for it in range(40):
        text = _random_text(rng, rng.randrange(20, 300), 2)
        tau, leaf = rng.choice([2, 3]), rng.choice([1, 2, 3])
        ref = oracle.build(text, tau, leaf, seed=1).export()
        assert oracle.build(text, tau, leaf, seed=99).export() == ref
        weak = oracle.build(text, tau, leaf, seed=7, modulus=331)  # forces collisions
        assert weak.export() == ref
        collided += sum(s["collisions"] for s in weak.stats())
    assert collided > 0


def test_fingerprint_values():
    text = bytes(workloads.random_bytes(300, 256, 4))
    q = (1 << 61) - 1
    B = oracle.base(5)
    assert 256 <= B < q
    # single symbol: phi = T[i] + 1 (symbols are byte + 1)
    assert all(oracle.fingerprint(text, i, 1, B) == text[i] + 1 for i in range(50))
    # empty string
    assert oracle.fingerprint(text, 3, 0, B) == 0
    # concatenation: phi(xy) = phi(x) * B^|y| + phi(y)
    for s, a, b in [(0, 10, 20), (5, 1, 100), (17, 64, 64), (0, 150, 150)]:
        fx = oracle.fingerprint(text, s, a, B)
        fy = oracle.fingerprint(text, s + a, b, B)
        assert oracle.fingerprint(text, s, a + b, B) == (fx * pow(B, b, q) + fy) % q
    # base 1 modulo a prime larger than the sum: phi is the plain symbol sum
    # (base() never returns 1, so call the Horner with an explicit base).
    assert oracle.fingerprint(text, 0, 300, 1) == sum(x + 1 for x in text)
    # rolling relation of section 4.3: phi(s..e) from phi(s-1..e-1)
    L = 37
    for s in range(1, 60):
        prev = oracle.fingerprint(text, s - 1, L, B)
        roll = (prev * B - (text[s - 1] + 1) * pow(B, L, q) + text[s + L - 1] + 1) % q
        assert oracle.fingerprint(text, s, L, B) == roll
    # a weak modulus reduces the same polynomial
    assert oracle.fingerprint(text, 0, 40, 300, 331) == \
        sum((x + 1) * pow(300, 39 - i, 331) for i, x in enumerate(text[:40])) % 331


def test_invalid_arguments():
    for args in [(b"", 2, 4), (b"abc", 1, 4), (b"abc", 2, 0)]:
        with pytest.raises(oracle.OracleError) as e:
            oracle.build(*args)
        assert e.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError):
        oracle.build(b"abcdef", 2, 1, level_sizes=[3, 2, 1])  # 3 is not a multiple of 2


def test_config1_shape():
    # The 1 MiB DNA workload: 16 levels of 2^19 ... 2^4, bit-exact with itself
    # under a second seed, valid pointers, and access spot checks.
    text = workloads.dna_copies()
    t = oracle.build(text, 2, 16, prune=True, seed=1)
    st = t.stats()
    assert [s["b"] for s in st] == [1 << (19 - l) for l in range(16)]
    assert st[0]["nblocks"] == 2 and st[0]["cov"] == 1 << 20
    tb = bytes(text)
    check_invariants(tb, t.export())
    idx = np.random.default_rng(0).integers(0, len(tb), 2000)
    assert bytes(t.access(int(i)) for i in idx) == bytes(tb[int(i)] for i in idx)
