"""Seeded synthetic texts shaped like the paper's repetitive inputs.

This module holds only input generation: no fingerprint, no block-tree
arithmetic.  Both the CUDA path and the CPU oracle are fed from it.

The paper evaluates on the Pizza&Chili repetitive corpus (section 5, Table 1:
DNA collections with sigma 5-15, versioned source code and wiki text with
sigma 89-236, average LZ77 phrase lengths 55-5227).  That corpus is not
available here; these generators stand in for it with the same shapes:

* ``dna_copies``     -- a random DNA seed string copied many times with point
                        substitutions (1 MiB, 16 copies of 64 KiB, 0.1 %);
* ``text_versions``  -- a Zipf(1.1) text over 96 printable symbols followed by
                        versions that each apply 0.05 % random edit runs
                        (substitute / insert / delete, 1-32 bytes) to the
                        previous version (256 MiB from a 4 MiB base);
* ``dna_genome``     -- a random genome over ACGT copied 64 times with 0.1 %
                        SNPs, 0.01 % indels of length 1-50 and rare N runs
                        (2 GiB from a 32 MiB genome);
* ``doc_mix``        -- many short documents of log-uniform length, each a
                        scaled-down versioned text with its own alphabet size.

Every generator takes a seed and is deterministic for a given numpy version
(numpy's PCG64 bit generator).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def zipf_alphabet(sigma: int) -> np.ndarray:
    """Byte values of a sigma-symbol alphabet: printable from 0x20 when it fits."""
    first = 0x20 if sigma <= 96 else 0x00
    return (first + np.arange(sigma)).astype(np.uint8)


def zipf_bytes(rng: np.random.Generator, count: int, sigma: int, s: float = 1.1) -> np.ndarray:
    """`count` symbols; the symbol of rank k has probability proportional to k^-s."""
    k = np.arange(1, sigma + 1, dtype=np.float64)
    p = k ** -s
    p /= p.sum()
    return zipf_alphabet(sigma)[rng.choice(sigma, size=count, p=p)]


def dna_copies(n: int = 1 << 20, seed_len: int = 1 << 16, sub_rate: float = 1e-3,
               seed: int = 0xB7EE0001) -> np.ndarray:
    """A uniform ACGT seed string of `seed_len` bytes, copied until `n` bytes;
    each position of each copy is replaced, with probability `sub_rate`, by a
    uniformly chosen different base."""
    rng = _rng(seed)
    base = rng.integers(0, 4, seed_len, dtype=np.uint8)
    reps = -(-n // seed_len)
    codes = np.tile(base, reps)[:n]
    hit = rng.random(n) < sub_rate
    shift = rng.integers(1, 4, n, dtype=np.uint8)
    codes[hit] = (codes[hit] + shift[hit]) % 4
    return ACGT[codes]


def _apply_edits(rng, v: np.ndarray, m: int, max_run: int, draw) -> np.ndarray:
    """Apply `m` edits at sorted uniform positions of `v`.  Each edit is a
    substitution, insertion or deletion (equally likely) of a run of
    U[1, max_run] bytes; new bytes come from `draw(count)`.  An edit whose
    position falls inside the run of the previous edit is dropped."""
    if m == 0 or len(v) == 0:
        return v.copy()
    pos = np.sort(rng.integers(0, len(v), m))
    kind = rng.integers(0, 3, m)
    run = rng.integers(1, max_run + 1, m)
    pool = draw(int(run.sum()))
    used = 0
    pieces = []
    cur = 0
    for p, k, r in zip(pos.tolist(), kind.tolist(), run.tolist()):
        if p < cur:
            continue
        pieces.append(v[cur:p])
        if k == 0:  # substitute
            r = min(r, len(v) - p)
            pieces.append(pool[used:used + r])
            used += r
            cur = p + r
        elif k == 1:  # insert before p
            pieces.append(pool[used:used + r])
            used += r
            cur = p
        else:  # delete
            cur = min(len(v), p + r)
    pieces.append(v[cur:])
    return np.concatenate(pieces)


def text_versions(n: int = 1 << 28, base_len: int = 4 << 20, sigma: int = 96,
                  edit_rate: float = 5e-4, max_run: int = 32, zipf_s: float = 1.1,
                  seed: int = 0xB7EE0002) -> np.ndarray:
    """Version 0 is a Zipf text of `base_len` bytes; version t+1 applies
    round(edit_rate * |v_t|) edit runs to version t.  The versions are
    concatenated until `n` bytes are reached."""
    rng = _rng(seed)
    draw = lambda c: zipf_bytes(rng, c, sigma, zipf_s)  # noqa: E731
    v = draw(base_len)
    parts = [v]
    total = len(v)
    while total < n:
        v = _apply_edits(rng, v, int(round(edit_rate * len(v))), max_run, draw)
        parts.append(v)
        total += len(v)
    return np.concatenate(parts)[:n]


def dna_genome(n: int = 1 << 31, genome_len: int = 32 << 20,
               snp_rate: float = 1e-3, indel_rate: float = 1e-4, indel_max: int = 50,
               nrun_rate: float = 1e-6, nrun_max: int = 20, seed: int = 0xB7EE0003) -> np.ndarray:
    """A uniform ACGT genome; every copy gets SNPs (a different base), indels
    (insertion or deletion, 50/50, of U[1, indel_max] random bases) and runs of
    'N' (start probability `nrun_rate`, length U[1, nrun_max]).  Copies are
    concatenated until `n` bytes (64 copies for the 2 GiB default)."""
    rng = _rng(seed)
    genome = rng.integers(0, 4, genome_len, dtype=np.uint8)
    out = np.empty(n, dtype=np.uint8)
    filled = 0
    while filled < n:
        g = genome.copy()
        hit = np.flatnonzero(rng.random(genome_len) < snp_rate)
        g[hit] = (g[hit] + rng.integers(1, 4, len(hit), dtype=np.uint8)) % 4
        s = ACGT[g]
        m_ind = rng.binomial(genome_len, indel_rate)
        pos = np.sort(rng.integers(0, genome_len, m_ind))
        ins = rng.random(m_ind) < 0.5
        ln = rng.integers(1, indel_max + 1, m_ind)
        pool = ACGT[rng.integers(0, 4, int(ln.sum()), dtype=np.uint8)]
        pieces, cur, used = [], 0, 0
        for p, is_ins, r in zip(pos.tolist(), ins.tolist(), ln.tolist()):
            if p < cur:
                continue
            pieces.append(s[cur:p])
            if is_ins:
                pieces.append(pool[used:used + r])
                used += r
                cur = p
            else:
                cur = min(len(s), p + r)
        pieces.append(s[cur:])
        s = np.concatenate(pieces)
        m_n = rng.binomial(len(s), nrun_rate)
        for p, r in zip(rng.integers(0, len(s), m_n).tolist(),
                        rng.integers(1, nrun_max + 1, m_n).tolist()):
            s[p:p + r] = ord("N")
        take = min(len(s), n - filled)
        out[filled:filled + take] = s[:take]
        filled += take
    return out


def random_bytes(n: int, sigma: int = 256, seed: int = 1) -> np.ndarray:
    """Uniform bytes over the first `sigma` byte values."""
    return _rng(seed).integers(0, sigma, n, dtype=np.uint8)


@dataclass
class Doc:
    text: np.ndarray
    sigma: int
    tau: int
    leaf_len: int


def doc_mix(ndocs: int, min_len: int = 4 << 10, max_len: int = 16 << 20,
            taus=(2, 4, 8), sigma_range=(4, 128), leaf_len: int = 32,
            seed: int = 0xB7EE0004) -> list[Doc]:
    """`ndocs` documents with log-uniform lengths in [min_len, max_len]; each
    is a versioned text (base = max(1 KiB, len/16)) with its own seed, an
    alphabet size uniform in `sigma_range` and tau drawn from `taus`."""
    rng = _rng(seed)
    docs = []
    for d in range(ndocs):
        u = rng.random()
        length = int(np.floor(np.exp(u * np.log(max_len / min_len)) * min_len))
        sigma = int(rng.integers(sigma_range[0], sigma_range[1] + 1))
        tau = int(rng.choice(taus))
        t = text_versions(n=length, base_len=max(1024, length // 16), sigma=sigma,
                          seed=int(rng.integers(0, 2**62)))
        docs.append(Doc(t, sigma, tau, leaf_len))
    return docs


@dataclass
class Arrival:
    t: float          # arrival time in seconds from the start
    doc: Doc


def serve_arrivals(rate: float = 2000.0, duration: float = 10.0, min_len: int = 1 << 10,
                   max_len: int = 64 << 20, seed: int = 0xB7EE0005) -> list[Arrival]:
    """Poisson arrivals (exponential gaps at `rate` per second) over
    `duration` seconds.  Each document has a log-uniform length in
    [min_len, max_len] and is, with equal probability, DNA-like (a random
    genome of len/16 bases copied with SNPs, indels and N runs; tau 4,
    leaf 64) or text-like (a Zipf text of len/16 bytes in versions; tau 4,
    leaf 32)."""
    rng = _rng(seed)
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        u = rng.random()
        length = int(np.floor(np.exp(u * np.log(max_len / min_len)) * min_len))
        s = int(rng.integers(0, 2**62))
        if rng.random() < 0.5:
            text = dna_genome(n=length, genome_len=max(1024, length // 16), seed=s)
            out.append(Arrival(t, Doc(text, 5, 4, 64)))
        else:
            text = text_versions(n=length, base_len=max(1024, length // 16), sigma=96, seed=s)
            out.append(Arrival(t, Doc(text, 96, 4, 32)))
    return out
