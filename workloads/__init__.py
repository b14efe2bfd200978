"""Seeded synthetic inputs for the SFA matcher: DFA tables and texts.

This module only *produces inputs*.  It contains no part of the matching
method (no SFA construction, no composition, no run of an automaton over a
text): both the CPU oracle (``oracle/``) and the CUDA path consume what it
returns, and neither of them is imported here.

Every DFA is returned as a :class:`DFA`: a total transition table over the
256 byte values (``delta[q, b]``, int32), an initial state ``q0`` and an
accept vector.  Bytes outside an automaton's alphabet go to the state the
construction documents (a dead state for the regular-expression automata of
Sect. VI, the root for the literal automata, column 0 for the random ones).

Randomness: numpy ``Generator`` objects seeded from an integer seed.  Large
texts are produced in fixed 16 MiB blocks, each from its own Philox stream
keyed by (seed, block index), so the bytes do not depend on the number of
worker threads.
"""
from __future__ import annotations

import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor
from typing import List, Optional, Sequence

import numpy as np

BASE64_ALPHABET = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
LOWER_ALPHABET = b"abcdefghijklmnopqrstuvwxyz"

_BLOCK = 16 << 20  # bytes per independently seeded text block


@dataclasses.dataclass
class DFA:
    """A complete DFA over bytes (Sect. II-B: |I| = 1, singleton images)."""

    delta: np.ndarray            # int32 [nq, 256]
    q0: int
    accept: np.ndarray           # uint8 [nq], 0/1
    alphabet: bytes              # the symbols the automaton is defined over
    name: str = ""
    literals: Optional[List[bytes]] = None      # literal automata only
    state_strings: Optional[List[bytes]] = None  # literal automata: trie path of each state
    dead: Optional[int] = None   # id of the sink state, if the automaton has one

    @property
    def nq(self) -> int:
        return int(self.delta.shape[0])


def _check(d: DFA) -> DFA:
    assert d.delta.dtype == np.int32 and d.delta.ndim == 2 and d.delta.shape[1] == 256
    assert d.delta.min() >= 0 and d.delta.max() < d.nq
    assert 0 <= d.q0 < d.nq
    d.accept = np.ascontiguousarray(d.accept, dtype=np.uint8)
    d.delta = np.ascontiguousarray(d.delta)
    return d


# ---------------------------------------------------------------------------
# Automata of the paper's examples and experiments
# ---------------------------------------------------------------------------

def dfa_ab_star() -> DFA:
    """D1 of Example 1: L(D1) = (ab)*; states 0, 1, 2 with 0 initial and final,
    0 -a-> 1, 1 -b-> 0, every other transition into the dead state 2."""
    delta = np.full((3, 256), 2, dtype=np.int32)
    delta[0, ord("a")] = 1
    delta[1, ord("b")] = 0
    acc = np.array([1, 0, 0], dtype=np.uint8)
    return _check(DFA(delta, 0, acc, b"ab", name="ab_star", dead=2))


def dfa_rn(n: int) -> DFA:
    """Minimal DFA of r_n = ([0-4]{n}[5-9]{n})* (Sect. VI-B): a loop of 2n
    states (state i < n expects [0-4], state i >= n expects [5-9]) plus a
    dead state 2n.  State 0 is initial and the only final state."""
    k = 2 * n
    dead = k
    delta = np.full((k + 1, 256), dead, dtype=np.int32)
    for i in range(k):
        digits = b"01234" if i < n else b"56789"
        for c in digits:
            delta[i, c] = (i + 1) % k
    acc = np.zeros(k + 1, dtype=np.uint8)
    acc[0] = 1
    return _check(DFA(delta, 0, acc, b"0123456789", name=f"r_{n}", dead=dead))


def dfa_ra(n: int) -> DFA:
    """Minimal DFA of r_n | a* (the r_a workload of Sect. VI-B, there with
    n = 500): the r_n loop plus a start state that also accepts runs of 'a'.

    States: 0 = start (accepting: the empty word is in both branches),
    1 .. 2n-1 = the loop positions after the first digit, 2n = 'a'-run state
    (accepting), 2n+1 = dead.  Reading a full loop from the start returns to
    loop position 0, which is represented by a separate accepting state
    ``loop0`` = 2n+2 (it differs from the start state because 'a' kills it)."""
    k = 2 * n
    start, arun, dead, loop0 = 0, k, k + 1, k + 2
    nq = k + 3
    delta = np.full((nq, 256), dead, dtype=np.int32)

    def loop_id(pos: int) -> int:  # pos in [0, k)
        return loop0 if pos == 0 else pos

    for src, pos in [(start, 0), (loop0, 0)] + [(i, i) for i in range(1, k)]:
        digits = b"01234" if pos < n else b"56789"
        for c in digits:
            delta[src, c] = loop_id((pos + 1) % k)
    delta[start, ord("a")] = arun
    delta[arun, ord("a")] = arun
    acc = np.zeros(nq, dtype=np.uint8)
    acc[[start, arun, loop0]] = 1
    return _check(DFA(delta, 0, acc, b"0123456789a", name=f"r_a{n}", dead=dead))


def dfa_even_odd(reps: int = 5) -> DFA:
    """Minimal DFA of (([02468][13579]){reps})* (Sect. VI-C, reps = 5):
    a loop of 2*reps states alternating even/odd digits plus a dead state."""
    k = 2 * reps
    dead = k
    delta = np.full((k + 1, 256), dead, dtype=np.int32)
    for i in range(k):
        digits = b"02468" if i % 2 == 0 else b"13579"
        for c in digits:
            delta[i, c] = (i + 1) % k
    acc = np.zeros(k + 1, dtype=np.uint8)
    acc[0] = 1
    return _check(DFA(delta, 0, acc, b"0123456789", name=f"even_odd{reps}", dead=dead))


def dfa_full_transformation(n: int) -> DFA:
    """A DFA whose letters generate the full transformation monoid T_n
    (the situation of Example 5 / Fact 2, where |S_d| = |D|^|D|).

    Letters: 'c' the cycle q -> q+1 mod n, 't' the transposition of 0 and 1,
    'm' the rank n-1 map sending n-1 to 0 and fixing the rest.  A cycle, a
    transposition and one idempotent of rank n-1 generate T_n (a textbook
    fact about transformation semigroups).  Every other byte acts as the
    identity.  State 0 is initial and final."""
    assert n >= 2
    delta = np.tile(np.arange(n, dtype=np.int32)[:, None], (1, 256))
    for q in range(n):
        delta[q, ord("c")] = (q + 1) % n
        delta[q, ord("t")] = {0: 1, 1: 0}.get(q, q)
        delta[q, ord("m")] = 0 if q == n - 1 else q
    acc = np.zeros(n, dtype=np.uint8)
    acc[0] = 1
    return _check(DFA(delta, 0, acc, b"cmt", name=f"full_T{n}"))


# ---------------------------------------------------------------------------
# Literal automata (KMP, Aho-Corasick): non-absorbing, every occurrence ends
# in an accepting state
# ---------------------------------------------------------------------------

def dfa_kmp(literal: bytes) -> DFA:
    """KMP automaton of one literal over the byte alphabet, non-absorbing.

    State j (0 <= j <= m) = length of the longest prefix of the literal that
    is a suffix of the text read so far; state m is the only final state.
    Built with the classic restart-state recurrence."""
    m = len(literal)
    assert m >= 1
    delta = np.zeros((m + 1, 256), dtype=np.int32)
    delta[0, literal[0]] = 1
    restart = 0
    for j in range(1, m + 1):
        delta[j, :] = delta[restart, :]
        if j < m:
            delta[j, literal[j]] = j + 1
            restart = int(delta[restart, literal[j]])
    acc = np.zeros(m + 1, dtype=np.uint8)
    acc[m] = 1
    strings = [literal[:j] for j in range(m + 1)]
    return _check(DFA(delta, 0, acc, bytes(sorted(set(literal))), name="kmp",
                      literals=[literal], state_strings=strings))


def dfa_aho_corasick(literals: Sequence[bytes]) -> DFA:
    """Aho-Corasick automaton (goto + failure completed into a DFA) of a
    literal set, over the byte alphabet, non-absorbing.

    A state is a trie node; its string is the path from the root.  After a
    text w the automaton is in the node of the longest suffix of w that is a
    prefix of some literal; a node is final when some literal is a suffix of
    its string."""
    lits = [bytes(l) for l in literals]
    assert lits and all(len(l) >= 1 for l in lits)
    children: List[dict] = [{}]
    strings: List[bytes] = [b""]
    for lit in lits:
        s = 0
        for c in lit:
            nxt = children[s].get(c)
            if nxt is None:
                nxt = len(children)
                children[s][c] = nxt
                children.append({})
                strings.append(strings[s] + bytes([c]))
            s = nxt
    nq = len(children)
    litset = set(lits)
    acc = np.zeros(nq, dtype=np.uint8)
    for s, st in enumerate(strings):
        acc[s] = any(st[i:] in litset for i in range(len(st)))
    delta = np.zeros((nq, 256), dtype=np.int32)
    fail = [0] * nq
    order = []
    queue = [0]
    while queue:
        s = queue.pop(0)
        order.append(s)
        queue.extend(children[s][c] for c in sorted(children[s]))
    for s in order:  # BFS order: fail[s] and its row are final before s
        if s == 0:
            row = np.zeros(256, dtype=np.int32)
        else:
            row = delta[fail[s]].copy()
        for c, t in children[s].items():
            row[c] = t
            fail[t] = 0 if s == 0 else int(delta[fail[s], c])
        delta[s] = row
    alpha = bytes(sorted(set(b"".join(lits))))
    return _check(DFA(delta, 0, acc, alpha, name="aho_corasick", literals=lits,
                      state_strings=strings))


def random_literals(count: int, min_len: int, max_len: int, alphabet: bytes,
                    seed: int) -> List[bytes]:
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    out = []
    for _ in range(count):
        ln = int(rng.integers(min_len, max_len + 1))
        out.append(bytes(alpha[rng.integers(0, len(alpha), size=ln)].tolist()))
    return out


def literal_set_automaton(seed: int, alphabet: bytes = LOWER_ALPHABET,
                          min_states: int = 8, max_states: int = 200) -> DFA:
    """An Aho-Corasick automaton of a seeded literal set whose size lands in
    [min_states, max_states]; literal sets are redrawn until it does."""
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        count = int(rng.integers(1, 31))
        lits = random_literals(count, 3, 9, alphabet, int(rng.integers(0, 2**62)))
        d = dfa_aho_corasick(lits)
        if min_states <= d.nq <= max_states:
            d.name = f"ac_set_{seed}"
            return d


def dfa_random(nq: int, nsym: int, seed: int, p_accept: float = 0.5) -> DFA:
    """Uniformly random complete DFA with nq states over symbols 0..nsym-1;
    each state is final with probability p_accept, q0 = 0.  Bytes >= nsym
    copy the column of symbol 0 (texts for it never contain them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    delta = np.empty((nq, 256), dtype=np.int32)
    delta[:, :nsym] = rng.integers(0, nq, size=(nq, nsym), dtype=np.int32)
    delta[:, nsym:] = delta[:, :1]
    acc = (rng.random(nq) < p_accept).astype(np.uint8)
    return _check(DFA(delta, 0, acc, bytes(range(nsym)), name=f"random_{nq}x{nsym}"))


# ---------------------------------------------------------------------------
# Texts
# ---------------------------------------------------------------------------

def _blocks(n: int):
    return [(i, i * _BLOCK, min(n, (i + 1) * _BLOCK)) for i in range((n + _BLOCK - 1) // _BLOCK)]


def _fill_parallel(n: int, seed: int, fn, threads: int = 8) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)

    def work(b):
        i, lo, hi = b
        rng = np.random.Generator(np.random.Philox(key=seed, counter=[0, 0, i, 0]))
        out[lo:hi] = fn(rng, hi - lo)

    blocks = _blocks(n)
    if len(blocks) <= 1:
        for b in blocks:
            work(b)
    else:
        with ThreadPoolExecutor(min(threads, len(blocks))) as ex:
            list(ex.map(work, blocks))
    return out


def text_uniform(n: int, alphabet: bytes, seed: int) -> np.ndarray:
    """n bytes drawn uniformly from `alphabet` (exactly uniform: bounded
    integers, not a quantised table)."""
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    m = len(alpha)
    if m == 256:
        return _fill_parallel(n, seed, lambda r, k: np.frombuffer(r.bytes(k), dtype=np.uint8))
    if m & (m - 1) == 0 and alpha.tolist() == list(range(m)):
        mask = m - 1
        return _fill_parallel(n, seed, lambda r, k: np.frombuffer(r.bytes(k), dtype=np.uint8) & mask)
    return _fill_parallel(n, seed, lambda r, k: alpha[r.integers(0, m, size=k, dtype=np.uint8)])


def text_rn_accepted(n: int, rn: int, seed: int) -> np.ndarray:
    """n bytes of an r_n word (Sect. VI-B's accepted texts): position i is a
    digit drawn uniformly from 0-4 when i mod 2*rn < rn, else from 5-9.  A
    prefix of whole periods is in L(r_n)."""
    out = np.empty(n, dtype=np.uint8)
    k = 2 * rn

    def work(b):
        i, lo, hi = b
        rng = np.random.Generator(np.random.Philox(key=seed, counter=[0, 0, i, 0]))
        low = rng.integers(0, 5, size=hi - lo, dtype=np.uint8)
        phase = (np.arange(lo, hi, dtype=np.int64) % k) >= rn
        out[lo:hi] = low + np.uint8(48) + phase.astype(np.uint8) * np.uint8(5)

    blocks = _blocks(n)
    with ThreadPoolExecutor(min(8, max(1, len(blocks)))) as ex:
        list(ex.map(work, blocks))
    return out


def zipf_table(alphabet: bytes, s: float, seed: int, bits: int = 16) -> np.ndarray:
    """Quantised inverse CDF of Zipf(s) over the alphabet: rank r (1-based)
    has probability proportional to r^-s, ranks are assigned to symbols by a
    seeded permutation.  Entry i of the returned 2^bits table is the symbol
    for uniform draws in [i/2^bits, (i+1)/2^bits); each probability is thus
    rounded to a multiple of 2^-bits (at most 1.5e-5 off for bits = 16)."""
    m = len(alphabet)
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = np.frombuffer(alphabet, dtype=np.uint8)[rng.permutation(m)]
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w / w.sum())
    size = 1 << bits
    mids = (np.arange(size, dtype=np.float64) + 0.5) / size
    ranks = np.minimum(np.searchsorted(cdf, mids, side="right"), m - 1)
    return perm[ranks].astype(np.uint8)


def text_zipf(n: int, alphabet: bytes, s: float, seed: int) -> np.ndarray:
    table = zipf_table(alphabet, s, seed)
    return _fill_parallel(n, seed + 1,
                          lambda r, k: np.take(table, np.frombuffer(r.bytes(2 * k), dtype=np.uint16)))


def plant(text: np.ndarray, literals: Sequence[bytes], slot: int, seed: int) -> List[int]:
    """Plant one literal per `slot` bytes, at a seeded uniform offset inside
    the slot (so plants never overlap).  Returns the start offsets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(text)
    starts = []
    for base in range(0, n - slot + 1, slot):
        lit = literals[int(rng.integers(0, len(literals)))]
        off = base + int(rng.integers(0, slot - len(lit) + 1))
        text[off:off + len(lit)] = np.frombuffer(lit, dtype=np.uint8)
        starts.append(off)
    return starts


def log_uniform_lengths(k: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=k)).astype(np.int64)


def stable_hash(i: int) -> int:
    """splitmix64 finaliser, used to pair text i with an automaton."""
    z = (i + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


# ---------------------------------------------------------------------------
# The five workloads (sizes are parameters so tests can shrink them)
# ---------------------------------------------------------------------------

SEED_SINGLE, SEED_LARGE, SEED_BATCH, SEED_SIM, SEED_SERVE = 1405001, 1405002, 1405003, 1405004, 1405005


def workload_single(n: int = 1 << 20, seed: int = SEED_SINGLE):
    """KMP automaton of one seeded 6-byte literal over a-z (7 states) and n
    bytes of uniform a-z text with one planted copy per n/64-byte slot."""
    lit = random_literals(1, 6, 6, LOWER_ALPHABET, seed)[0]
    d = dfa_kmp(lit)
    text = text_uniform(n, LOWER_ALPHABET, seed + 10)
    slot = max(len(lit), n // 64)
    plant(text, [lit], slot, seed + 20)
    return d, text


def workload_large(n: int = 1 << 30, seed: int = SEED_LARGE):
    """Aho-Corasick automaton of 16 seeded literals of length 4..12 over the
    64-symbol base64 alphabet, and n bytes of Zipf(1.1) text over that
    alphabet with one planted literal per 64 KiB."""
    lits = random_literals(16, 4, 12, BASE64_ALPHABET, seed)
    d = dfa_aho_corasick(lits)
    text = text_zipf(n, BASE64_ALPHABET, 1.1, seed + 10)
    plant(text, lits, 1 << 16, seed + 20)
    return d, text


def workload_batch_automata(count: int = 8, seed: int = SEED_BATCH) -> List[DFA]:
    return [literal_set_automaton(seed * 100 + i) for i in range(count)]


def workload_batch_lengths(k: int = 4096, lo: int = 256, hi: int = 16 << 20,
                           seed: int = SEED_BATCH) -> np.ndarray:
    return log_uniform_lengths(k, lo, hi, seed + 1)


def workload_batch_pairing(k: int, n_automata: int) -> np.ndarray:
    return np.array([stable_hash(i) % n_automata for i in range(k)], dtype=np.int64)


def workload_sim_automata(seed: int = SEED_SIM) -> List[DFA]:
    return [dfa_random(nq, 16, seed + nq) for nq in (16, 32, 64)]


def workload_sim_automata_large(seed: int = SEED_SIM) -> List[DFA]:
    """Random complete DFAs of 128 and 256 states over 16 symbols (the same
    recipe as the simulation workload, past its 64 states)."""
    return [dfa_random(nq, 16, seed + nq) for nq in (128, 256)]


def workload_sim_text(n: int = 4 << 30, seed: int = SEED_SIM) -> np.ndarray:
    return text_uniform(n, bytes(range(16)), seed + 10)


def workload_serving_automata(count: int = 32, seed: int = SEED_SERVE) -> List[DFA]:
    return [literal_set_automaton(seed * 100 + i) for i in range(count)]


def workload_serving_requests(count: int, rate_per_s: float, seed: int = SEED_SERVE,
                              median: int = 64 << 10, sigma: float = 1.5,
                              cap: int = 64 << 20, n_automata: int = 32):
    """Poisson arrivals: (arrival time in s, text length, automaton index)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    lens = np.minimum(np.exp(rng.normal(math.log(median), sigma, size=count)), cap)
    lens = np.maximum(lens, 1).astype(np.int64)
    which = rng.integers(0, n_automata, size=count)
    return arrivals, lens, which
