"""Oracle for the SFA matcher — TEST INFRASTRUCTURE ONLY.

Plain CPU implementations of what the paper (Sin'ya, Matsuzaki, Sassa,
"Simultaneous Finite Automata", ICPP 2013) computes, written from its
definitions and algorithms.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_1405_0562_gb300``) and never imports it; the
two meet only through the seeded inputs of ``workloads``.

Functions and where they come from
----------------------------------
``dfa_run``        Alg. 2 (sequential DFA), extended with the count of
                   prefixes w[1..i], i = 1..n, that end in a final state.
                   (C, ``oracle.c``.)
``sfa_build``      Alg. 4 (correspondence construction) with the DFA
                   simplification of Sect. V-A; FIFO worklist.  (C.)
``sfa_accepting``  F_s of Definition 1 for I = {q0}: f(q0) in F.
``sfa_run``        the per-thread loop of Alg. 5.  (C.)
``compose``        reverse composition f . g := g o f (Sect. II-A).
``alg5``           Alg. 5: chunk runs from f_I, then the parallel (tree of
                   ``compose``) or the sequential reduction.
``alg3``           Alg. 3: per-chunk vectors T_i[q], then either reduction.
``witness``        a word w_f with f_I -w_f-> f, from the BFS parent links.
``bruteforce_*``   literal matching by direct substring comparison.

Pins (``tests/test_oracle_pins.py``; none re-types a formula of this file):
Example 1's six mappings and the run over ``abab``; Example 2's chunk states
and compositions; the printed D-SFA sizes of Sect. VI (r_5 = 109, r_50 = 10099,
(([02468][13579]){5})* = 21) and their closed form k^2 + k - 1 (k = 2n);
|S_d| = n^n for generators of the full transformation monoid (Fact 2);
|Q_s| equal to the number of distinct maps delta^w found by brute-force
enumeration of words; delta^w(q) of each state's witness word recomputed by
walking the DFA; brute-force literal counts and final states against
``dfa_run``; ``alg3``/``alg5`` equal to ``dfa_run`` for 1..64 chunks.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no -march)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.oracle_dfa_run.argtypes = [P, i32, i32, P, P, u64, P]
        lib.oracle_dfa_run.restype = i32
        lib.oracle_sfa_build.argtypes = [P, i32, P, i32, i64, P, P, P, P]
        lib.oracle_sfa_build.restype = i64
        lib.oracle_sfa_run.argtypes = [P, i32, P, i32, P, u64]
        lib.oracle_sfa_run.restype = i32
        lib.oracle_alg5_chunks.argtypes = [P, i32, P, P, P, i32, P, i32]
        lib.oracle_alg5_chunks.restype = ctypes.c_int
        lib.oracle_alg3_chunks.argtypes = [P, i32, P, P, i32, P, i32]
        lib.oracle_alg3_chunks.restype = ctypes.c_int
        lib.oracle_dfa_chunks.argtypes = [P, P, P, P, P, i32, P, P, i32]
        lib.oracle_dfa_chunks.restype = ctypes.c_int
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(text) -> np.ndarray:
    if isinstance(text, (bytes, bytearray)):
        return np.frombuffer(bytes(text), dtype=np.uint8)
    return np.ascontiguousarray(text, dtype=np.uint8)


def _dfa_arrays(delta, accept):
    d = np.ascontiguousarray(delta, dtype=np.int32)
    a = np.ascontiguousarray(accept, dtype=np.uint8)
    assert d.ndim == 2 and d.shape[1] == 256 and a.shape == (d.shape[0],)
    return d, a


# ---------------------------------------------------------------------------
# Alg. 2
# ---------------------------------------------------------------------------

def dfa_run(delta, q0: int, accept, text, start: Optional[int] = None):
    """Alg. 2 from `start` (default q0) over `text`.

    Returns (final state, accept bit of the final state, number of positions
    i in 1..n with delta^(q, w[1..i]) in F).  The empty prefix is not counted."""
    d, a = _dfa_arrays(delta, accept)
    t = _u8(text)
    q = q0 if start is None else start
    cnt = np.zeros(1, dtype=np.uint64)
    f = _lib().oracle_dfa_run(_ptr(d), d.shape[0], int(q), _ptr(a), _ptr(t), t.size, _ptr(cnt))
    return int(f), int(a[f]), int(cnt[0])


def dfa_run_chunks(delta, accept, text, bounds, starts, threads: int = 1):
    """Alg. 2 over each chunk [bounds[i], bounds[i+1]) from starts[i]."""
    d, a = _dfa_arrays(delta, accept)
    t = _u8(text)
    b = np.ascontiguousarray(bounds, dtype=np.uint64)
    s = np.ascontiguousarray(starts, dtype=np.int32)
    p = b.size - 1
    fin = np.zeros(p, dtype=np.int32)
    cnt = np.zeros(p, dtype=np.uint64)
    _lib().oracle_dfa_chunks(_ptr(d), _ptr(a), _ptr(t), _ptr(b), _ptr(s), p, _ptr(fin), _ptr(cnt), threads)
    return fin, cnt


# ---------------------------------------------------------------------------
# Alg. 4, Definition 1
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SFA:
    maps: np.ndarray      # int32 [S, nq]: maps[f, q] = f(q); row 0 is f_I
    delta: np.ndarray     # int32 [S, nsym]: id of f . delta^{symbols[k]}
    parent: np.ndarray    # int32 [S]
    psym: np.ndarray      # int32 [S]
    symbols: bytes

    @property
    def size(self) -> int:
        return int(self.maps.shape[0])

    @property
    def sym_index(self) -> np.ndarray:
        idx = np.full(256, -1, dtype=np.int32)
        for k, c in enumerate(self.symbols):
            idx[c] = k
        return idx


def sfa_build(delta, symbols: Optional[bytes] = None, cap: int = 1 << 18) -> Optional[SFA]:
    """Alg. 4 over the alphabet `symbols` (default: all 256 bytes).

    Returns None when more than `cap` states are reached."""
    d = np.ascontiguousarray(delta, dtype=np.int32)
    nq = d.shape[0]
    syms = bytes(range(256)) if symbols is None else bytes(symbols)
    sy = np.frombuffer(syms, dtype=np.uint8).copy()
    maps = np.zeros((cap, nq), dtype=np.int32)
    sdelta = np.zeros((cap, len(syms)), dtype=np.int32)
    parent = np.zeros(cap, dtype=np.int32)
    psym = np.zeros(cap, dtype=np.int32)
    n = _lib().oracle_sfa_build(_ptr(d), nq, _ptr(sy), len(syms), cap, _ptr(maps), _ptr(sdelta),
                                _ptr(parent), _ptr(psym))
    if n == -2:
        raise MemoryError("oracle_sfa_build")
    if n < 0:
        return None
    return SFA(maps[:n].copy(), sdelta[:n].copy(), parent[:n].copy(), psym[:n].copy(), syms)


def sfa_accepting(sfa: SFA, q0: int, accept) -> np.ndarray:
    """F_s (Definition 1) for I = {q0}: f is final iff f(q0) is final."""
    a = np.asarray(accept, dtype=np.uint8)
    return a[sfa.maps[:, q0]].astype(bool)


def witness(sfa: SFA, f: int) -> bytes:
    """A word w with f_I -w-> f, read off the BFS parent links."""
    out = []
    while sfa.parent[f] >= 0:
        out.append(sfa.symbols[sfa.psym[f]])
        f = int(sfa.parent[f])
    return bytes(reversed(out))


def sfa_run(sfa: SFA, text, start: int = 0) -> int:
    """The loop of one thread of Alg. 5: f <- delta_s[f, sigma]."""
    t = _u8(text)
    f = _lib().oracle_sfa_run(_ptr(sfa.delta), len(sfa.symbols), _ptr(sfa.sym_index), start, _ptr(t), t.size)
    if f < 0:
        raise ValueError("text has a byte outside the SFA's alphabet")
    return int(f)


def sfa_id_of(sfa: SFA, mapping) -> int:
    m = np.asarray(mapping, dtype=np.int32)
    hits = np.nonzero((sfa.maps == m[None, :]).all(axis=1))[0]
    return int(hits[0]) if hits.size else -1


# ---------------------------------------------------------------------------
# Composition and the two parallel algorithms
# ---------------------------------------------------------------------------

def compose(f, g) -> np.ndarray:
    """Reverse composition f . g := g o f on transformations (Sect. II-A):
    (f . g)(q) = g(f(q))."""
    f = np.asarray(f)
    g = np.asarray(g)
    return g[f]


def _reduce_parallel(vectors):
    """T_1 . T_2 . ... . T_p by a balanced tree of `compose` (associativity)."""
    level = [np.asarray(v) for v in vectors]
    while len(level) > 1:
        nxt = [compose(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def equal_bounds(n: int, p: int) -> np.ndarray:
    return np.array([(n * i) // p for i in range(p + 1)], dtype=np.uint64)


def alg5(sfa: SFA, text, bounds, q0: int, threads: int = 1, reduction: str = "sequential"):
    """Alg. 5 over the chunks [bounds[i], bounds[i+1]).

    Returns (chunk SFA states f_i, final DFA state).  'parallel' computes
    f_fin = f_1 . ... . f_p and S_fin = f_fin(q0); 'sequential' computes
    S <- f_i(S) for i = 1..p starting from {q0}."""
    t = _u8(text)
    b = np.ascontiguousarray(bounds, dtype=np.uint64)
    p = b.size - 1
    out = np.zeros(p, dtype=np.int32)
    rc = _lib().oracle_alg5_chunks(_ptr(sfa.delta), len(sfa.symbols), _ptr(sfa.sym_index), _ptr(t),
                                   _ptr(b), p, _ptr(out), threads)
    if rc:
        raise ValueError("text has a byte outside the SFA's alphabet")
    if reduction == "parallel":
        f_fin = _reduce_parallel([sfa.maps[f] for f in out])
        return out, int(f_fin[q0])
    s = q0
    for f in out:
        s = int(sfa.maps[f, s])
    return out, s


def alg3(delta, text, bounds, q0: int, threads: int = 1, reduction: str = "sequential"):
    """Alg. 3: per-chunk T_i[q] for every q, then the parallel reduction
    T = T_1 . ... . T_p, q_final = T[q0], or the sequential one
    q_final <- T_i[q_final]."""
    d = np.ascontiguousarray(delta, dtype=np.int32)
    t = _u8(text)
    b = np.ascontiguousarray(bounds, dtype=np.uint64)
    p = b.size - 1
    T = np.zeros((p, d.shape[0]), dtype=np.int32)
    _lib().oracle_alg3_chunks(_ptr(d), d.shape[0], _ptr(t), _ptr(b), p, _ptr(T), threads)
    if reduction == "parallel":
        return T, int(_reduce_parallel(list(T))[q0])
    s = q0
    for i in range(p):
        s = int(T[i, s])
    return T, s


def match_chunked(delta, q0: int, accept, text, bounds, threads: int = 1):
    """(final, accept bit, count) by Alg. 3 for the entering states of the
    chunks (sequential reduction) followed by Alg. 2 on every chunk from its
    entering state; equals dfa_run by Theorem 3."""
    d, a = _dfa_arrays(delta, accept)
    T, _ = alg3(d, text, bounds, q0, threads)
    starts = np.zeros(T.shape[0], dtype=np.int32)
    s = q0
    for i in range(T.shape[0]):
        starts[i] = s
        s = int(T[i, s])
    fin, cnt = dfa_run_chunks(d, a, text, bounds, starts, threads)
    return s, int(a[s]), int(cnt.sum())


# ---------------------------------------------------------------------------
# Brute force for literal automata
# ---------------------------------------------------------------------------

def bruteforce_literal_count(literals: Sequence[bytes], text) -> int:
    """#{i in 1..n : some literal l with |l| <= i equals w[i-|l| .. i)}."""
    t = bytes(_u8(text))
    ends = set()
    for lit in literals:
        start = t.find(lit)
        while start >= 0:
            ends.add(start + len(lit))
            start = t.find(lit, start + 1)
    return len(ends)


def bruteforce_final_string(state_strings: Sequence[bytes], text) -> bytes:
    """The longest suffix of the text that is one of the given strings (the
    literal prefixes); the literal automata end in the state with that
    string."""
    t = bytes(_u8(text))
    strings = set(state_strings)
    for k in range(min(len(t), max(len(s) for s in strings)), -1, -1):
        if t[len(t) - k:] in strings:
            return t[len(t) - k:]
    raise AssertionError("the empty string is always a state string")
