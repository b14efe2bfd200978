"""Regular-expression oracle -- TEST INFRASTRUCTURE ONLY.

Plain Python, written from the definitions; it shares no code with the
library's front end (``csrc/regex.cpp``) and never imports the package.

``parse``          the expression syntax of the library (bytes; see
                   ``include/sfa.h``) to a tree of tuples.
``ends``           the set of j with text[i:j] in L(e): a backtracking
                   (exhaustive) matcher that follows the meaning of each
                   operator -- concatenation, union, star as a least fixpoint,
                   counted repetition as repeated concatenation.
``prefix_counts``  the library's count semantics from ``ends``: positions
                   i in 1..n whose prefix text[:i] is in L(e), or (search)
                   at which an occurrence of e ends.
``position_nfa``   McNaughton and Yamada's position automaton (Sect. VI's
                   first step): states 0 and the positions, first/last/follow
                   from the textbook rules.
``nsfa_alg4``      Definition 1 / Alg. 4 on that NFA: correspondences f with
                   f_I(q) = {q}, f . delta^sigma.
``nsfa_words``     the same set by brute force: every delta-hat^w for words w,
                   longer and longer, until no new one appears.

Pins (``tests/test_regex.py``): ``ends`` against Python's ``re`` (fullmatch)
on every short text over small alphabets; ``nsfa_alg4`` against
``nsfa_words``; the N-SFA of (ab)* against Example 1's six mappings.
"""
from __future__ import annotations

import itertools
from functools import lru_cache
from typing import FrozenSet, Optional, Tuple

ALL = frozenset(range(256))
DIGITS = frozenset(range(ord("0"), ord("9") + 1))
WORDS = DIGITS | frozenset(range(ord("a"), ord("z") + 1)) | frozenset(range(ord("A"), ord("Z") + 1)) | {ord("_")}
SPACES = frozenset(b" \t\n\r\f\v")


class RegexSyntaxError(ValueError):
    pass


def parse(pattern: bytes, dotall: bool = False):
    """Recursive descent over: alt := cat ('|' cat)*; cat := rep*;
    rep := atom ('*' | '+' | '?' | '{m}' | '{m,}' | '{m,n}')*."""
    p = bytes(pattern)
    pos = [0]

    def peek():
        return p[pos[0]] if pos[0] < len(p) else None

    def take():
        c = p[pos[0]]
        pos[0] += 1
        return c

    def err():
        raise RegexSyntaxError(f"at byte {pos[0]} of {p!r}")

    def escape():
        if peek() is None:
            err()
        c = chr(take())
        table = {"d": DIGITS, "D": ALL - DIGITS, "w": WORDS, "W": ALL - WORDS, "s": SPACES, "S": ALL - SPACES,
                 "n": {10}, "t": {9}, "r": {13}, "f": {12}, "v": {11}, "0": {0}}
        if c in table:
            return frozenset(table[c])
        if c == "x":
            h = p[pos[0]:pos[0] + 2]
            try:
                v = int(h.decode(), 16)
            except (ValueError, UnicodeDecodeError):
                err()
            if len(h) != 2:
                err()
            pos[0] += 2
            return frozenset({v})
        if c.isalnum():
            err()
        return frozenset({ord(c)})

    def single(s):
        return next(iter(s)) if len(s) == 1 else None

    def klass():
        neg = peek() == ord("^")
        if neg:
            take()
        members = set()
        first = True
        while peek() is not None and (peek() != ord("]") or first):
            first = False
            if peek() == ord("\\"):
                take()
                s = escape()
                lo = single(s)
                if lo is None:
                    members |= s
                    continue
            else:
                lo = take()
            if peek() == ord("-") and pos[0] + 1 < len(p) and p[pos[0] + 1] != ord("]"):
                take()
                if peek() == ord("\\"):
                    take()
                    hi = single(escape())
                    if hi is None:
                        err()
                else:
                    hi = take()
                if hi < lo:
                    err()
                members |= set(range(lo, hi + 1))
            else:
                members.add(lo)
        if peek() is None:
            err()
        take()
        return ("set", frozenset(ALL - members if neg else members))

    def atom():
        c = peek()
        if c is None:
            err()
        if c == ord("("):
            take()
            if p[pos[0]:pos[0] + 2] == b"?:":
                pos[0] += 2
            e = alt()
            if peek() != ord(")"):
                err()
            take()
            return e
        if c == ord("["):
            take()
            return klass()
        if c == ord("."):
            take()
            return ("set", ALL if dotall else ALL - {10})
        if c == ord("\\"):
            take()
            return ("set", escape())
        if chr(c) in ")|*+?{]}^$":
            err()
        take()
        return ("set", frozenset({c}))

    def number():
        s = pos[0]
        while peek() is not None and ord("0") <= peek() <= ord("9"):
            take()
        if pos[0] == s:
            err()
        v = int(p[s:pos[0]])
        if v > 1000:
            err()
        return v

    def rep():
        e = atom()
        while peek() is not None and chr(peek()) in "*+?{":
            c = chr(take())
            if c == "*":
                e = ("star", e)
            elif c == "+":
                e = ("plus", e)
            elif c == "?":
                e = ("opt", e)
            else:
                m = number()
                n: Optional[int] = m
                if peek() == ord(","):
                    take()
                    n = None if peek() == ord("}") else number()
                if peek() != ord("}"):
                    err()
                take()
                if n is not None and n < m:
                    err()
                e = ("rep", e, m, n)
        return e

    def cat():
        parts = []
        while peek() is not None and peek() not in (ord("|"), ord(")")):
            parts.append(rep())
        e = ("eps",)
        for x in parts:
            e = x if e == ("eps",) else ("cat", e, x)
        return e

    def alt():
        e = cat()
        while peek() == ord("|"):
            take()
            e = ("alt", e, cat())
        return e

    tree = alt()
    if pos[0] != len(p):
        err()
    return tree


def ends(tree, text: bytes, i: int) -> FrozenSet[int]:
    """{ j : text[i:j] in L(tree) } (every parse explored)."""
    text = bytes(text)

    @lru_cache(maxsize=None)
    def go(node, k):
        kind = node[0]
        if kind == "eps":
            return frozenset({k})
        if kind == "set":
            return frozenset({k + 1}) if k < len(text) and text[k] in node[1] else frozenset()
        if kind == "cat":
            out = set()
            for j in go(node[1], k):
                out |= go(node[2], j)
            return frozenset(out)
        if kind == "alt":
            return go(node[1], k) | go(node[2], k)
        if kind == "opt":
            return frozenset({k}) | go(node[1], k)
        if kind in ("star", "plus"):
            # the least set containing k (star) and closed under one more
            # match of the operand
            seen = {k}
            todo = [k]
            while todo:
                x = todo.pop()
                for j in go(node[1], x):
                    if j not in seen:
                        seen.add(j)
                        todo.append(j)
            if kind == "star":
                return frozenset(seen)
            # plus: at least one match of the operand
            out = set()
            for j in go(node[1], k):
                out |= go(("star", node[1]), j)
            return frozenset(out)
        if kind == "rep":
            _, sub, m, n = node
            cur = {k}
            for _ in range(m):
                cur = set().union(*(go(sub, x) for x in cur)) if cur else set()
            if n is None:
                out = set()
                for x in cur:
                    out |= go(("star", sub), x)
                return frozenset(out)
            out = set(cur)
            for _ in range(n - m):
                cur = set().union(*(go(sub, x) for x in cur)) if cur else set()
                out |= cur
            return frozenset(out)
        raise AssertionError(kind)

    return go(tree, i)


def prefix_counts(pattern: bytes, text: bytes, search: bool = False, dotall: bool = False) -> Tuple[int, int]:
    """(accept bit of the whole text, number of positions i in 1..n counted):
    anchored, i is counted when text[:i] is in L; search, when some
    text[j:i] is."""
    tree = parse(pattern, dotall)
    text = bytes(text)
    n = len(text)
    hit = set(ends(tree, text, 0))
    if search:
        for j in range(1, n + 1):
            hit |= ends(tree, text, j)
    count = sum(1 for i in range(1, n + 1) if i in hit)
    return int(n in hit), count


def position_nfa(pattern: bytes, search: bool = False, dotall: bool = False):
    """(number of states, delta as {(q, byte): frozenset}, final states):
    states 0 (initial) and the positions 1..P of the expression's symbol
    sets, left to right; counted repetitions are expanded first."""
    tree = parse(pattern, dotall)

    def expand(node):
        kind = node[0]
        if kind == "rep":
            _, sub, m, n = node
            out = None
            for _ in range(m):
                out = sub if out is None else ("cat", out, sub)
            if n is None:
                tail = ("star", sub)
            else:
                tail = None
                for _ in range(n - m):
                    tail = ("opt", sub if tail is None else ("cat", sub, tail))
            if tail is not None:
                out = tail if out is None else ("cat", out, tail)
            return expand(out if out is not None else ("eps",))
        if kind in ("cat", "alt"):
            return (kind, expand(node[1]), expand(node[2]))
        if kind in ("star", "plus", "opt"):
            return (kind, expand(node[1]))
        return node

    syms = [None]
    follow = {0: set()}

    def walk(node):
        """(nullable, first, last) of node; follow filled as a side effect."""
        kind = node[0]
        if kind == "eps":
            return True, set(), set()
        if kind == "set":
            syms.append(node[1])
            k = len(syms) - 1
            follow[k] = set()
            return False, {k}, {k}
        if kind == "cat":
            na, fa, la = walk(node[1])
            nb, fb, lb = walk(node[2])
            for x in la:
                follow[x] |= fb
            return na and nb, fa | (fb if na else set()), lb | (la if nb else set())
        if kind == "alt":
            na, fa, la = walk(node[1])
            nb, fb, lb = walk(node[2])
            return na or nb, fa | fb, la | lb
        na, fa, la = walk(node[1])
        if kind in ("star", "plus"):
            for x in la:
                follow[x] |= fa
        return (True if kind != "plus" else na), fa, la

    nullable, first, last = walk(expand(tree))
    follow[0] = set(first)
    P = len(syms) - 1
    delta = {}
    for q in range(P + 1):
        for b in range(256):
            s = frozenset(x for x in follow[q] if b in syms[x])
            if search and q == 0:
                s = s | {0}
            delta[(q, b)] = s
    final = set(last) | ({0} if nullable else set())
    return P + 1, delta, frozenset(final)


def _classes(nq, delta):
    """One byte per class of bytes with equal columns of delta."""
    seen, reps = {}, []
    for b in range(256):
        col = tuple(delta[(q, b)] for q in range(nq))
        if col not in seen:
            seen[col] = b
            reps.append(b)
    return reps


def _step(f, b, nq, delta):
    """f . delta^b for a correspondence f (a tuple of frozensets)."""
    return tuple(frozenset().union(*(delta[(x, b)] for x in f[q])) if f[q] else frozenset() for q in range(nq))


def nsfa_alg4(pattern: bytes, search: bool = False, dotall: bool = False, cap: int = 100000) -> Optional[int]:
    """|Q_s| of the N-SFA by Alg. 4 (FIFO worklist from f_I), or None past cap."""
    nq, delta, _ = position_nfa(pattern, search, dotall)
    reps = _classes(nq, delta)
    fi = tuple(frozenset({q}) for q in range(nq))
    seen = {fi}
    todo = [fi]
    while todo:
        f = todo.pop(0)
        for b in reps:
            g = _step(f, b, nq, delta)
            if g not in seen:
                if len(seen) >= cap:
                    return None
                seen.add(g)
                todo.append(g)
    return len(seen)


def nsfa_words(pattern: bytes, search: bool = False, dotall: bool = False, max_len: int = 12) -> Optional[int]:
    """|{ delta-hat^w : |w| <= L }| for growing L, every word of each length
    enumerated, until a length adds no new correspondence (then the set is
    closed: a longer word's correspondence extends a shorter one's), or
    None if max_len is reached first."""
    nq, delta, _ = position_nfa(pattern, search, dotall)
    reps = _classes(nq, delta)

    def hat(word):
        f = tuple(frozenset({q}) for q in range(nq))
        for b in word:
            f = _step(f, b, nq, delta)
        return f

    found = {hat(())}
    for length in range(1, max_len + 1):
        new = {hat(w) for w in itertools.product(reps, repeat=length)} - found
        if not new:
            return len(found)
        found |= new
    return None
