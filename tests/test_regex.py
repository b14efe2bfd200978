"""The regular-expression front end (Sect. VI's pipeline: McNaughton-Yamada,
Alg. 1, minimisation) and the N-SFA (Definition 1 / Alg. 4 over
correspondences).

The oracle (``oracle/regex.py``) is pinned first: its matcher against
Python's ``re`` on every short text over small alphabets, its N-SFA by
Alg. 4 against brute-force enumeration of words, and the N-SFA of (ab)*
against Example 1's six mappings.  Then the library's DFAs against the
oracle's matcher (counts and accept bits, anchored and search forms), its
N-SFA sizes against the oracle's, and its minimal DFA sizes against the
sizes printed in Sect. VI."""
import itertools
import random
import re

import numpy as np
import pytest

import oracle
from oracle import regex as R
from conftest import read_golden

PATTERNS = [
    (b"(ab)*", b"abx"),
    (b"he|she|his|hers", b"hersix"),
    (b"a(b|c)*d", b"abcdx"),
    (b"x[0-9]{2,3}y?", b"x01y"),
    (b"[^a]b+", b"abc"),
    (b"(a|b)*abb", b"ab"),
    (b"(?:ab|a)(bc|c)?", b"abc"),
    (b"a{0}b|c{2,}", b"abc"),
    (b"\\d\\w\\s", b"a1 _"),
    (b"[a-c][^b-c].", b"abcd\n"),
    (b"(a*)*b", b"ab"),
    (b"", b"ab"),
    (b"a||b", b"ab"),
    (b"[\\x61-\\x62]\\x63", b"abc"),
]


def texts_over(alpha, max_len):
    for n in range(max_len + 1):
        for t in itertools.product(alpha, repeat=n):
            yield bytes(t)


# ---------------------------------------------------------------------------
# pins of the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pattern,alpha", PATTERNS)
def test_oracle_matcher_equals_python_re(pattern, alpha):
    rx = re.compile(pattern)
    tree = R.parse(pattern)
    for t in texts_over(alpha, 5):
        got = len(t) in R.ends(tree, t, 0)
        assert got == (rx.fullmatch(t) is not None), (pattern, t)


@pytest.mark.parametrize("pattern,alpha", PATTERNS[:8])
def test_oracle_search_counts_equal_python_re(pattern, alpha):
    rx = re.compile(pattern)
    rng = random.Random(len(pattern))
    for _ in range(60):
        t = bytes(rng.choice(alpha) for _ in range(rng.randint(0, 9)))
        want = sum(1 for i in range(1, len(t) + 1) if any(rx.fullmatch(t[j:i]) for j in range(i + 1)))
        assert R.prefix_counts(pattern, t, search=True)[1] == want, (pattern, t)


@pytest.mark.parametrize("pattern", [b"(ab)*", b"a(b|c)*d", b"(a|b)*abb", b"he|she", b"(ab|ba)*", b"a{2,3}b*"])
def test_oracle_nsfa_alg4_equals_words(pattern):
    assert R.nsfa_alg4(pattern) == R.nsfa_words(pattern)


def test_oracle_nsfa_of_ab_star_is_example1():
    """The position NFA of (ab)* is deterministic (no dead state: missing
    transitions give the empty set), so its N-SFA is Example 1's D-SFA of
    (ab)*: six mappings (tests/golden/example1_ab_star.txt)."""
    maps = [r for r in read_golden("example1_ab_star.txt") if r[0] == "map"]
    assert R.nsfa_alg4(b"(ab)*") == R.nsfa_words(b"(ab)*") == len(maps) == 6


def test_oracle_syntax_errors():
    for bad in (b"a(b", b"(", b"*a", b"a{2,1}", b"[abc", b"a)", b"\\q", b"\\x4", b"a{1001}", b"^a", b"a$"):
        with pytest.raises(R.RegexSyntaxError):
            R.parse(bad)


# ---------------------------------------------------------------------------
# the library's front end against the oracle (host only)
# ---------------------------------------------------------------------------

sfa = pytest.importorskip("paper_1405_0562_gb300")


def run_dfa(delta, q0, acc, t):
    q, c = q0, 0
    for b in t:
        q = int(delta[q, b])
        c += int(acc[q])
    return int(acc[q]), c


@pytest.mark.parametrize("search", [False, True])
@pytest.mark.parametrize("pattern,alpha", PATTERNS)
def test_library_dfa_equals_oracle(pattern, alpha, search):
    delta, q0, acc, info = sfa.regex_dfa(pattern, search=search)
    assert info["nq"] == delta.shape[0] and 0 <= delta.min() and delta.max() < info["nq"]
    full, _, _, _ = sfa.regex_dfa(pattern, search=search, minimize=False)
    assert info["nq"] <= full.shape[0]
    rng = random.Random(7 + search)
    cases = list(texts_over(alpha, 4)) + [bytes(rng.choice(alpha) for _ in range(rng.randint(5, 14)))
                                          for _ in range(80)]
    for t in cases:
        want = R.prefix_counts(pattern, t, search=search)
        assert run_dfa(delta, q0, acc, t) == want, (pattern, t)
        # the unminimised subset automaton accepts the same prefixes
        assert run_dfa(full, 0, sfa.regex_dfa(pattern, search=search, minimize=False)[2], t) == want


def test_minimisation_is_minimal():
    """Partition refinement of the minimised DFA (final or not, then the
    blocks of the successors, to a fixpoint), recomputed here, leaves every
    state in a block of its own: no two states are equivalent."""
    for pattern, _ in PATTERNS:
        delta, q0, acc, info = sfa.regex_dfa(pattern, search=True)
        nq = info["nq"]
        # one byte per class of bytes with equal columns
        seen, bytes_ = {}, []
        for b in range(256):
            k = tuple(delta[:, b])
            if k not in seen:
                seen[k] = b
                bytes_.append(b)
        part = [int(a) for a in acc]
        while True:
            key = [tuple([part[q]] + [part[int(delta[q, b])] for b in bytes_]) for q in range(nq)]
            ids = {k: i for i, k in enumerate(sorted(set(key)))}
            new = [ids[k] for k in key]
            if len(set(new)) == len(set(part)):
                break
            part = new
        assert len(set(part)) == nq, pattern


def test_printed_dfa_sizes_from_expressions():
    """|D| of Sect. VI for the expressions themselves: r_n = ([0-4]{n}[5-9]{n})*
    (10 and 100 states for n = 5, 50) and (([02468][13579]){5})* (10): the
    minimal DFA has those states plus the dead one; its D-SFA has the printed
    |S_d| (tests/golden/sfa_sizes.txt) plus the all-dead mapping."""
    rows = {(r[0], int(r[1])): (int(r[2]), int(r[3])) for r in read_golden("sfa_sizes.txt")}
    for (fam, n), expr in (((("r_n", 5)), b"([0-4]{5}[5-9]{5})*"), (("r_n", 50), b"([0-4]{50}[5-9]{50})*"),
                           (("even_odd", 5), b"(([02468][13579]){5})*")):
        D, Sd = rows[(fam, n)]
        delta, q0, acc, info = sfa.regex_dfa(expr)
        assert info["nq"] - 1 == D
        a = sfa.Automaton(delta, q0, acc, host_only=True)
        assert a.info()["n_sfa_states"] - 1 == Sd


@pytest.mark.parametrize("pattern", [b"(ab)*", b"a(b|c)*d", b"(a|b)*abb", b"he|she", b"(ab|ba)*", b"a{2,3}b*",
                                     b"he|she|his|hers", b"x[0-9]{2,3}y?"])
def test_library_nsfa_equals_oracle(pattern):
    for search in (False, True):
        assert sfa.regex_nsfa_states(pattern, search=search) == R.nsfa_alg4(pattern, search=search), pattern


def test_library_syntax_errors_and_limits():
    for bad in (b"a(b", b"(", b"*a", b"a{2,1}", b"[abc", b"a)", b"\\q", b"\\x4", b"a{1001}", b"^a", b"a$"):
        with pytest.raises(sfa.SfaError) as e:
            sfa.regex_dfa(bad)
        assert e.value.code == sfa.ERR_INVALID
    # an expression past 4096 positions
    with pytest.raises(sfa.SfaError) as e:
        sfa.regex_dfa(b"[ab]{1000}[ab]{1000}[ab]{1000}[ab]{1000}[ab]{1000}")
    assert e.value.code == sfa.ERR_UNSUPPORTED
    # an N-SFA past its cap
    assert sfa.regex_nsfa_states(b"(a|b)*a(a|b){6}", cap=100) is None


def test_regex_to_handle_on_host():
    a = sfa.Automaton.from_regex(b"([0-4]{5}[5-9]{5})*", host_only=True)
    assert a.info()["n_sfa_states"] == 110
    L = sfa.lib()
    import ctypes
    h = ctypes.c_void_p()
    opts = sfa.CompileOpts(0, 0, sfa.COMPILE_HOST_ONLY, 0)
    pat = b"he|she|his|hers"
    assert L.sfa_regex_compile(pat, len(pat), sfa.REGEX_SEARCH, ctypes.byref(opts), ctypes.byref(h)) == sfa.OK
    L.sfa_destroy(h)


# ---------------------------------------------------------------------------
# on the GPU
# ---------------------------------------------------------------------------

@pytest.mark.gpu
def test_regex_handles_on_gpu():
    """Handles compiled from expressions (search form) matched on the GPU:
    against the oracle's matcher on short texts, and against Alg. 2 over the
    expression's DFA on 4 MiB."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)
    for pattern, alpha in PATTERNS[:10]:
        delta, q0, acc, _ = sfa.regex_dfa(pattern, search=True)
        a = sfa.Automaton(delta, q0, acc)
        rng = np.random.default_rng(len(pattern))
        alphabet = np.frombuffer(alpha, np.uint8)
        for n in (0, 1, 97, 2000):
            t = alphabet[rng.integers(0, alphabet.size, n)]
            out = a.match(torch.from_numpy(t).cuda())
            torch.cuda.synchronize()
            f, accf, st, cnt = sfa.decode(out)[0]
            assert st == 0 and (accf, cnt) == R.prefix_counts(pattern, bytes(t), search=True), (pattern, n)
        t = alphabet[rng.integers(0, alphabet.size, 4 << 20)]
        out = a.match(torch.from_numpy(t).cuda())
        torch.cuda.synchronize()
        f, accf, c = oracle.dfa_run(delta, q0, acc, t)
        assert sfa.decode(out)[0] == (f, accf, 0, c), pattern
