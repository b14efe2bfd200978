"""Host-side logic of the product, on the CPU: the C ABI loads and exports
every symbol of include/sfa.h, and the D-SFA tables that sfa_compile builds
agree with the oracle's independent correspondence construction.  No test
here launches GPU work (handles are compiled host-only)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1405_0562_gb300 as sfa
import workloads as W
from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "sfa.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfa_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    declared = header_functions()
    assert declared == sorted(sfa.EXPORTED)
    lib = sfa.lib()
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_covers_codes():
    for code in range(0, -9, -1):
        assert sfa.strerror(code) != "unknown error code"
    assert sfa.strerror(-99) == "unknown error code"


def host(d, **kw):
    return sfa.Automaton.from_dfa(d, host_only=True, **kw)


def product_maps(a):
    """Non-constant mappings of the product, in the caller's state numbering,
    plus the reached constants, as a set of tuples."""
    info = a.info()
    nr = info["n_reachable"]
    orig = a.export(sfa.TABLE_ORIG)
    maps = a.export(sfa.TABLE_MAPS).reshape(-1, nr) if info["n_nonconst"] else np.zeros((0, nr), np.uint8)
    return orig, maps


def to_orig(vec_kept, orig, nq):
    """A mapping over kept states (kept numbering) as a mapping over the
    caller's states (only the reachable ones are defined)."""
    out = np.full(nq, -1, dtype=np.int64)
    out[orig] = orig[np.asarray(vec_kept, dtype=np.int64)]
    return out


AUTOMATA = [
    ("ab_star", W.dfa_ab_star),
    ("r3", lambda: W.dfa_rn(3)),
    ("r5", lambda: W.dfa_rn(5)),
    ("ra2", lambda: W.dfa_ra(2)),
    ("even_odd5", lambda: W.dfa_even_odd(5)),
    ("T4", lambda: W.dfa_full_transformation(4)),
    ("kmp", lambda: W.dfa_kmp(b"abcaab")),
    ("ac", lambda: W.dfa_aho_corasick([b"he", b"she", b"his", b"hers"])),
    ("ac_set", lambda: W.literal_set_automaton(11)),
    ("single", lambda: W.workload_single(1 << 12)[0]),
]


@pytest.mark.parametrize("name,make", AUTOMATA)
def test_sizes_equal_oracle(name, make):
    d = make()
    s = oracle.sfa_build(d.delta)          # over all 256 byte values
    info = host(d).info()
    assert info["mode"] == sfa.MODE_SFA
    assert info["n_reachable"] == d.nq     # generators give accessible DFAs
    assert info["n_sfa_states"] == s.size


@pytest.mark.parametrize("name,make", AUTOMATA)
def test_tables_equal_oracle_construction(name, make):
    """Same set of mappings as the oracle, and every row of the product's
    transition table leads where the oracle's does."""
    d = make()
    s = oracle.sfa_build(d.delta)
    a = host(d)
    info = a.info()
    nr, ncls = info["n_reachable"], info["ncls"]
    orig, maps = product_maps(a)
    cls = a.export(sfa.TABLE_CLASS)
    dfa = a.export(sfa.TABLE_DFA).reshape(nr, 256)
    oracle_ids = {tuple(m): i for i, m in enumerate(s.maps)}
    prod = {}
    for k in range(maps.shape[0]):
        v = tuple(to_orig(maps[k], orig, d.nq))
        assert v in oracle_ids
        prod[k] = oracle_ids[v]
    consts = {oracle_ids[tuple(m)] for m in s.maps if len(set(m.tolist())) == 1}
    assert len(prod) + len(consts) == s.size
    # the kept DFA is the caller's DFA renumbered
    for i in range(nr):
        assert (orig[dfa[i]] == d.delta[orig[i]]).all()
    # final states last
    fa = nr - info["n_accepting"]
    assert all(d.accept[orig[i]] == (i >= fa) for i in range(nr))
    if maps.shape[0] == 0:
        return
    nc = a.export(sfa.TABLE_NC).reshape(-1, ncls)
    rng = np.random.default_rng(0)
    for k in range(maps.shape[0]):
        for b in rng.integers(0, 256, 24).tolist() + list(d.alphabet):
            e = int(nc[k, cls[b]])
            nxt, acc = e & 0x3FFFFFFF, e >> 30
            want = s.maps[s.delta[prod[k], b]]          # oracle: f . delta^b
            if nxt < nr:
                got = np.full(d.nq, orig[nxt])
                fin = [bool(d.accept[orig[nxt]])]
            else:
                got = to_orig(maps[nxt - nr], orig, d.nq)
                fin = [bool(d.accept[x]) for x in got[orig]]
            assert (got[orig] == want[orig]).all()
            assert acc == (1 if all(fin) else (2 if any(fin) else 0))


def test_example1_product_numbering():
    """Constant mappings take the id of their value; the others follow in
    FIFO order of Alg. 4, f_I first (the numbering of Example 1 minus f3)."""
    d = W.dfa_ab_star()
    a = host(d)
    info = a.info()
    assert (info["n_sfa_states"], info["n_nonconst"]) == (6, 5)
    orig, maps = product_maps(a)
    got = [tuple(to_orig(m, orig, 3)) for m in maps]
    assert got == [(0, 1, 2), (1, 2, 2), (2, 0, 2), (0, 2, 2), (2, 1, 2)]   # f0 f1 f2 f4 f5


def test_printed_sizes_via_product():
    """Every size printed in Sect. VI (tests/golden/sfa_sizes.txt), counted by
    the product's construction.  r_500 and r_a have more than 256 states:
    16-bit ids, with the point mappings counted but not stored."""
    from conftest import read_golden
    make = {"r_n": W.dfa_rn, "r_a": W.dfa_ra, "even_odd": W.dfa_even_odd}
    for fam, n, D, Sd in ((r[0], int(r[1]), int(r[2]), int(r[3])) for r in read_golden("sfa_sizes.txt")):
        d = make[fam](n)
        info = host(d).info()
        assert info["n_reachable"] - 1 == D             # the sink is not counted
        assert info["n_sfa_states"] - 1 == Sd           # nor the all-sink mapping (a constant)
        if info["n_reachable"] > 256:
            assert info["id_bits"] == 16 and info["n_stored"] < 4 * info["n_reachable"]
            assert info["placement"] == sfa.PLACE_SMEM_DFA_CLASSES | sfa.PLACE_GLOBAL_NC
        else:
            assert info["id_bits"] == 8 and info["n_stored"] == info["n_nonconst"]


@pytest.mark.parametrize("n", [127, 128, 129, 300, 1000])
def test_rn_sizes_across_the_id_width(n):
    """k^2 + k - 1 non-constant D-SFA states for r_n (k = 2n; the closed
    form the oracle pins on n <= 6), on both sides of 256 reachable states:
    n = 127 stores every mapping, n >= 128 keeps the k^2 point mappings
    implicit."""
    k = 2 * n
    info = host(W.dfa_rn(n)).info()
    assert info["n_nonconst"] == k * k + k - 1
    assert info["id_bits"] == (8 if n <= 127 else 16)


def test_cap_switches_to_simulation():
    d = W.dfa_full_transformation(5)
    assert host(d, cap_states=100).info()["mode"] == sfa.MODE_SIM
    info = host(d, cap_states=3125).info()
    assert info["mode"] == sfa.MODE_SFA and info["n_sfa_states"] == 3125
    with pytest.raises(sfa.SfaError) as e:
        host(d, cap_states=100, mode=sfa.MODE_SFA)
    assert e.value.code == sfa.ERR_UNSUPPORTED
    assert host(d, mode=sfa.MODE_SIM).info()["mode"] == sfa.MODE_SIM


def test_random_dfas_exceed_default_cap():
    for d in W.workload_sim_automata():
        info = host(d).info()
        assert info["mode"] == sfa.MODE_SIM, d.name


@pytest.mark.parametrize("nq", [65, 100, 128, 129, 200, 256])
def test_simulation_up_to_256_states(nq):
    """Alg. 3 serves every DFA of up to 256 states: random complete DFAs past
    the D-SFA cap compile in simulation mode (the cycle automaton, whose
    D-SFA is the nq rotations, stays a D-SFA unless forced)."""
    info = host(W.dfa_random(nq, 16, seed=nq)).info()
    assert info["mode"] == sfa.MODE_SIM and info["n_reachable"] <= nq
    cyc = np.tile((np.arange(nq, dtype=np.int32)[:, None] + 1) % nq, (1, 256))
    acc = (np.arange(nq) % 3 == 0).astype(np.uint8)
    a = sfa.Automaton(cyc, 0, acc, host_only=True)
    assert a.info()["mode"] == sfa.MODE_SFA and a.info()["n_sfa_states"] == nq
    a = sfa.Automaton(cyc, 0, acc, host_only=True, mode=sfa.MODE_SIM)
    assert a.info()["mode"] == sfa.MODE_SIM and a.info()["n_reachable"] == nq


def test_unreachable_states_are_trimmed():
    d = W.dfa_ab_star()
    delta = np.concatenate([d.delta, np.full((2, 256), 3, dtype=np.int32)])   # states 3, 4 unreachable
    acc = np.concatenate([d.accept, [1, 0]]).astype(np.uint8)
    a = sfa.Automaton(delta, 0, acc, host_only=True)
    info = a.info()
    assert (info["nq"], info["n_reachable"], info["n_sfa_states"]) == (5, 3, 6)


@pytest.mark.parametrize("case,code", [
    ("nq0", sfa.ERR_INVALID), ("nq4096", sfa.ERR_UNSUPPORTED), ("range", sfa.ERR_INVALID),
    ("q0", sfa.ERR_INVALID),
])
def test_invalid_dfas(case, code):
    L = sfa.lib()
    h = ctypes.c_void_p()
    opts = sfa.CompileOpts(0, 0, sfa.COMPILE_HOST_ONLY, 0)
    nq, q0 = 4, 0
    delta = np.zeros((4, 256), dtype=np.int32)
    if case == "nq0":
        nq = 0
    elif case == "nq4096":
        nq = 4096
        delta = np.zeros((4096, 256), dtype=np.int32)
    elif case == "range":
        delta[2, 7] = 4
    elif case == "q0":
        q0 = 4
    acc = np.zeros(max(nq, 1), dtype=np.uint8)
    rc = L.sfa_compile(delta.ctypes.data, nq, q0, acc.ctypes.data, ctypes.byref(opts), ctypes.byref(h))
    assert rc == code


def test_host_only_handle_refuses_matching():
    a = host(W.dfa_ab_star())
    L = sfa.lib()
    out = ctypes.c_void_p(0)
    assert L.sfa_match(a.handle, None, 0, ctypes.c_void_p(16), None) == sfa.ERR_HOST_ONLY
    assert L.sfa_match(a.handle, None, 0, out, None) == sfa.ERR_INVALID   # NULL result pointer


def test_class_compression_is_exact():
    """Bytes in one class have equal columns in the caller's DFA."""
    d = W.workload_large(1 << 12)[0]
    a = host(d)
    cls = a.export(sfa.TABLE_CLASS)
    for c in np.unique(cls):
        cols = d.delta[:, cls == c]
        assert (cols == cols[:, :1]).all()
    # and different classes differ somewhere
    reps = [int(np.nonzero(cls == c)[0][0]) for c in np.unique(cls)]
    assert len({tuple(d.delta[:, b]) for b in reps}) == len(reps)


def test_noalloc_refusals_need_no_device():
    """sfa_match_noalloc decides every refusal before it enqueues work or looks
    up its array: checked here with host-only handles (no GPU in this
    process), which it refuses after the argument and mode checks."""
    L = sfa.lib()
    L.sfa_match_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_void_p]
    big = host(W.workload_large(1 << 12)[0])              # 127 states: ~135 B of scratch per tile
    fake = ctypes.c_void_p(1 << 20)                        # never dereferenced
    # texts past 2^40 bytes are invalid; the longest valid one gets as far as
    # the check for device tables
    assert L.sfa_match_noalloc(big.handle, fake, (1 << 40) + 1, fake, None) == sfa.ERR_INVALID
    assert L.sfa_match_noalloc(big.handle, fake, 1 << 40, fake, None) == sfa.ERR_HOST_ONLY
    assert L.sfa_match_noalloc(big.handle, None, 16, fake, None) == sfa.ERR_INVALID
    assert L.sfa_match_noalloc(big.handle, fake, 16, None, None) == sfa.ERR_INVALID
    sim = host(W.workload_sim_automata()[0])
    assert L.sfa_match_noalloc(sim.handle, fake, 16, fake, None) == sfa.ERR_UNSUPPORTED
    # a valid call still needs the handle's device tables
    assert L.sfa_match_noalloc(big.handle, fake, 1 << 20, fake, None) == sfa.ERR_HOST_ONLY


def _kept_dfa(a):
    """The handle's kept DFA in the caller's ids: {(orig q, byte): orig q'},
    and the caller id of every kept id."""
    orig = a.export(sfa.TABLE_ORIG)
    dfa = a.export(sfa.TABLE_DFA).reshape(-1, 256)
    return orig, dfa


@pytest.mark.parametrize("make", [lambda: W.workload_large(1 << 12)[0], lambda: W.workload_batch_automata(3)[2],
                                  lambda: W.dfa_rn(5), lambda: W.dfa_kmp(b"abcaab")])
def test_bank_numbering_is_a_renumbering(make):
    """The numbering chosen against bank conflicts (uniform model, or a
    sample's) is a permutation of the breadth-first one that keeps the final
    states last, and the kept DFA is the same automaton under it: row
    orig_of[i] of the caller's table, renumbered, for every kept id i."""
    d = make()
    base = host(d, bank_tune=False)
    acc = np.asarray(d.accept, dtype=bool)
    rng = np.random.default_rng(4)
    sample = np.frombuffer(d.alphabet, np.uint8)[rng.integers(0, len(d.alphabet), 1 << 16)]
    tuned = [host(d), host(d, sample=sample)]
    o0, D0 = _kept_dfa(base)
    nfin = int((~acc[o0]).sum())
    assert not acc[o0[:nfin]].any() and acc[o0[nfin:]].all()
    for a in tuned:
        o1, D1 = _kept_dfa(a)
        assert sorted(o1.tolist()) == sorted(o0.tolist())
        assert not acc[o1[:nfin]].any() and acc[o1[nfin:]].all()   # final states last
        kept_of = {int(q): i for i, q in enumerate(o1)}
        for i, q in enumerate(o1):
            assert [kept_of[int(x)] for x in d.delta[q]] == D1[i].tolist()
        # the D-SFA has as many states either way (Alg. 4 is structural)
        assert a.info()["n_sfa_states"] == base.info()["n_sfa_states"]
        assert a.info()["n_nonconst"] == base.info()["n_nonconst"]


def test_bank_numbering_moves_the_hot_states():
    """On the 127-state Aho-Corasick automaton the search does renumber, and
    deterministically (two compiles give the same tables)."""
    d = W.workload_large(1 << 12)[0]
    o0, _ = _kept_dfa(host(d, bank_tune=False))
    o1, D1 = _kept_dfa(host(d))
    o2, D2 = _kept_dfa(host(d))
    assert (o1 != o0).any()
    assert (o1 == o2).all() and (D1 == D2).all()


def test_compile_sample_arguments():
    d = W.dfa_ab_star()
    delta = np.ascontiguousarray(d.delta, dtype=np.int32)
    acc = np.ascontiguousarray(d.accept, dtype=np.uint8)
    opts = sfa.CompileOpts(0, 0, sfa.COMPILE_HOST_ONLY, 0)
    h = ctypes.c_void_p()
    L = sfa.lib()
    assert L.sfa_compile_sample(delta.ctypes.data, d.nq, d.q0, acc.ctypes.data, ctypes.byref(opts), None, 5,
                                ctypes.byref(h)) == sfa.ERR_INVALID
    assert L.sfa_compile_sample(delta.ctypes.data, d.nq, d.q0, acc.ctypes.data, ctypes.byref(opts), None, 0,
                                ctypes.byref(h)) == sfa.OK
    L.sfa_destroy(h)
    short = np.zeros(10, np.uint8)   # too short for the model: the uniform one is used
    assert L.sfa_compile_sample(delta.ctypes.data, d.nq, d.q0, acc.ctypes.data, ctypes.byref(opts),
                                short.ctypes.data, short.size, ctypes.byref(h)) == sfa.OK
    L.sfa_destroy(h)


def test_wide_set_point_entries_are_the_mappings_they_stand_for():
    """16-bit-id tables: every row entry of a stored mapping f on class c is
    f . delta^c -- a constant, a point mapping (NC_POINT, source s), a
    set-point mapping (NC_POINT | NC_SET, source set from SFA_TABLE_SETS) or
    a stored mapping -- recomputed here from the exported DFA and mappings."""
    for d in (W.dfa_ra(150), W.dfa_rn(140)):
        a = host(d)
        info = a.info()
        assert info["id_bits"] == 16
        nr, ncls = info["n_reachable"], info["ncls"]
        cdfa = a.export(sfa.TABLE_CDFA16).reshape(nr, ncls).astype(np.int64)
        maps = a.export(sfa.TABLE_MAPS16).reshape(-1, nr).astype(np.int64)
        nc = a.export(sfa.TABLE_NC).reshape(-1, ncls)
        words = (nr + 31) // 32
        sets = a.export(sfa.TABLE_SETS).reshape(-1, words) if d.name.startswith("r_a") else None
        sink = [q for q in range(nr) if (cdfa[q] == q).all() and q < nr - info["n_accepting"]][0]
        n_sets = 0
        for h in range(maps.shape[0]):
            for c in range(ncls):
                g = cdfa[maps[h], c]
                e = int(nc[h, c])
                if e & (1 << 29):
                    p = e & 0xFFF
                    fld = (e >> 12) & 0xFFF
                    if e & (1 << 28):
                        n_sets += 1
                        src = {q for q in range(nr) if sets[fld][q >> 5] >> (q & 31) & 1}
                        assert len(src) >= 2
                    else:
                        src = {fld}
                    want = np.array([p if q in src else sink for q in range(nr)])
                    assert np.array_equal(g, want), (d.name, h, c)
                else:
                    ident = e & 0x1FFFFFFF
                    if ident < nr:
                        assert (g == ident).all()
                    else:
                        assert np.array_equal(g, maps[ident - nr])
        assert (n_sets > 0) == d.name.startswith("r_a")
