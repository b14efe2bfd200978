"""GPU parity: every result of the CUDA path (through the C ABI) equals the
CPU oracle's, bit for bit (all outputs are integers: final state, accept
bit, uint64 count; tolerance 0)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1405_0562_gb300 as sfa
    sfa.lib()
    torch.cuda.set_device(0)
    yield


def sfa_mod():
    import paper_1405_0562_gb300 as sfa
    return sfa


def gpu_match(a, text_np, **launch):
    t = torch.from_numpy(np.ascontiguousarray(text_np, dtype=np.uint8)).cuda()
    out = a.match(t, **launch)
    torch.cuda.synchronize()
    return sfa_mod().decode(out)[0]


def expect(d, text_np):
    f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, text_np)
    return (f, acc, 0, c)


def text_for(d, n, seed):
    rng = np.random.default_rng(seed)
    alpha = np.frombuffer(d.alphabet, dtype=np.uint8)
    t = alpha[rng.integers(0, len(alpha), n)]
    if d.name.startswith(("r_", "even_odd")) and n > 0:
        # mostly accepted text with rare errors, so counts are large; k is
        # the length of the automaton's loop
        k = d.nq - 3 if d.name.startswith("r_a") else d.nq - 1
        base = []
        for i in range(n):
            pos = i % k
            if d.name.startswith("even_odd"):
                base.append(b"02468"[rng.integers(0, 5)] if pos % 2 == 0 else b"13579"[rng.integers(0, 5)])
            else:
                base.append(b"01234"[rng.integers(0, 5)] if pos < k // 2 else b"56789"[rng.integers(0, 5)])
        t = np.array(base, dtype=np.uint8)
        flips = rng.integers(0, n, max(1, n // 5000))
        t[flips] = alpha[rng.integers(0, len(alpha), flips.size)]
    return t


AUTOMATA = {
    "ab_star": W.dfa_ab_star,
    "r3": lambda: W.dfa_rn(3),
    "r5": lambda: W.dfa_rn(5),
    "ra2": lambda: W.dfa_ra(2),
    "even_odd5": lambda: W.dfa_even_odd(5),
    "T4": lambda: W.dfa_full_transformation(4),
    "kmp": lambda: W.dfa_kmp(b"abcaab"),
    "ac": lambda: W.dfa_aho_corasick([b"he", b"she", b"his", b"hers"]),
    "ac_set": lambda: W.literal_set_automaton(11),
    "rand8": lambda: W.dfa_random(8, 4, seed=3),
    "single": lambda: W.workload_single(1 << 12)[0],
    "one_state": lambda: W.DFA(np.zeros((1, 256), np.int32), 0, np.ones(1, np.uint8), b"ab", name="one"),
}


@pytest.mark.parametrize("name", sorted(AUTOMATA))
@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, 65536 + 13, 1 << 20])
def test_default_shape(name, n):
    d = AUTOMATA[name]()
    a = sfa_mod().Automaton.from_dfa(d)
    t = text_for(d, n, seed=n)
    assert gpu_match(a, t) == expect(d, t)


@pytest.mark.parametrize("name", ["ab_star", "r3", "ac", "rand8", "T4"])
def test_forced_chunk_counts_1_to_64(name):
    """Theorem 3: any division gives the same result (1..64 chunks)."""
    d = AUTOMATA[name]()
    a = sfa_mod().Automaton.from_dfa(d)
    for n in (0, 5, 3001):
        t = text_for(d, n, seed=7)
        want = expect(d, t)
        for p in range(1, 65):
            assert gpu_match(a, t, forced_chunks=p) == want, (n, p)
            assert gpu_match(a, t, forced_chunks=p, block_threads=128, chains=1) == want, (n, p)


@pytest.mark.parametrize("threads,chains", [(128, 1), (128, 2), (128, 4), (256, 1), (256, 2), (256, 4),
                                            (512, 1), (512, 2)])
@pytest.mark.parametrize("chunk", [1, 7, 16, 100, 1024])
def test_launch_shapes(threads, chains, chunk):
    for name in ("ac_set", "r5", "even_odd5"):
        d = AUTOMATA[name]()
        a = sfa_mod().Automaton.from_dfa(d)
        t = text_for(d, 200_003, seed=chunk)
        assert gpu_match(a, t, block_threads=threads, chains=chains, chunk_bytes=chunk) == expect(d, t), name


SMALL_LENS = [0, 1, 2, 15, 16, 17, 31, 63, 64, 65, 1000, 1023, 1024, 1025, 16383, 16384, 16385, 16400,
              16401, 32768, 49151, 65519, 65535, 65536]


@pytest.mark.parametrize("name", sorted(AUTOMATA))
def test_short_texts_one_cta(name):
    """Texts up to 16 KiB with the automatic shape take the one-CTA kernel
    (no scratch, no look-back), longer ones up to 1 MiB a cluster of such
    CTAs: every length around the chunk sizes (16 to 64 bytes per thread),
    the one-CTA limit and the first cluster sizes, start offsets modulo 16,
    and Lemma 1 streaming with short pieces.  Simulation-mode handles and
    explicit shapes keep the persistent kernel."""
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    a = sfa.Automaton.from_dfa(d)
    base = text_for(d, (64 << 10) + 64, seed=len(name))
    dev = torch.from_numpy(base).cuda()
    for n in SMALL_LENS:
        for off in (0, 1, 7, 15):
            if off + n > base.size:
                continue
            out = a.match(dev[off:off + n])
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == expect(d, base[off:off + n]), (name, n, off)
    # Lemma 1 pieces of a few hundred bytes, then one past the limit
    cuts = [0, 5, 300, 301, 4000, 20000, 65536 + 3, base.size]
    out = a.match(dev[:cuts[1]])
    for i in range(1, len(cuts) - 1):
        a.match_continue(dev[cuts[i]:cuts[i + 1]], out)
    torch.cuda.synchronize()
    assert sfa.decode(out)[0] == expect(d, base)


def _perm7():
    """Sum of the bytes mod 7: every symbol permutes the states, so no chunk
    mapping is ever constant (every group and CTA aggregate is a vector)."""
    q = np.arange(7, dtype=np.int64)[:, None]
    b = np.arange(256, dtype=np.int64)[None, :]
    acc = np.zeros(7, np.uint8)
    acc[0] = 1
    return W.DFA(((q + b) % 7).astype(np.int32), 0, acc, bytes(range(97, 105)), name="perm7")


CLUSTER_LENS = [16385, 20000, 32769, 65537, 100_003, 131_072, 262_147, 524_287, (1 << 20) - 1, 1 << 20]


@pytest.mark.parametrize("name", ["ac_set", "r5", "ra2", "T4", "rand8", "one_state", "single", "perm7"])
def test_short_texts_cluster(name):
    """Texts of 16 KiB to 1 MiB take the cluster form of the short-text
    kernel (2 to 16 CTAs exchanging their aggregates through distributed
    shared memory): lengths from just past one CTA to the 1 MiB limit and
    just past it (the persistent kernel), unaligned starts, and Lemma 1
    streaming across pieces of cluster size.  perm7 keeps every aggregate a
    |Q|-vector; ac_set's are constants; r5/ra2's point and set-point
    mappings."""
    sfa = sfa_mod()
    d = _perm7() if name == "perm7" else AUTOMATA[name]()
    a = sfa.Automaton.from_dfa(d)
    base = text_for(d, (1 << 20) + 4096, seed=len(name) + 11)
    dev = torch.from_numpy(base).cuda()
    for n in CLUSTER_LENS + [(1 << 20) + 1]:
        for off in (0, 9):
            if off + n > base.size:
                continue
            out = a.match(dev[off:off + n])
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == expect(d, base[off:off + n]), (name, n, off)
    cuts = [0, 3, 40_000, 40_001, 300_000, 300_016, 1_000_000, base.size]
    out = a.match(dev[:cuts[1]])
    for i in range(1, len(cuts) - 1):
        a.match_continue(dev[cuts[i]:cuts[i + 1]], out)
    torch.cuda.synchronize()
    assert sfa.decode(out)[0] == expect(d, base)


@pytest.mark.parametrize("name", ["ab_star", "r5", "ac_set", "T4", "rand8", "kmp", "one_state"])
@pytest.mark.parametrize("n", [0, 1, 33, 4096, 100_003, 1 << 21])
def test_tilings_agree(name, n):
    """Warp tiles and CTA tiles: the same results as the oracle."""
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    a = sfa.Automaton.from_dfa(d)
    t = text_for(d, n, seed=n + 3)
    want = expect(d, t)
    for tiling in (sfa.TILING_WARP, sfa.TILING_CTA):
        for threads in (256, 512, 1024):
            for chunk in (0, 16, 64, 1000):
                got = gpu_match(a, t, block_threads=threads, chains=1, chunk_bytes=chunk, tiling=tiling)
                assert got == want, (tiling, threads, chunk)


@pytest.mark.parametrize("name", ["rand8", "T4", "even_odd5", "r3"])
def test_tilings_agree_simulation(name):
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    a = sfa.Automaton(d.delta, d.q0, d.accept, mode=sfa.MODE_SIM)
    for n in (0, 77, 70_001, 1 << 20):
        t = text_for(d, n, seed=n + 5)
        want = expect(d, t)
        for tiling in (sfa.TILING_WARP, sfa.TILING_CTA):
            for threads in (128, 256):
                for chunk in (0, 16, 4096):
                    got = gpu_match(a, t, block_threads=threads, chains=1, chunk_bytes=chunk, tiling=tiling)
                    assert got == want, (tiling, threads, chunk, n)


@pytest.mark.parametrize("n", [80 << 20, (96 << 20) + 4093])
def test_two_level_text(n):
    """Long texts with automatic chunks take two levels of chunk lengths;
    also unaligned (level B then has no tensor map) and under max_ctas."""
    sfa = sfa_mod()
    d, t = W.workload_large(n)
    a = sfa.Automaton.from_dfa(d)
    want = expect(d, t)
    assert gpu_match(a, t) == want
    buf = torch.from_numpy(np.concatenate([np.zeros(3, np.uint8), t])).cuda()
    out = a.match(buf[3:])
    torch.cuda.synchronize()
    assert sfa.decode(out)[0] == want
    assert gpu_match(a, t, max_ctas=100) == want


@pytest.mark.parametrize("rn", [5, 50])
def test_rn_accepted_texts(rn):
    """Sect. VI-B's automata on accepted texts (the chunk mappings never
    become constant; the count pass reruns most of each chunk), clean and
    with a few wrong digits; default, CTA/warp tilings and a two-level size."""
    sfa = sfa_mod()
    d = W.dfa_rn(rn)
    a = sfa.Automaton.from_dfa(d)
    for n, flips in ((8 << 20, 0), ((8 << 20) + 7, 5), (96 << 20, 0)):
        t = W.text_rn_accepted(n, rn, 11 + n)
        if flips:
            rng = np.random.default_rng(n)
            t[rng.integers(0, n, flips)] = ord("7")
        want = expect(d, t)
        assert gpu_match(a, t) == want, n
        if n < (64 << 20):
            assert gpu_match(a, t, tiling=sfa.TILING_WARP, block_threads=512, chains=1) == want
            assert gpu_match(a, t, block_threads=256, chains=2, chunk_bytes=1000) == want


def test_warp_tiles_with_max_ctas():
    """Warp-tile look-back over thousands of tiles with few resident CTAs."""
    sfa = sfa_mod()
    for name in ("r5", "ac_set", "T4"):
        d = AUTOMATA[name]()
        a = sfa.Automaton.from_dfa(d)
        t = text_for(d, 300_000, seed=1)
        for ctas in (1, 2, 7):
            got = gpu_match(a, t, chunk_bytes=16, block_threads=256, chains=1, max_ctas=ctas,
                            tiling=sfa.TILING_WARP)
            assert got == expect(d, t)


def test_many_tiles_with_max_ctas():
    """Look-back over hundreds of tiles with few resident CTAs."""
    for name in ("r5", "ac_set", "T4"):
        d = AUTOMATA[name]()
        a = sfa_mod().Automaton.from_dfa(d)
        t = text_for(d, 300_000, seed=1)
        for ctas in (1, 2, 7):
            assert gpu_match(a, t, chunk_bytes=16, block_threads=128, chains=1, max_ctas=ctas) == expect(d, t)


@pytest.mark.parametrize("offset", range(16))
def test_unaligned_text(offset):
    d = AUTOMATA["ac_set"]()
    a = sfa_mod().Automaton.from_dfa(d)
    base = text_for(d, 100_000, seed=2)
    buf = torch.from_numpy(base).cuda()
    for n in (0, 1, 17, 4095, 60_000):
        view = buf[offset:offset + n]
        out = a.match(view, chunk_bytes=48)
        torch.cuda.synchronize()
        assert sfa_mod().decode(out)[0] == expect(d, base[offset:offset + n])


@pytest.mark.parametrize("offset", [1, 3, 8, 15])
def test_unaligned_text_automatic_chunks(offset):
    """Texts that start off a 16-byte boundary: the chunks are anchored at
    the first boundary (chunk 0 takes the bytes before it), so the tensor
    maps cover them too.  Lengths shorter than, equal to and just past the
    origin, several tiles with a ragged tail, both tilings, forced chunk
    counts (no anchoring) and the simulation path."""
    sfa = sfa_mod()
    for name in ("ac_set", "r5", "T4"):
        d = AUTOMATA[name]()
        a = sfa.Automaton.from_dfa(d)
        base = text_for(d, (3 << 20) + 64, seed=offset)
        buf = torch.from_numpy(base).cuda()
        org = (16 - offset) % 16
        for n in (0, 1, org - 1, org, org + 1, 4095, 600_001, (3 << 20) + 7):
            if n < 0:
                continue
            want = expect(d, base[offset:offset + n])
            view = buf[offset:offset + n]
            for launch in ({}, {"tiling": sfa.TILING_WARP}, {"chunk_bytes": 64}, {"chunk_bytes": 48},
                           {"forced_chunks": 37}, {"block_threads": 128, "chains": 2, "chunk_bytes": 256}):
                out = a.match(view, **launch)
                torch.cuda.synchronize()
                assert sfa.decode(out)[0] == want, (name, n, launch)
    d = AUTOMATA["rand8"]()
    a = sfa.Automaton(d.delta, d.q0, d.accept, mode=sfa.MODE_SIM)
    base = text_for(d, 700_064, seed=offset)
    buf = torch.from_numpy(base).cuda()
    for n in (5, 70_001, 700_000):
        out = a.match(buf[offset:offset + n])
        torch.cuda.synchronize()
        assert sfa.decode(out)[0] == expect(d, base[offset:offset + n]), n


def test_batch_of_unaligned_views():
    """A batch of views at every offset of one buffer (texts shorter than
    their origin included), alone and in the mix, with its CUDA graph."""
    sfa = sfa_mod()
    autos_d = W.workload_batch_automata(3) + [W.dfa_rn(3)]
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    rng = np.random.default_rng(7)
    lens = [int(x) for x in rng.integers(0, 20, 12)] + [int(x) for x in rng.integers(100, 3 << 20, 36)]
    gaps = rng.integers(0, 16, len(lens))
    total = int(sum(lens) + gaps.sum()) + 16
    big = W.text_uniform(total, W.LOWER_ALPHABET, 99)
    dev = torch.from_numpy(big).cuda()
    views, hs, want, pos = [], [], [], 1
    for i, n in enumerate(lens):
        pos += int(gaps[i])
        j = i % len(autos)
        views.append(dev[pos:pos + n])
        hs.append(autos[j])
        want.append(expect(autos_d[j], big[pos:pos + n]))
        pos += n
    b = sfa.Batch(hs, views)
    for graph in (False, True, True):
        out = torch.zeros(16 * len(views), dtype=torch.uint8, device="cuda")
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        assert sfa.decode(out) == want
    for i in range(0, len(views), 5):
        out = hs[i].match(views[i])
        torch.cuda.synchronize()
        assert sfa.decode(out)[0] == want[i], i


def test_state_numberings_agree():
    """The breadth-first numbering, the one chosen against bank conflicts by
    the uniform model and the one chosen on a text sample all give the
    oracle's results: alone, in a batch, and on a two-level text."""
    sfa = sfa_mod()
    d, t = W.workload_large(80 << 20)
    cases = [(d, t)] + [(x, text_for(x, 3 << 20, seed=i)) for i, x in enumerate(W.workload_batch_automata(4))]
    cases.append((W.dfa_rn(5), W.text_rn_accepted(2 << 20, 5, 3)))
    for dd, tt in cases:
        want = expect(dd, tt)
        autos = [sfa.Automaton.from_dfa(dd, bank_tune=False), sfa.Automaton.from_dfa(dd),
                 sfa.Automaton.from_dfa(dd, sample=tt[:1 << 20])]
        dev = torch.from_numpy(tt).cuda()
        for a in autos:
            out = a.match(dev)
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == want
        views = [dev[:1000], dev[1000:1 << 20], dev[(1 << 20) + 5:]]
        b = sfa.Batch(autos, views)
        out = b.launch()
        torch.cuda.synchronize()
        got = sfa.decode(out)
        for v, (lo, hi) in enumerate(((0, 1000), (1000, 1 << 20), ((1 << 20) + 5, tt.size))):
            assert got[v] == expect(dd, tt[lo:hi]), v


@pytest.mark.parametrize("name", ["r3", "r5", "ra2", "even_odd5", "ab_star"])
def test_point_mappings(name):
    """Automata with an absorbing non-final state: chunk mappings of one live
    state (the rest dead) are followed through the DFA rows and counted for
    their source state only.  Texts from cleanly accepted to random (chunks
    that die into the sink early, late, or never), every tiling, short
    chunks, forced chunk counts, and a batch."""
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    a = sfa.Automaton.from_dfa(d)
    alpha = np.frombuffer(d.alphabet, np.uint8)
    rng = np.random.default_rng(len(name))
    texts = []
    for n, rate in (((1 << 20) + 11, 0), ((1 << 20) + 3, 1 / 5000), (600_001, 1 / 300), (300_007, 1 / 20),
                    (200_003, 1.0)):
        t = text_for(d, n, seed=n)
        flips = rng.random(n) < rate
        t[flips] = alpha[rng.integers(0, alpha.size, int(flips.sum()))]
        texts.append(t)
    for t in texts:
        want = expect(d, t)
        for launch in ({}, {"tiling": sfa.TILING_WARP}, {"tiling": sfa.TILING_CTA, "chunk_bytes": 100},
                       {"chunk_bytes": 16, "block_threads": 128, "chains": 2}, {"forced_chunks": 64}):
            assert gpu_match(a, t, **launch) == want, (name, t.size, launch)
    dev = [torch.from_numpy(t).cuda() for t in texts]
    out = sfa.Batch([a] * len(dev), dev).launch()
    torch.cuda.synchronize()
    assert sfa.decode(out) == [expect(d, t) for t in texts]


def test_literal_boundaries_inside_chunks():
    """Plants straddling chunk and tile boundaries."""
    lit = b"needle!"
    d = W.dfa_kmp(lit)
    a = sfa_mod().Automaton.from_dfa(d)
    t = W.text_uniform(1 << 16, W.LOWER_ALPHABET, 5)
    for chunk in (16, 64, 256):
        for s in range(chunk - len(lit) + 1, chunk + 1):
            t2 = t.copy()
            for base in range(0, len(t2) - 2 * chunk, 7 * chunk):
                t2[base + s:base + s + len(lit)] = np.frombuffer(lit, np.uint8)
            assert gpu_match(a, t2, chunk_bytes=chunk, block_threads=128, chains=1) == expect(d, t2)


# ---------------------------------------------------------------------------
# simulation mode (Alg. 3 vectors)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("idx", range(3))
def test_simulation_random_dfas(idx):
    d = W.workload_sim_automata()[idx]
    a = sfa_mod().Automaton.from_dfa(d)
    assert a.info()["mode"] == sfa_mod().MODE_SIM
    t = W.text_uniform((1 << 22) + 5, bytes(range(16)), 100 + idx)
    assert gpu_match(a, t) == expect(d, t)
    for chunk in (64, 1000, 8192):
        assert gpu_match(a, t[:300_001], chunk_bytes=chunk) == expect(d, t[:300_001])


@pytest.mark.parametrize("name", ["ab_star", "r3", "T4", "kmp", "rand8", "even_odd5", "one_state"])
def test_forced_simulation_small(name):
    """Forced simulation, including chunks that never converge (r3 and T4
    contain permutations), exercises the chunk-vector scan."""
    d = AUTOMATA[name]()
    a = sfa_mod().Automaton.from_dfa(d, mode=sfa_mod().MODE_SIM)
    assert a.info()["mode"] == sfa_mod().MODE_SIM
    for n in (0, 1, 33, 5000, 100_003):
        t = text_for(d, n, seed=n)
        want = expect(d, t)
        assert gpu_match(a, t) == want
        assert gpu_match(a, t, chunk_bytes=16, block_threads=128, chains=1) == want
        assert gpu_match(a, t, chunk_bytes=40, block_threads=128, chains=2) == want
    t = text_for(d, 2000, seed=9)
    for p in range(1, 65):
        assert gpu_match(a, t, forced_chunks=p) == expect(d, t)


@pytest.mark.parametrize("nq", [65, 100, 128, 200, 256])
def test_simulation_large_random_dfas(nq):
    """Alg. 3 past 64 states: vectors of 128 and 256 entries in shared
    memory.  Random complete DFAs over 16 symbols, 1 MiB and 256 MiB, the
    automatic shape, short chunks (many chunks still a vector at their end,
    combined through their scratch vectors) and forced chunk counts."""
    sfa = sfa_mod()
    d = W.dfa_random(nq, 16, seed=1405004 + nq)
    a = sfa.Automaton.from_dfa(d)
    assert a.info()["mode"] == sfa.MODE_SIM
    t = W.text_uniform(256 << 20, bytes(range(16)), 77 + nq)
    assert gpu_match(a, t) == expect(d, t)
    small = t[:(1 << 20) + 7]
    want = expect(d, small)
    assert gpu_match(a, small) == want
    for launch in ({"chunk_bytes": 64}, {"chunk_bytes": 1000}, {"forced_chunks": 37}, {"forced_chunks": 1},
                   {"block_threads": 128, "chains": 1, "chunk_bytes": 256}):
        assert gpu_match(a, small, **launch) == want, launch


@pytest.mark.parametrize("nq", [100, 200, 256])
def test_simulation_permutations_never_converge(nq):
    """A cycle automaton forced into simulation mode: every chunk vector is
    a rotation to its end (no chunk ever becomes constant), so every chunk
    is combined through its scratch vector."""
    sfa = sfa_mod()
    delta = np.tile((np.arange(nq, dtype=np.int32)[:, None] + 1) % nq, (1, 256))
    delta[:, ord("b")] = (np.arange(nq, dtype=np.int32) + 2) % nq
    acc = (np.arange(nq) % 7 == 3).astype(np.uint8)
    d = W.DFA(delta, 0, acc, b"ab", name=f"cycle{nq}")
    a = sfa.Automaton.from_dfa(d, mode=sfa.MODE_SIM)
    t = text_for(d, (1 << 20) + 3, seed=nq)
    want = expect(d, t)
    for launch in ({}, {"chunk_bytes": 64}, {"forced_chunks": 64}):
        assert gpu_match(a, t, **launch) == want, launch


def test_full_transformation_6():
    """The generators of the full transformation monoid T_6 (Fact 2): the
    D-SFA has 6^6 = 46656 states (under the default cap, so D-SFA mode with
    its non-constant rows in L2), and the same DFA in simulation mode."""
    sfa = sfa_mod()
    d = W.dfa_full_transformation(6)
    a = sfa.Automaton.from_dfa(d)
    assert a.info()["mode"] == sfa.MODE_SFA and a.info()["n_sfa_states"] == 6 ** 6
    s = sfa.Automaton.from_dfa(d, mode=sfa.MODE_SIM)
    t = text_for(d, (16 << 20) + 5, seed=6)
    want = expect(d, t)
    for h in (a, s):
        assert gpu_match(h, t) == want
        assert gpu_match(h, t[:100_001], chunk_bytes=64) == expect(d, t[:100_001])
        for p in (1, 7, 64):
            assert gpu_match(h, t[:30_001], forced_chunks=p) == expect(d, t[:30_001])


# ---------------------------------------------------------------------------
# 16-bit state ids (more than 256 reachable states)
# ---------------------------------------------------------------------------

def _wide_ac():
    """An Aho-Corasick automaton of 40 seeded literals over a-z: 308 states,
    synchronising (its chunks become constant mappings)."""
    rng = np.random.default_rng(5)
    lits = [bytes(rng.choice(list(W.LOWER_ALPHABET), size=int(rng.integers(6, 11))).tolist()) for _ in range(40)]
    return W.dfa_aho_corasick(lits)


def _wide_cycle(nq=300):
    """A permutation automaton without a sink: its D-SFA is nq rotations,
    all stored, and no chunk ever becomes constant."""
    delta = np.tile((np.arange(nq, dtype=np.int32)[:, None] + 1) % nq, (1, 256))
    delta[:, ord("b")] = (np.arange(nq, dtype=np.int32) + 7) % nq
    acc = (np.arange(nq) % 11 == 4).astype(np.uint8)
    return W.DFA(delta, 0, acc, b"ab", name=f"cycle{nq}")


WIDE = {
    "r128": lambda: W.dfa_rn(128),
    "r500": lambda: W.dfa_rn(500),
    "ra500": lambda: W.dfa_ra(500),
    "ac308": _wide_ac,
    "cycle300": _wide_cycle,
}


def _wide_texts(name, d, n, seed):
    """Accepted r_n / r_a texts with errors at several rates (chunks that die
    into the sink early, late or never), uniform text otherwise."""
    rng = np.random.default_rng(seed)
    if name.startswith("r"):
        rn = 128 if name == "r128" else 500
        base = W.text_rn_accepted(n, rn, seed)
        out = [base.copy()]
        for rate in (1 / 200_000, 1 / 3000, 1 / 50):
            t = base.copy()
            flips = rng.random(n) < rate
            t[flips] = np.frombuffer(b"0123456789a", np.uint8)[rng.integers(0, 11, int(flips.sum()))]
            out.append(t)
        return out
    alpha = np.frombuffer(d.alphabet, np.uint8)
    return [alpha[rng.integers(0, alpha.size, n)]]


@pytest.mark.parametrize("name", sorted(WIDE))
def test_wide_ids(name):
    """Automata past 256 states: 16-bit ids, class-indexed DFA rows in
    shared memory, point mappings followed without being stored.  Automatic
    shape (two levels on the longer texts), CTA shapes, short chunks, forced
    chunk counts, unaligned views and Lemma 1 streaming."""
    sfa = sfa_mod()
    d = WIDE[name]()
    a = sfa.Automaton.from_dfa(d)
    info = a.info()
    assert info["id_bits"] == 16 and info["mode"] == sfa.MODE_SFA
    for t in _wide_texts(name, d, (24 << 20) + 5, seed=len(name)):
        want = expect(d, t)
        dev = torch.from_numpy(t).cuda()
        for launch in ({}, {"block_threads": 256, "chains": 2, "chunk_bytes": 4096}, {"chunk_bytes": 100},
                       {"forced_chunks": 61}):
            out = a.match(dev, **launch)
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == want, (name, launch)
        small = t[:200_003]
        for launch in ({"block_threads": 128, "chains": 1, "chunk_bytes": 16}, {"forced_chunks": 1}):
            assert gpu_match(a, small, **launch) == expect(d, small), launch
        for off in (1, 7):
            out = a.match(dev[off:off + 3_000_001])
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == expect(d, t[off:off + 3_000_001])
        out = a.match(dev[:(5 << 20) + 3])
        a.match_continue(dev[(5 << 20) + 3:], out)
        torch.cuda.synchronize()
        assert sfa.decode(out)[0] == want
        for n in (0, 1, 999):
            assert gpu_match(a, t[:n]) == expect(d, t[:n])


def test_wide_ids_full_size():
    """r_500 on 1 GiB of an accepted text and r_a on 1 GiB of 'a' (the
    paper's Sect. VI-B workloads), in the bench's launch configuration."""
    sfa = sfa_mod()
    d = W.dfa_rn(500)
    t = W.text_rn_accepted(1 << 30, 500, 1405500)
    got = gpu_match(sfa.Automaton.from_dfa(d), t)
    assert got == expect(d, t) and got[3] == (1 << 30) // 1000
    d = W.dfa_ra(500)
    t = np.full(1 << 30, ord("a"), dtype=np.uint8)
    got = gpu_match(sfa.Automaton.from_dfa(d), t)
    assert got == expect(d, t) and got[3] == 1 << 30


def test_wide_ids_in_batches_and_noalloc():
    """A batch mixing byte-id and 16-bit-id automata (the latter matched by
    per-text launches), and the no-allocation entry on a 16-bit-id handle."""
    sfa = sfa_mod()
    ds = [W.dfa_rn(128), _wide_ac(), AUTOMATA["ac_set"](), W.dfa_rn(5)]
    autos = [sfa.Automaton.from_dfa(d) for d in ds]
    texts, hs, want = [], [], []
    for i, n in enumerate((0, 1000, 1 << 20, 77_777, 3 << 20, 5)):
        j = i % len(ds)
        t = _wide_texts("r128", ds[j], n, i)[0] if j in (0, 3) else text_for(ds[j], n, seed=i)
        if j == 3:
            t = W.text_rn_accepted(n, 5, i)
        texts.append(torch.from_numpy(t).cuda())
        hs.append(autos[j])
        want.append(expect(ds[j], t))
    b = sfa.Batch(hs, texts)
    for graph in (False, True):
        out = torch.zeros(16 * len(texts), dtype=torch.uint8, device="cuda")
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        assert sfa.decode(out) == want
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    a = autos[0]
    a.match_noalloc(texts[4], out)
    torch.cuda.synchronize()
    assert sfa.decode(out)[0] == want[4]


# ---------------------------------------------------------------------------
# streaming (Lemma 1), host path, batches, timeouts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["ac_set", "r5", "rand8"])
def test_match_continue_pieces(name):
    d = AUTOMATA[name]()
    a = sfa_mod().Automaton.from_dfa(d)
    t = text_for(d, 500_000, seed=4)
    tt = torch.from_numpy(t).cuda()
    rng = np.random.default_rng(0)
    cuts = np.sort(rng.integers(0, len(t), 9)).tolist()
    bounds = [0] + cuts + [len(t)]
    out = a.match(tt[:bounds[1]])
    for i in range(1, len(bounds) - 1):
        a.match_continue(tt[bounds[i]:bounds[i + 1]], out, chunk_bytes=64)
    torch.cuda.synchronize()
    assert sfa_mod().decode(out)[0] == expect(d, t)


def _oracle_map(d, text):
    """delta^(q, text) for every state reachable from q0, -1 for the rest
    (Alg. 2 from each state)."""
    seen, todo = {d.q0}, [d.q0]
    while todo:
        q = todo.pop()
        for t in np.unique(d.delta[q]):
            if int(t) not in seen:
                seen.add(int(t))
                todo.append(int(t))
    m = np.full(d.nq, -1, dtype=np.int32)
    for q in seen:
        m[q] = oracle.dfa_run(d.delta, d.q0, d.accept, text, start=q)[0]
    return m


@pytest.mark.parametrize("name", ["ac_set", "r5", "rand8", "T4", "kmp", "ab_star", "one_state"])
def test_match_map_equals_oracle(name):
    """sfa_match_map: the slice mapping over every kept state (Lemma 1) and
    the result from q0, for short and long texts (two levels), CTA shapes,
    forced chunk counts, an unaligned view and the simulation path."""
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    handles = [sfa.Automaton.from_dfa(d)]
    if name in ("rand8", "T4", "r5"):
        handles.append(sfa.Automaton.from_dfa(d, mode=sfa.MODE_SIM))
    base = text_for(d, (24 << 20) + 77, seed=11)
    dev = torch.from_numpy(base).cuda()
    for lo, hi in ((0, 0), (0, 1), (3, 4099), (0, 1 << 20), (5, (24 << 20) + 77)):
        t = base[lo:hi]
        want_map = _oracle_map(d, t)
        want = expect(d, t)
        for a in handles:
            for launch in ({}, {"chunk_bytes": 64, "block_threads": 128, "chains": 2}, {"forced_chunks": 33}):
                out, m = a.match_map(dev[lo:hi], **launch)
                torch.cuda.synchronize()
                assert sfa.decode(out)[0] == want, (lo, hi, launch)
                assert np.array_equal(m.cpu().numpy(), want_map), (lo, hi, launch)


def test_match_map_then_continue_splits_a_text():
    """The split of one text on one device: the mappings of the slices
    before a slice give its entering state; sfa_match_continue from there
    gives its count; the sum and the last final state are the text's."""
    from paper_1405_0562_gb300 import split
    sfa = sfa_mod()
    for d, t in (W.workload_large(64 << 20), (W.dfa_rn(5), W.text_rn_accepted(8 << 20, 5, 1))):
        a = sfa.Automaton.from_dfa(d)
        dev = torch.from_numpy(t).cuda()
        cuts = [0, 1000, 1000, (3 << 20) + 5, t.size - 17, t.size]
        maps, outs = [], []
        for i in range(len(cuts) - 1):
            o, m = a.match_map(dev[cuts[i]:cuts[i + 1]])
            maps.append(m.cpu().numpy())
            outs.append(o)
        s = split.entering_states(maps, d.q0)
        total = 0
        for i in range(len(cuts) - 1):
            rec = torch.from_numpy(split.result_record(s[i])).cuda()
            a.match_continue(dev[cuts[i]:cuts[i + 1]], rec)
            torch.cuda.synchronize()
            f, acc, st, c = sfa.decode(rec)[0]
            assert st == 0
            total += c
        assert (f, acc, 0, total) == expect(d, t)


def test_match_host_pinned_and_pageable():
    d, t = W.workload_large(150 << 20)   # several 64 MiB pieces
    a = sfa_mod().Automaton.from_dfa(d)
    want = expect(d, t)
    assert a.match_host(t) == want
    pinned = torch.from_numpy(t).pin_memory()
    assert a.match_host(pinned) == want
    assert a.match_host(t[:0]) == expect(d, t[:0])


@pytest.mark.parametrize("name", ["ac_set", "r5", "rand8", "one_state"])
def test_match_host_short_pinned_in_place(name):
    """Short pinned texts (up to 256 KiB) are read in place by the short-text
    kernel (no staging copy): every length class up to and past 1 MiB, unaligned starts,
    a pageable copy of each and an explicit shape (the copying path) agree
    with the oracle; the next call on the same handle is unaffected."""
    sfa = sfa_mod()
    d = AUTOMATA[name]()
    a = sfa.Automaton.from_dfa(d)
    base = text_for(d, (1 << 20) + 64, seed=5)
    pinned = torch.from_numpy(base).pin_memory()
    for n in (1, 15, 1000, 16384, 16385, 65537, 300_001, 1 << 20, (1 << 20) + 1):
        for off in (0, 3):
            if off + n > base.size:
                continue
            want = expect(d, base[off:off + n])
            assert a.match_host(pinned[off:off + n]) == want, (name, n, off)
            assert a.match_host(base[off:off + n]) == want, (name, n, off)
            assert a.match_host(pinned[off:off + n], block_threads=256, chains=1) == want, (name, n, off)


def test_batch_mixed_and_graph():
    sfa = sfa_mod()
    autos_d = W.workload_batch_automata(4) + [W.dfa_rn(3), W.workload_sim_automata()[0]]
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    rng = np.random.default_rng(3)
    lens = [0, 1, 16, 255, 256, 4097, 100_000, 1 << 20, 3, 70_001, 2 << 20, 999]
    texts, hs, ds = [], [], []
    for i, n in enumerate(lens):
        j = int(rng.integers(0, len(autos)))
        d = autos_d[j]
        texts.append(text_for(d, n, seed=i))
        hs.append(autos[j])
        ds.append(d)
    tt = [torch.from_numpy(x).cuda() for x in texts]
    want = [expect(d, x) for d, x in zip(ds, texts)]
    out = sfa.match_batch(hs, tt)
    torch.cuda.synchronize()
    assert sfa.decode(out) == want
    b = sfa.Batch(hs, tt)
    for graph in (False, True, True):
        out = torch.zeros(16 * len(lens), dtype=torch.uint8, device="cuda")
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        assert sfa.decode(out) == want
    # each result alone equals the result in the mix
    for i in range(len(lens)):
        assert gpu_match(hs[i], texts[i]) == want[i]


def test_batch_with_simulation_texts_in_persistent_launches():
    """Simulation-mode texts of a batch run in persistent launches too: one
    per vector size (16, 32, 64, 128, 256 entries) beside the D-SFA launch,
    whatever the number of texts; every result equals the oracle's, by plain
    launch and by CUDA graph."""
    sfa = sfa_mod()
    sims = [W.dfa_random(nq, 16, seed=50 + nq) for nq in (12, 30, 60, 100, 200)]
    dsfa = W.workload_batch_automata(2)
    autos_d = sims + dsfa
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    assert [a.info()["mode"] for a in autos] == [sfa.MODE_SIM] * 5 + [sfa.MODE_SFA] * 2
    rng = np.random.default_rng(11)
    lens = [0, 1, 15, 64, 1000, 4096, 70_001, 1 << 20, 3 << 20, 8 << 20]
    texts, hs, want = [], [], []
    for i in range(30):
        j = i % len(autos)
        n = lens[i % len(lens)]
        d = autos_d[j]
        t = text_for(d, n, seed=i) if j >= len(sims) else W.text_uniform(n, bytes(range(16)), 900 + i)
        texts.append(torch.from_numpy(t).cuda())
        hs.append(autos[j])
        want.append(expect(d, t))
    b = sfa.Batch(hs, texts)
    for graph in (False, True, True):
        out = torch.zeros(16 * len(texts), dtype=torch.uint8, device="cuda")
        n0 = sfa.kernel_launch_count()
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        assert sfa.decode(out) == want, graph
        assert sfa.kernel_launch_count() - n0 == 6        # one D-SFA launch, five vector sizes
    out = sfa.match_batch(hs, texts)
    torch.cuda.synchronize()
    assert sfa.decode(out) == want


def test_timeout_status_is_reported():
    """A tile that never publishes: its successor's bounded wait runs out,
    the launch completes and the result is flagged; the next launch is
    clean."""
    sfa = sfa_mod()
    d = AUTOMATA["r5"]()
    a = sfa.Automaton.from_dfa(d)
    t = text_for(d, 100_000, seed=1)
    import time
    t0 = time.time()
    got = gpu_match(a, t, chunk_bytes=16, block_threads=128, chains=1, timeout_us=50_000,
                    debug_flags=sfa.DEBUG_SKIP_PUBLISH)
    assert time.time() - t0 < 30
    assert got[2] == sfa.STATUS_TIMEOUT
    assert gpu_match(a, t, chunk_bytes=16, block_threads=128, chains=1) == expect(d, t)
    # the same with warp tiles: warp tile 1 never publishes
    t0 = time.time()
    got = gpu_match(a, t, chunk_bytes=16, block_threads=256, chains=1, timeout_us=50_000,
                    debug_flags=sfa.DEBUG_SKIP_PUBLISH, tiling=sfa.TILING_WARP)
    assert time.time() - t0 < 30
    assert got[2] == sfa.STATUS_TIMEOUT
    assert gpu_match(a, t, chunk_bytes=16, block_threads=256, chains=1, tiling=sfa.TILING_WARP) == expect(d, t)


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration bench.py times
# ---------------------------------------------------------------------------

def test_full_single_1MiB():
    d, t = W.workload_single()
    a = sfa_mod().Automaton.from_dfa(d)
    got = gpu_match(a, t)
    assert got == expect(d, t)
    assert got[3] == oracle.bruteforce_literal_count(d.literals, t) >= 64


def test_full_large_1GiB():
    d, t = W.workload_large()
    a = sfa_mod().Automaton.from_dfa(d)
    assert gpu_match(a, t) == expect(d, t)


def test_full_simulation_4GiB():
    t = W.workload_sim_text()
    tt = torch.from_numpy(t).cuda()
    for d in W.workload_sim_automata():
        a = sfa_mod().Automaton.from_dfa(d)
        out = a.match(tt)
        torch.cuda.synchronize()
        got = sfa_mod().decode(out)[0]
        assert got == expect(d, t), d.name
    del tt


def test_text_longer_than_2_32():
    """Texts of 2^32 + 2^20 + 13 bytes: 64-bit offsets and chunk positions,
    the two-level split of automatic chunks above 4 GiB, a count above 2^32
    (the one-state automaton whose every prefix is accepted: count = n), and
    Lemma 1 streaming with a piece boundary just below and exactly at 2^32.
    Every field against the oracle's Alg. 2, tolerance 0."""
    sfa = sfa_mod()
    n = (1 << 32) + (1 << 20) + 13
    t = W.workload_sim_text(n)
    one = AUTOMATA["one_state"]()
    sim16 = W.workload_sim_automata()[0]
    d_ac, t_ac = W.workload_large(n)
    for d, text in ((one, t), (sim16, t), (d_ac, t_ac)):
        want = expect(d, text)
        if d is one:
            assert want == (0, 1, 0, n)
        a = sfa.Automaton.from_dfa(d)
        tt = torch.from_numpy(text).cuda()
        launches = [{}, {"tiling": sfa.TILING_WARP}] if d is not sim16 else [{}]
        for launch in launches:
            out = a.match(tt, **launch)
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == want, (d.name, launch)
        for cut in ((1 << 32) - 7, 1 << 32):
            out = a.match(tt[:cut])
            a.match_continue(tt[cut:], out)
            torch.cuda.synchronize()
            assert sfa.decode(out)[0] == want, (d.name, cut)
        del tt
        torch.cuda.empty_cache()


def test_full_batch_4096_texts():
    from concurrent.futures import ThreadPoolExecutor
    sfa = sfa_mod()
    autos_d = W.workload_batch_automata()
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    lens = W.workload_batch_lengths()
    pair = W.workload_batch_pairing(len(lens), len(autos))
    total = int(lens.sum())
    big = W.text_uniform(total, W.LOWER_ALPHABET, W.SEED_BATCH + 2)
    offs = np.concatenate([[0], np.cumsum(lens)])
    dev = torch.from_numpy(big).cuda()
    texts = [dev[offs[i]:offs[i + 1]] for i in range(len(lens))]
    b = sfa.Batch([autos[p] for p in pair], texts)
    out = b.launch(graph=True)
    torch.cuda.synchronize()
    got = sfa.decode(out)

    def ref(i):
        d = autos_d[pair[i]]
        return expect(d, big[offs[i]:offs[i + 1]])

    with ThreadPoolExecutor(16) as ex:
        want = list(ex.map(ref, range(len(lens))))
    assert got == want
