"""The launch-shape autotuner: its candidate list and cache on the CPU, and
on the GPU a tuning run whose every candidate must give the same result
(the tuner raises otherwise) and whose choice matches the oracle."""
import json

import numpy as np
import pytest

import workloads as W


def test_candidates_start_with_the_automatic_shape():
    from paper_1405_0562_gb300 import autotune
    info = {"mode": 1, "n_reachable": 127, "ncls": 56, "n_nonconst": 400}
    c = autotune.candidates(info, 1 << 30)
    assert c[0] == {}
    assert {"block_threads": 512, "chains": 1, "tiling": 2} in c
    # every other CTA shape also with the automatic chunk length (two levels)
    assert {"block_threads": 1024, "chains": 1} in c and {"block_threads": 256, "chains": 2} in c
    assert {"block_threads": 512, "chains": 1} not in c   # the automatic shape itself, listed first
    assert len({json.dumps(x, sort_keys=True) for x in c}) == len(c)
    sim = autotune.candidates({"mode": 2, "n_reachable": 16, "ncls": 16, "n_nonconst": 0}, 1 << 30)
    assert sim[0] == {} and all(x.get("block_threads", 128) in (128, 256) for x in sim)
    # a small text drops the chunk lengths that would hold it many times over
    small = autotune.candidates(info, 4096)
    assert all(x.get("chunk_bytes", 0) * x.get("block_threads", 1) * x.get("chains", 1) <= 2 * 4096
               or x.get("chunk_bytes", 0) == autotune.SFA_CHUNKS[0] for x in small)


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_1405_0562_gb300 import autotune
    monkeypatch.setenv("SFA_TUNE_CACHE", str(tmp_path / "tune.json"))
    autotune._store({"k": {"shape": {"chunk_bytes": 1024}, "ms": 1.0, "GBps": 2.0}})
    assert autotune._load()["k"]["shape"] == {"chunk_bytes": 1024}
    assert autotune.bucket(1) == 1 << 20 and autotune.bucket((1 << 24) + 1) == 1 << 25


@pytest.mark.gpu
def test_tune_agrees_with_the_oracle(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    import paper_1405_0562_gb300 as sfa
    from paper_1405_0562_gb300 import autotune
    monkeypatch.setenv("SFA_TUNE_CACHE", str(tmp_path / "tune.json"))
    d, t = W.workload_large(4 << 20)
    a = sfa.Automaton.from_dfa(d)
    tt = torch.from_numpy(t).cuda()
    shape = autotune.tune(a, tt, reps=2)
    assert autotune.cached(a, t.size) == shape
    out = a.match(tt, **shape)
    torch.cuda.synchronize()
    f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
    assert sfa.decode(out)[0] == (f, acc, 0, c)


def test_batch_key_and_candidates():
    """Batch plans are keyed by the automaton mix and a coarse length
    histogram; the candidates start with the default plan and never
    repeat."""
    from paper_1405_0562_gb300 import autotune
    infos = [{"mode": 1, "n_reachable": 60, "ncls": 20}, {"mode": 1, "n_reachable": 90, "ncls": 24}]
    k1 = autotune.batch_key(infos, [300, 5000, 1 << 20, 1 << 20], "dev")
    assert k1 == autotune.batch_key(infos[::-1], [1 << 20, 300, 1 << 20, 5000], "dev")   # order-free
    assert k1 != autotune.batch_key(infos[:1], [300, 5000, 1 << 20, 1 << 20], "dev")
    assert k1 != autotune.batch_key(infos, [300, 300, 300, 1 << 20], "dev")
    c = autotune.batch_candidates()
    assert c[0] == {} and len({json.dumps(x, sort_keys=True) for x in c}) == len(c)


@pytest.mark.gpu
def test_tune_batch_agrees_with_the_oracle(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    import paper_1405_0562_gb300 as sfa
    from paper_1405_0562_gb300 import autotune
    monkeypatch.setenv("SFA_TUNE_CACHE", str(tmp_path / "tune.json"))
    autos_d = W.workload_batch_automata(4)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    lens = W.workload_batch_lengths(96, hi=4 << 20)
    pair = W.workload_batch_pairing(len(lens), len(autos))
    big = W.text_uniform(int(lens.sum()), W.LOWER_ALPHABET, 12)
    offs = np.concatenate([[0], np.cumsum(lens)])
    dev = torch.from_numpy(big).cuda()
    texts = [dev[offs[i]:offs[i + 1]] for i in range(len(lens))]
    hs = [autos[p] for p in pair]
    shape = autotune.tune_batch(hs, texts, reps=1)
    assert autotune.tune_batch(hs, texts) == shape           # from the cache
    out = sfa.Batch(hs, texts, **shape).launch(graph=True)
    torch.cuda.synchronize()
    want = []
    for i in range(len(lens)):
        d = autos_d[pair[i]]
        f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, big[offs[i]:offs[i + 1]])
        want.append((f, acc, 0, c))
    assert sfa.decode(out) == want
