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
