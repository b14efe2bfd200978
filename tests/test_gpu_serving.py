"""Continuous batching: reserved batch plans refilled with sfa_batch_update,
and the Server loop.  Every result must equal the text's result alone and
the oracle's (integers, tolerance 0)."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sfa():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1405_0562_gb300 as m
    m.lib()
    torch.cuda.set_device(0)
    return m


def expect(d, t):
    f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
    return (f, acc, 0, c)


def test_reserved_plan_refilled(sfa):
    autos_d = W.workload_serving_automata(6)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    nr_max = max(a.info()["n_reachable"] for a in autos)
    L = sfa.lib()
    opts = sfa.LaunchOpts(512, 256, 2, 0, 0, 0, 0, 0)
    plan = ctypes.c_void_p()
    assert L.sfa_batch_reserve(64, 4096, nr_max, ctypes.byref(opts), ctypes.byref(plan)) == sfa.OK
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(1)
    try:
        for rnd in range(5):
            k = int(rng.integers(1, 40))
            lens = [int(x) for x in rng.integers(0, 300_000, k)]
            which = [int(x) for x in rng.integers(0, len(autos), k)]
            texts = [W.text_uniform(n, W.LOWER_ALPHABET, 100 * rnd + i) for i, n in enumerate(lens)]
            dev = [torch.from_numpy(t).cuda() for t in texts]
            hs = (ctypes.c_void_p * k)(*[autos[j].handle.value for j in which])
            ptrs = (ctypes.c_void_p * k)(*[x.data_ptr() if x.numel() else 0 for x in dev])
            ln = (ctypes.c_uint64 * k)(*lens)
            out = torch.zeros(16 * 64, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            assert L.sfa_batch_update(plan, hs, ptrs, ln, k, stream.cuda_stream) == sfa.OK
            fn = L.sfa_batch_graph_launch if rnd % 2 else L.sfa_batch_launch
            assert fn(plan, out.data_ptr(), stream.cuda_stream) == sfa.OK
            stream.synchronize()
            got = sfa.decode(out[:16 * k])
            assert got == [expect(autos_d[j], t) for j, t in zip(which, texts)], rnd
    finally:
        L.sfa_batch_destroy(plan)


def test_reserved_plan_refilled_from_host(sfa):
    """sfa_batch_update_host: pinned host texts copied into a device arena
    and matched by the refilled plan, several rounds on one stream."""
    autos_d = W.workload_serving_automata(5)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    nr_max = max(a.info()["n_reachable"] for a in autos)
    L = sfa.lib()
    opts = sfa.LaunchOpts(1024, 512, 1, 0, 0, 0, 0, 0)
    plan = ctypes.c_void_p()
    assert L.sfa_batch_reserve(64, 8192, nr_max, ctypes.byref(opts), ctypes.byref(plan)) == sfa.OK
    stream = torch.cuda.Stream()
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(2)
    try:
        for rnd in range(4):
            k = int(rng.integers(1, 50))
            lens = [int(x) for x in rng.integers(0, 500_000, k)]
            which = [int(x) for x in rng.integers(0, len(autos), k)]
            texts = [torch.from_numpy(W.text_uniform(n, W.LOWER_ALPHABET, 70 * rnd + i)).pin_memory()
                     for i, n in enumerate(lens)]
            offs = np.concatenate([[0], np.cumsum([(n + 255) // 256 * 256 for n in lens])])
            assert offs[-1] <= arena.numel()
            hs = (ctypes.c_void_p * k)(*[autos[j].handle.value for j in which])
            src = (ctypes.c_void_p * k)(*[t.data_ptr() if t.numel() else 0 for t in texts])
            dst = (ctypes.c_void_p * k)(*[arena.data_ptr() + int(o) for o in offs[:k]])
            ln = (ctypes.c_uint64 * k)(*lens)
            out = torch.zeros(16 * 64, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            assert L.sfa_batch_update_host(plan, hs, src, dst, ln, k, stream.cuda_stream) == sfa.OK
            assert L.sfa_batch_launch(plan, out.data_ptr(), stream.cuda_stream) == sfa.OK
            stream.synchronize()
            got = sfa.decode(out[:16 * k])
            assert got == [expect(autos_d[j], t.numpy()) for j, t in zip(which, texts)], rnd
        # NULL host pointer with a nonzero length: refused before any copy
        bad = (ctypes.c_void_p * 1)(0)
        one = (ctypes.c_uint64 * 1)(10)
        h1 = (ctypes.c_void_p * 1)(autos[0].handle.value)
        d1 = (ctypes.c_void_p * 1)(arena.data_ptr())
        assert L.sfa_batch_update_host(plan, h1, bad, d1, one, 1, stream.cuda_stream) == sfa.ERR_INVALID
    finally:
        L.sfa_batch_destroy(plan)


def test_reserved_plan_refuses_over_capacity(sfa):
    """A real text that needs more tiles than the plan holds is refused by
    sfa_batch_update (nothing is launched)."""
    d = W.workload_serving_automata(1)[0]
    a = sfa.Automaton.from_dfa(d)
    L = sfa.lib()
    opts = sfa.LaunchOpts(512, 256, 2, 0, 0, 0, 0, 0)
    plan = ctypes.c_void_p()
    assert L.sfa_batch_reserve(4, 2, a.info()["n_reachable"], ctypes.byref(opts), ctypes.byref(plan)) == sfa.OK
    stream = torch.cuda.Stream()
    try:
        t = torch.from_numpy(W.text_uniform(4 << 20, W.LOWER_ALPHABET, 3)).cuda()   # 16 tiles of 256 KiB
        hs = (ctypes.c_void_p * 1)(a.handle.value)
        ptrs = (ctypes.c_void_p * 1)(t.data_ptr())
        ln = (ctypes.c_uint64 * 1)(t.numel())
        assert L.sfa_batch_update(plan, hs, ptrs, ln, 1, stream.cuda_stream) == sfa.ERR_INVALID
        five = (ctypes.c_void_p * 5)(*([a.handle.value] * 5))
        p5 = (ctypes.c_void_p * 5)(*([t.data_ptr()] * 5))
        l5 = (ctypes.c_uint64 * 5)(*([16] * 5))
        assert L.sfa_batch_update(plan, five, p5, l5, 5, stream.cuda_stream) == sfa.ERR_INVALID   # > 4 texts
        stream.synchronize()
    finally:
        L.sfa_batch_destroy(plan)


def test_server_results_equal_alone(sfa):
    from paper_1405_0562_gb300 import serve
    autos_d = W.workload_serving_automata(8)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    arrivals, lens, which = W.workload_serving_requests(300, rate_per_s=20000.0, n_automata=len(autos),
                                                       median=16 << 10, cap=2 << 20)
    reqs = []
    for i in range(len(lens)):
        t = W.text_uniform(int(lens[i]), W.LOWER_ALPHABET, 7000 + i)
        reqs.append(serve.Request(i, int(which[i]), torch.from_numpy(t).pin_memory(), float(arrivals[i])))
    srv = serve.Server(autos, hbm_budget=64 << 20, max_batch=64, slots=3)
    try:
        done = srv.run(reqs)
    finally:
        srv.close()
    assert len(done) == len(reqs)
    assert srv.batches < len(reqs)          # requests were batched
    for r in done:
        t = r.text.numpy()
        assert r.result == expect(autos_d[r.automaton], t), r.rid
    # one request at a time gives the same results
    alone = serve.one_at_a_time(autos, [serve.Request(r.rid, r.automaton, r.text, 0.0) for r in done[:40]],
                                realtime=False)
    by_id = {r.rid: r.result for r in done}
    for r in alone:
        assert r.result == by_id[r.rid]
    # a 3 MiB arena and small batches: admission waits for memory, every
    # request still completes with the same result
    srv = serve.Server(autos, hbm_budget=3 << 20, max_batch=8, slots=2)
    try:
        again = srv.run([serve.Request(r.rid, r.automaton, r.text, 0.0) for r in done], realtime=False)
        st = srv.stats()
    finally:
        srv.close()
    assert len(again) == len(done) and st["queued"] == 0 and st["in_flight"] == 0 and st["arena_used"] == 0
    assert st["requests"] == len(done) and st["batches"] >= len(done) // 8
    for r in again:
        assert r.result == by_id[r.rid], r.rid


def test_copy_in_kernel_and_copies(sfa):
    """sfa_batch_update_host copies pinned texts with one kernel (same or
    different address modulo 16 on both sides; lengths around the 16-byte
    vectors and the 64 KiB units) and pageable texts with cudaMemcpyAsync:
    the arena holds exactly the host bytes afterwards and every result
    equals the oracle's."""
    autos_d = W.workload_serving_automata(3)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    nr_max = max(a.info()["n_reachable"] for a in autos)
    L = sfa.lib()
    opts = sfa.LaunchOpts(1024, 512, 1, 0, 0, 0, 0, 0)
    plan = ctypes.c_void_p()
    assert L.sfa_batch_reserve(64, 8192, nr_max, ctypes.byref(opts), ctypes.byref(plan)) == sfa.OK
    stream = torch.cuda.Stream()
    big = torch.from_numpy(W.text_uniform(16 << 20, W.LOWER_ALPHABET, 77)).pin_memory()
    arena = torch.zeros(32 << 20, dtype=torch.uint8, device="cuda")
    lens = [0, 1, 15, 16, 17, 100, 65535, 65536, 65537, 131072 + 3, 3 << 20, 5 << 20]
    try:
        for shift in (0, 1, 8, 15):
            srcs, dsts, texts, keep = [], [], [], []
            pos, dpos = 3, 256
            for i, n in enumerate(lens):
                if i % 3 == 2:
                    t = W.text_uniform(n, W.LOWER_ALPHABET, 500 + i)     # pageable: one copy each
                    keep.append(t)
                    srcs.append(t.ctypes.data if n else 0)
                    texts.append(t)
                    off = 0
                else:
                    srcs.append(big.data_ptr() + pos)                    # pinned: the copy kernel
                    texts.append(big[pos:pos + n].numpy())
                    off = pos & 15
                    pos += n + 7
                d = dpos + (off + shift) % 16
                dsts.append(arena.data_ptr() + d)
                dpos = (d + n + 255) // 256 * 256
            k = len(lens)
            which = [i % len(autos) for i in range(k)]
            hs = (ctypes.c_void_p * k)(*[autos[j].handle.value for j in which])
            src = (ctypes.c_void_p * k)(*srcs)
            dst = (ctypes.c_void_p * k)(*dsts)
            ln = (ctypes.c_uint64 * k)(*lens)
            out = torch.zeros(16 * 64, dtype=torch.uint8, device="cuda")
            arena.zero_()
            torch.cuda.synchronize()
            assert L.sfa_batch_update_host(plan, hs, src, dst, ln, k, stream.cuda_stream) == sfa.OK
            assert L.sfa_batch_launch(plan, out.data_ptr(), stream.cuda_stream) == sfa.OK
            stream.synchronize()
            host = arena.cpu().numpy()
            for i, n in enumerate(lens):
                o = dsts[i] - arena.data_ptr()
                assert np.array_equal(host[o:o + n], texts[i]), (shift, i, n)
            assert sfa.decode(out[:16 * k]) == [expect(autos_d[j], t) for j, t in zip(which, texts)], shift
    finally:
        L.sfa_batch_destroy(plan)


def test_server_slots_overlap_and_spans(sfa):
    """The server with device timing: every batch reports its span; batches
    of different slots are in flight at the same time (their spans, from
    CUDA events on the slots' streams, intersect); results equal the
    oracle's.  Requests all arrive at once, from one pinned buffer."""
    from paper_1405_0562_gb300 import serve
    autos_d = W.workload_serving_automata(8)
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    _, lens, which = W.workload_serving_requests(1500, rate_per_s=1.0, n_automata=len(autos))
    total = int(lens.sum())
    host = torch.from_numpy(W.text_uniform(total, W.LOWER_ALPHABET, 31)).pin_memory()
    offs = np.concatenate([[0], np.cumsum(lens)])
    reqs = [serve.Request(i, int(which[i]), host[offs[i]:offs[i + 1]], 0.0) for i in range(len(lens))]
    srv = serve.Server(autos, hbm_budget=1 << 30, max_batch=128, slots=3, timing=True)
    try:
        done = srv.run(reqs, realtime=False)
        spans = srv.spans()
        batches = srv.batches
    finally:
        srv.close()
    assert len(done) == len(reqs)
    assert len(spans) == batches and sum(s["requests"] for s in spans) == len(reqs)
    assert sum(s["bytes"] for s in spans) == total
    for s in spans:
        assert s["copy_start_ms"] <= s["copy_end_ms"] <= s["match_end_ms"]
    overlap = any(a["slot"] != b["slot"] and a["copy_start_ms"] < b["match_end_ms"] and
                  b["copy_start_ms"] < a["match_end_ms"] for a in spans for b in spans)
    assert overlap
    for r in done[::17]:
        assert r.result == expect(autos_d[r.automaton], r.text.numpy()), r.rid
