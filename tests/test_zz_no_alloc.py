"""sfa_match_noalloc: the entry point for callers that cannot allocate device
memory while matching (a host program that owns all device memory through
its own pool, or a loop that cannot pay for cudaMalloc/cudaFree).  Its
output must equal sfa_match's, exactly (integer results, tolerance 0), on
two calls in a row that reuse the one fixed scratch array.  Every call here
passes real device buffers with their true lengths; the refusals of texts
that do not fit are checked on the CPU (tests/test_host_compile.py), where no
device is touched.

This file is named so that pytest collects it last."""
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
    L = m.lib()
    L.sfa_match_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                    ctypes.c_void_p]
    L.sfa_match_noalloc.restype = ctypes.c_int
    torch.cuda.set_device(0)
    return m


def noalloc(sfa, a, text, out, stream):
    n = text.numel()
    return sfa.lib().sfa_match_noalloc(a.handle, text.data_ptr() if n else None, n, out.data_ptr(),
                                       stream.cuda_stream)


def test_noalloc_equals_match_twice(sfa):
    # 96 MiB: long enough for the two-level split of automatic chunks
    cases = [W.workload_large(48 << 20), W.workload_large(96 << 20), W.workload_single()]
    d3 = W.dfa_rn(4)
    t3 = np.frombuffer(b"01235678" * 100_000 + b"0", dtype=np.uint8).copy()
    t3[::9973] = ord("9")
    cases.append((d3, t3))
    stream = torch.cuda.Stream()
    for d, t in cases:
        a = sfa.Automaton.from_dfa(d)
        tt = torch.from_numpy(t).cuda()
        ref = a.match(tt, stream=stream)
        stream.synchronize()
        want = sfa.decode(ref)[0]
        f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
        assert want == (f, acc, 0, c)
        for _ in range(2):
            out = torch.full((16,), 0xAB, dtype=torch.uint8, device="cuda")
            assert noalloc(sfa, a, tt, out, stream) == sfa.OK
            stream.synchronize()
            assert sfa.decode(out)[0] == want
        # the same text from an address off a 16-byte boundary
        view = tt[5:]
        ref = a.match(view, stream=stream)
        out = torch.zeros(16, dtype=torch.uint8, device="cuda")
        assert noalloc(sfa, a, view, out, stream) == sfa.OK
        stream.synchronize()
        f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t[5:])
        assert sfa.decode(out)[0] == sfa.decode(ref)[0] == (f, acc, 0, c)
        # a shorter text right after a longer one: stale descriptors must not leak
        out = torch.zeros(16, dtype=torch.uint8, device="cuda")
        assert noalloc(sfa, a, tt[:1000], out, stream) == sfa.OK
        stream.synchronize()
        f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t[:1000])
        assert sfa.decode(out)[0] == (f, acc, 0, c)


def test_noalloc_allocates_nothing(sfa):
    """On a fresh handle (no sfa_match call has given it scratch of its own),
    once a first call has loaded the kernels, further calls leave the
    device's free memory and torch's pool exactly as they were: the scratch
    is the fixed array, nothing is allocated on the device."""
    d, t = W.workload_large(32 << 20)
    a = sfa.Automaton.from_dfa(d)
    stream = torch.cuda.Stream()
    tt = torch.from_numpy(t).cuda()
    outs = [torch.zeros(16, dtype=torch.uint8, device="cuda") for _ in range(3)]
    assert noalloc(sfa, a, tt, outs[0], stream) == sfa.OK
    stream.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for o in outs[1:]:
        assert noalloc(sfa, a, tt, o, stream) == sfa.OK
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
    for o in outs:
        assert sfa.decode(o)[0] == (f, acc, 0, c)
