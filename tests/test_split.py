"""One text split over several ranks (Lemma 1, Theorem 3): the exchange of
slice mappings (one all-gather), the entering state of every slice, the sum
of the counts.  The host logic runs here on the CPU with world sizes 2 and 3
on gloo, the slices' mappings and results coming from the oracle (Alg. 2 from
every state); the GPU test runs the same exchange with the library's
sfa_match_map and sfa_match_continue, two ranks on the one GPU (their kernels
never wait on one another: the exchange is on the host)."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _record(final, acc, count):
    rec = np.zeros(16, dtype=np.uint8)
    rec[:4] = np.frombuffer(np.uint32(final).tobytes(), np.uint8)
    rec[4] = acc
    rec[8:] = np.frombuffer(np.uint64(count).tobytes(), np.uint8)
    return torch.from_numpy(rec)


def _reachable(d):
    seen, todo = {d.q0}, [d.q0]
    while todo:
        q = todo.pop()
        for t in np.unique(d.delta[q]):
            if int(t) not in seen:
                seen.add(int(t))
                todo.append(int(t))
    return seen


class OracleSlices:
    """The two per-slice operations of the split, computed by the oracle."""

    def __init__(self, d):
        self.d = d
        self.kept = _reachable(d)

    def match_map(self, text, stream=None):
        t = text.numpy()
        m = np.full(self.d.nq, -1, dtype=np.int32)
        for q in self.kept:
            m[q] = oracle.dfa_run(self.d.delta, self.d.q0, self.d.accept, t, start=q)[0]
        return _record(*oracle.dfa_run(self.d.delta, self.d.q0, self.d.accept, t)), torch.from_numpy(m)

    def match_continue(self, text, rec, stream=None):
        import paper_1405_0562_gb300 as sfa
        s, _, _, c0 = sfa.decode(rec)[0]
        f, acc, c = oracle.dfa_run(self.d.delta, self.d.q0, self.d.accept, text.numpy(), start=s)
        return _record(f, acc, c0 + c)


CASES = {
    "ac": lambda: W.dfa_aho_corasick([b"he", b"she", b"his", b"hers"]),
    "r3": lambda: W.dfa_rn(3),
    "rand8": lambda: W.dfa_random(8, 4, seed=3),
}


def _text(name, d, n, seed):
    rng = np.random.default_rng(seed)
    if name == "r3":
        base = np.frombuffer((b"012567" * (n // 6 + 1))[:n], np.uint8).copy()
        base[rng.integers(0, n, max(1, n // 500))] = ord("9")
        return base
    alpha = np.frombuffer(d.alphabet, np.uint8)
    return alpha[rng.integers(0, alpha.size, n)]


def _worker(rank, world, port, q, on_gpu):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    from paper_1405_0562_gb300 import split
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        results = []
        for name, make in sorted(CASES.items()):
            d = make()
            n = 200_003 if on_gpu else 5_003
            text = _text(name, d, n, seed=world)
            # cuts at seeded positions, an empty slice among them
            rng = np.random.default_rng(7 + world)
            cuts = sorted(int(x) for x in rng.integers(0, n, world - 1))
            if world > 2:
                cuts[1] = cuts[0]
            bounds = [0] + cuts + [n]
            piece = text[bounds[rank]:bounds[rank + 1]]
            if on_gpu:
                import paper_1405_0562_gb300 as sfa
                torch.cuda.set_device(0)
                a = sfa.Automaton.from_dfa(d)
                got = split.match_split(a, torch.from_numpy(piece.copy()).cuda(), d.q0)
            else:
                got = split.match_split(OracleSlices(d), torch.from_numpy(piece.copy()), d.q0)
            f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, text)
            results.append((name, got, (f, acc, 0, c)))
        q.put((rank, results))
    finally:
        dist.destroy_process_group()


def _run(world, on_gpu):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, on_gpu)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for rank, results in got:
        for name, res, want in results:
            assert res == want, (rank, name, res, want)


def test_entering_states_compose_in_order():
    from paper_1405_0562_gb300 import split
    maps = [np.array([1, 2, 0, -1]), np.array([0, 0, 2, -1]), np.array([2, 1, 0, -1])]
    assert split.entering_states(maps, 0) == [0, 1, 0]
    assert split.entering_states(maps, 2) == [2, 0, 0]
    with pytest.raises(ValueError):
        split.entering_states([np.array([-1, 0]), np.array([0, 1])], 0)


@pytest.mark.parametrize("world", [2, 3])
def test_split_exchange_on_cpu(world):
    _run(world, on_gpu=False)


@pytest.mark.gpu
def test_split_on_gpu_two_ranks():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    _run(2, on_gpu=True)
