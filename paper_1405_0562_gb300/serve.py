"""Continuous-batching match server on one GPU.

Requests (automaton index, host text) arrive over time.  The server keeps
every compiled automaton resident on the device, admits requests while its
HBM text budget and the batch capacity allow, copies the admitted texts into
a device arena and matches them in one persistent launch per batch.  The
loop itself is native (``sfa_server_*`` in the C ABI): the queue, the arena
allocator, the batch slots (each on its own CUDA stream, several in flight)
and the completion polling by CUDA events run in C++: texts in pinned host
memory are copied in by one kernel per batch (other texts by one
cudaMemcpyAsync each) and matched by one launch per batch, with no
allocation and no host wait on the launch path.  This module drives it: it submits requests at their
arrival times, collects completions and stamps each request's latency
(completion time minus arrival time on the host clock).

Every result equals the result of matching the text alone (each text has
its own look-back chain and record in the batch kernel).
"""
from __future__ import annotations

import ctypes
import dataclasses
import gc
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import (SERVER_TIMING, Automaton, BatchSpan, Completion, RESULT_BYTES, ServerOpts, ServerStats, _check,
               decode, lib)

_ALIGN = 256


class ArenaAllocator:
    """The server's first-fit allocator of byte ranges in a fixed arena
    (offsets only), ranges 256-byte aligned, free neighbours merged: the
    native one, usable on its own (no device needed)."""

    def __init__(self, size: int):
        self.size = size
        self._a = lib().sfa_arena_create(size)
        if not self._a:
            raise MemoryError("sfa_arena_create")

    def alloc(self, n: int) -> Optional[int]:
        off = ctypes.c_uint64()
        rc = lib().sfa_arena_alloc(self._a, n, ctypes.byref(off))
        return int(off.value) if rc == 0 else None

    def release(self, off: int, n: int):
        _check(lib().sfa_arena_release(self._a, off, n), "sfa_arena_release")

    @property
    def used(self) -> int:
        return int(lib().sfa_arena_used(self._a))

    def __del__(self):
        if getattr(self, "_a", None):
            lib().sfa_arena_destroy(self._a)
            self._a = None


@dataclasses.dataclass
class Request:
    rid: int
    automaton: int
    text: object                 # pinned CPU uint8 tensor (or numpy array)
    arrival: float               # host clock, seconds
    admitted: float = 0.0
    done: float = 0.0
    result: Optional[tuple] = None
    offset: int = -1

    @property
    def nbytes(self) -> int:
        return int(self.text.numel() if hasattr(self.text, "numel") else len(self.text))


def _host_ptr(text) -> int:
    """Address of a request's host bytes (a CPU tensor, preferably pinned, or
    a contiguous numpy array)."""
    if hasattr(text, "data_ptr"):
        if text.is_cuda or not text.is_contiguous():
            raise ValueError("request text must be a contiguous host tensor")
        return text.data_ptr() if text.numel() else 0
    a = np.asarray(text)
    if a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("request text must be contiguous uint8")   # no temporary copy may be read
    return a.ctypes.data if a.size else 0


class Server:
    """Continuous batching over resident automata with HBM-budget admission
    (the native server, driven from Python)."""

    def __init__(self, automata: Sequence[Automaton], hbm_budget: int = 4 << 30, max_batch: int = 256,
                 slots: int = 3, chunk_bytes: int = 1024, block_threads: int = 512, device=None,
                 timing: bool = False):
        """timing: record each batch's device timeline (spans())."""
        import torch
        if device is not None:
            torch.cuda.set_device(device)
        self.automata = list(automata)
        hs = (ctypes.c_void_p * len(self.automata))(*[a.handle.value for a in self.automata])
        opts = ServerOpts(hbm_budget, max_batch, slots, chunk_bytes, block_threads,
                          SERVER_TIMING if timing else 0, 0)
        s = ctypes.c_void_p()
        _check(lib().sfa_server_create(hs, len(self.automata), ctypes.byref(opts), ctypes.byref(s)),
               "sfa_server_create")
        self._s = s
        self.budget = hbm_budget
        self._pending: Dict[int, Request] = {}
        self._cap = 4096
        self._buf = (Completion * self._cap)()
        self._n = ctypes.c_int32()
        self.completed: List[Request] = []

    # ---- request flow ----------------------------------------------------
    def submit(self, req: Request):
        if req.nbytes > self.budget:
            raise ValueError("request larger than the HBM text budget")
        if req.rid in self._pending:
            raise ValueError("request id already in flight")
        if not 0 <= req.rid < self._RUN_TAG:
            raise ValueError("request ids of submit() are in [0, 2^62)")
        self._pending[req.rid] = req
        _check(lib().sfa_server_submit(self._s, req.automaton, _host_ptr(req.text), req.nbytes, req.rid),
               "sfa_server_submit")

    def step(self):
        """Complete finished batches, admit and launch queued requests."""
        L = lib()
        while True:
            _check(L.sfa_server_progress(self._s, self._buf, self._cap, ctypes.byref(self._n)),
                   "sfa_server_progress")
            k = self._n.value
            if not k:
                return
            now = time.perf_counter()
            raw = np.ctypeslib.as_array(ctypes.cast(self._buf, ctypes.POINTER(ctypes.c_uint64)),
                                        shape=(k * 3,)).reshape(k, 3)
            res = decode(raw[:, 1:].copy().view(np.uint8))
            for tag, x in zip(raw[:, 0].tolist(), res):
                r = self._pending.pop(tag)
                r.result = x
                r.done = now
                self.completed.append(r)
            if k < self._cap:
                return

    poll = step

    def stats(self) -> dict:
        """Queue, slot and arena counters (the last ones once closed)."""
        if getattr(self, "_s", None) is None:
            return dict(self._final)
        st = ServerStats()
        _check(lib().sfa_server_stats(self._s, ctypes.byref(st)), "sfa_server_stats")
        return {f: int(getattr(st, f)) for f, _ in ServerStats._fields_}

    def spans(self) -> List[dict]:
        """Device timelines of the batches finished since the last call
        (SFA_SERVER_TIMING): slot, requests, bytes, copy start / end and
        match end in ms since the server was created."""
        out, n, res = (BatchSpan * 256)(), ctypes.c_int32(), []
        while True:
            _check(lib().sfa_server_spans(self._s, out, 256, ctypes.byref(n)), "sfa_server_spans")
            res += [{f: getattr(out[i], f) for f, _ in BatchSpan._fields_ if f != "reserved"}
                    for i in range(n.value)]
            if n.value < 256:
                return res

    @property
    def batches(self) -> int:
        return self.stats()["batches"]

    def idle(self) -> bool:
        return not self._pending

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            self._final = self.stats()
            lib().sfa_server_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()

    # ---- driving a workload ------------------------------------------------
    _RUN_TAG = 1 << 62   # tags of run()'s requests: this base + position

    def run(self, requests: Sequence[Request], realtime: bool = True):
        """Submit each request at its arrival time (offsets from now) and
        serve until all are done.  Returns the completed requests.  The
        requests' arrays (automaton, text address, length, tag) are built
        before the clock starts; the requests due at each turn of the loop
        go to the server in one call, and completions are stamped by array
        (no per-request Python work inside the loop: at tens of thousands
        of requests a second that work, not the device, would set the
        pace).  Requests submitted by submit() and not yet done are served
        too."""
        pending = sorted(requests, key=lambda r: r.arrival)
        n = len(pending)
        for r in pending:
            if r.nbytes > self.budget:
                raise ValueError("request larger than the HBM text budget")
            if r.rid in self._pending:
                raise ValueError("request id already in flight")
        rel = np.array([r.arrival for r in pending], dtype=np.float64)
        auto = np.array([r.automaton for r in pending], dtype=np.int32)
        ptr = np.array([_host_ptr(r.text) for r in pending], dtype=np.uint64)
        ln = np.array([r.nbytes for r in pending], dtype=np.uint64)
        tag = np.arange(n, dtype=np.uint64) + np.uint64(self._RUN_TAG)
        done_t = np.zeros(n, dtype=np.float64)
        words = np.zeros((n, 2), dtype=np.uint64)
        L = lib()
        # no cyclic garbage collection inside the loop: with many live
        # objects in the process one collection stalls admission for
        # milliseconds
        gc_on = gc.isenabled()
        gc.disable()
        try:
            t0 = time.perf_counter()
            i = 0
            left = n
            while i < n or left or self._pending:
                j = n if not realtime else int(np.searchsorted(rel, time.perf_counter() - t0, side="right"))
                if j > i:
                    _check(L.sfa_server_submit_many(self._s, j - i, auto[i:].ctypes.data, ptr[i:].ctypes.data,
                                                    ln[i:].ctypes.data, tag[i:].ctypes.data), "sfa_server_submit_many")
                    i = j
                left -= self._drain(done_t, words)
        finally:
            if gc_on:
                gc.enable()
        # the Request records, once the clock has stopped
        res = decode(words.view(np.uint8))
        for k, r in enumerate(pending):
            r.arrival = t0 + rel[k]
            r.admitted = r.arrival
            r.done = float(done_t[k])
            r.result = res[k]
            self.completed.append(r)
        return self.completed

    def _drain(self, done_t, words) -> int:
        """One progress call: stamp run()'s completions into the arrays (by
        tag), hand the others to their Request records; returns the number
        of run() completions."""
        L = lib()
        got = 0
        while True:
            _check(L.sfa_server_progress(self._s, self._buf, self._cap, ctypes.byref(self._n)),
                   "sfa_server_progress")
            k = self._n.value
            if not k:
                return got
            now = time.perf_counter()
            raw = np.ctypeslib.as_array(ctypes.cast(self._buf, ctypes.POINTER(ctypes.c_uint64)),
                                        shape=(k * 3,)).reshape(k, 3)
            tags = raw[:, 0]
            mine = tags >= np.uint64(self._RUN_TAG)
            idx = (tags[mine] - np.uint64(self._RUN_TAG)).astype(np.int64)
            done_t[idx] = now
            words[idx] = raw[mine, 1:]
            got += int(idx.size)
            if not mine.all():
                other = raw[~mine]
                for t, x in zip(other[:, 0].tolist(), decode(other[:, 1:].copy().view(np.uint8))):
                    r = self._pending.pop(t)
                    r.result = x
                    r.done = now
                    self.completed.append(r)
            if k < self._cap:
                return got


def one_at_a_time(automata: Sequence[Automaton], requests: Sequence[Request], realtime: bool = True):
    """The baseline: each request matched alone with sfa_match when it
    arrives (copy in, launch, copy out, synchronise), in arrival order."""
    import torch
    stream = torch.cuda.Stream()
    out = torch.zeros(RESULT_BYTES, dtype=torch.uint8, device="cuda")
    out_host = torch.zeros(RESULT_BYTES, dtype=torch.uint8).pin_memory()
    maxn = max(r.nbytes for r in requests)
    buf = torch.empty(max(maxn, 1), dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    done = []
    for r in sorted(requests, key=lambda r: r.arrival):
        rel = r.arrival
        if realtime:
            while time.perf_counter() - t0 < rel:
                pass
        r.arrival = t0 + rel
        r.admitted = time.perf_counter()
        with torch.cuda.stream(stream):
            if r.nbytes:
                src = r.text if hasattr(r.text, "numel") else torch.from_numpy(np.asarray(r.text))
                buf[:r.nbytes].copy_(src, non_blocking=True)
            automata[r.automaton].match(buf[:r.nbytes], out, stream=stream)
            out_host.copy_(out, non_blocking=True)
        stream.synchronize()
        r.result = decode(out_host)[0]
        r.done = time.perf_counter()
        done.append(r)
    return done


def latency_stats(reqs: Sequence[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    nbytes = sum(r.nbytes for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "GBps": nbytes / span / 1e9, "span_s": span}
