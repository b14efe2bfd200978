"""Continuous-batching match server on one GPU.

Requests (automaton index, host text) arrive over time.  The server keeps
every compiled automaton resident on the device, admits requests while its
HBM text budget and the batch capacity allow, copies the admitted texts into
a device arena and matches them in one persistent launch per batch
(``sfa_batch_update`` + ``sfa_batch_launch``: no allocation, no host
synchronisation on the launch path).  Several batch slots, each on its own
CUDA stream, are in flight at once: requests that arrive while a batch runs
are admitted into the next free slot as soon as memory frees up, so their
copies and kernels overlap the running batch.  Completion is detected by
polling CUDA events; each request's latency is completion time minus arrival
time on the host clock.

Every result equals the result of matching the text alone (each text has
its own look-back chain and record in the batch kernel).
"""
from __future__ import annotations

import bisect
import ctypes
import dataclasses
import time
from collections import deque
from typing import List, Optional, Sequence

import numpy as np

from . import (Automaton, LaunchOpts, RESULT_BYTES, _check, _stream_ptr, decode, lib)

_ALIGN = 256


class ArenaAllocator:
    """First-fit allocator of byte ranges in a fixed device arena (offsets
    only; the memory is one tensor).  Ranges are 256-byte aligned."""

    def __init__(self, size: int):
        self.size = size
        self.free: List[List[int]] = [[0, size]]   # sorted [start, end)
        self.used = 0

    def alloc(self, n: int) -> Optional[int]:
        n = max(_ALIGN, (n + _ALIGN - 1) // _ALIGN * _ALIGN)
        for i, (s, e) in enumerate(self.free):
            if e - s >= n:
                if e - s == n:
                    self.free.pop(i)
                else:
                    self.free[i][0] = s + n
                self.used += n
                return s
        return None

    def release(self, off: int, n: int):
        n = max(_ALIGN, (n + _ALIGN - 1) // _ALIGN * _ALIGN)
        self.used -= n
        i = bisect.bisect_left(self.free, [off, off + n])
        self.free.insert(i, [off, off + n])
        # merge with neighbours
        if i + 1 < len(self.free) and self.free[i][1] == self.free[i + 1][0]:
            self.free[i][1] = self.free[i + 1][1]
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1][1] = self.free[i][1]
            self.free.pop(i)


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


class _Slot:
    def __init__(self, torch, max_texts, max_tiles, nr_max, opts, device):
        self.stream = torch.cuda.Stream(device=device)
        self.out = torch.zeros(max_texts * RESULT_BYTES, dtype=torch.uint8, device=device)
        self.out_host = torch.zeros(max_texts * RESULT_BYTES, dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()
        self.reqs: List[Request] = []
        b = ctypes.c_void_p()
        _check(lib().sfa_batch_reserve(max_texts, max_tiles, nr_max, ctypes.byref(opts), ctypes.byref(b)),
               "sfa_batch_reserve")
        self.plan = b

    def close(self):
        if self.plan is not None and self.plan.value:
            lib().sfa_batch_destroy(self.plan)
            self.plan = None


class Server:
    """Continuous batching over resident automata with HBM-budget admission."""

    def __init__(self, automata: Sequence[Automaton], hbm_budget: int = 4 << 30, max_batch: int = 512,
                 slots: int = 3, chunk_bytes: int = 1024, block_threads: int = 512, device=None):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.automata = list(automata)
        nr_max = max(a.info()["n_reachable"] for a in self.automata)
        self.arena = torch.empty(hbm_budget, dtype=torch.uint8, device=self.device)
        self.alloc = ArenaAllocator(hbm_budget)
        self.max_batch = max_batch
        self.opts = LaunchOpts(chunk_bytes, block_threads, 1, 0, 0, 0, 0, 0)
        cpt = block_threads
        max_tiles = max_batch + hbm_budget // (cpt * chunk_bytes) + 1
        self.slots = [_Slot(torch, max_batch, max_tiles, nr_max, self.opts, self.device) for _ in range(slots)]
        self.free_slots = deque(self.slots)
        self.busy: List[_Slot] = []
        self.queue: deque = deque()
        self.completed: List[Request] = []
        self.batches = 0
        self.batched_requests = 0

    # ---- request flow ----------------------------------------------------
    def submit(self, req: Request):
        if req.nbytes > self.alloc.size:
            raise ValueError("request larger than the HBM text budget")
        self.queue.append(req)

    def poll(self):
        """Complete every slot whose batch has finished."""
        still = []
        for s in self.busy:
            if s.event.query():
                now = time.perf_counter()
                res = decode(s.out_host[:len(s.reqs) * RESULT_BYTES])
                for r, x in zip(s.reqs, res):
                    r.result = x
                    r.done = now
                    self.alloc.release(r.offset, r.nbytes)
                    self.completed.append(r)
                s.reqs = []
                self.free_slots.append(s)
            else:
                still.append(s)
        self.busy = still

    def admit_and_launch(self):
        """Fill free slots from the queue (FIFO, while memory allows) and
        launch them."""
        torch = self.torch
        while self.free_slots and self.queue:
            slot = self.free_slots[0]
            take: List[Request] = []
            while self.queue and len(take) < self.max_batch:
                r = self.queue[0]
                off = self.alloc.alloc(r.nbytes)
                if off is None:
                    break
                r.offset = off
                take.append(self.queue.popleft())
            if not take:
                return
            self.free_slots.popleft()
            now = time.perf_counter()
            k = len(take)
            hs = (ctypes.c_void_p * k)(*[self.automata[r.automaton].handle.value for r in take])
            base = self.arena.data_ptr()
            ptrs = (ctypes.c_void_p * k)(*[base + r.offset for r in take])
            lens = (ctypes.c_uint64 * k)(*[r.nbytes for r in take])
            srcs = (ctypes.c_void_p * k)(*[_host_ptr(r.text) for r in take])
            for r in take:
                r.admitted = now
            with torch.cuda.stream(slot.stream):
                sp = _stream_ptr(slot.stream)
                # copies of the texts into the arena and the new work list,
                # enqueued natively on the slot's stream
                _check(lib().sfa_batch_update_host(slot.plan, hs, srcs, ptrs, lens, k, sp), "sfa_batch_update_host")
                _check(lib().sfa_batch_launch(slot.plan, slot.out.data_ptr(), sp), "sfa_batch_launch")
                slot.out_host[:k * RESULT_BYTES].copy_(slot.out[:k * RESULT_BYTES], non_blocking=True)
                slot.event.record(slot.stream)
            slot.reqs = take
            self.busy.append(slot)
            self.batches += 1
            self.batched_requests += k

    def step(self):
        self.poll()
        self.admit_and_launch()

    def idle(self) -> bool:
        return not self.queue and not self.busy

    def close(self):
        for s in self.slots:
            s.close()

    # ---- driving a workload ------------------------------------------------
    def run(self, requests: Sequence[Request], realtime: bool = True):
        """Submit each request at its arrival time (offsets from now) and
        serve until all are done.  Returns the completed requests."""
        t0 = time.perf_counter()
        pending = sorted(requests, key=lambda r: r.arrival)
        rel = [r.arrival for r in pending]
        i = 0
        while i < len(pending) or not self.idle():
            now = time.perf_counter() - t0
            while i < len(pending) and (not realtime or rel[i] <= now):
                r = pending[i]
                r.arrival = t0 + rel[i]
                self.submit(r)
                i += 1
            self.step()
        return self.completed


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
