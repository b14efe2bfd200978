"""GB300 (sm_103a) matcher for simultaneous finite automata.

Thin ctypes binding of the C ABI in ``include/sfa.h``; every step of the
matching path runs in the CUDA kernels of ``libsfa.so``.  PyTorch supplies
device memory and streams only.  There is no CPU fallback: when the library
is missing, or no GPU is present, calls that need the device raise.

    import paper_1405_0562_gb300 as sfa
    a = sfa.Automaton(delta, q0, accept)          # Alg. 4 on the host + upload
    out = a.match(text_cuda_u8)                   # Alg. 5 on the GPU
    final, accept_final, status, count = sfa.decode(out)[0]
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsfa.so")

# sfa.h constants
OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NO_DEVICE, ERR_HOST_ONLY = 0, -1, -2, -3, -4, -5, -6, -7
ERR_SCRATCH_LIMIT = -8
NOALLOC_SCRATCH_BYTES = 4 << 20
MODE_AUTO, MODE_SFA, MODE_SIM = 0, 1, 2
COMPILE_HOST_ONLY, COMPILE_NO_BANK_TUNE = 1, 2
STATUS_OK, STATUS_TIMEOUT = 0, 1
DEBUG_SKIP_PUBLISH = 1
TABLE_CLASS, TABLE_DFA, TABLE_NC, TABLE_MAPS, TABLE_ORIG, TABLE_CDFA16, TABLE_MAPS16, TABLE_SETS = 0, 1, 2, 3, 4, 5, 6, 7
PLACE_SMEM_DFA, PLACE_SMEM_DFA_CLASSES, PLACE_GLOBAL_NC, PLACE_SMEM_VECTORS = 1, 2, 4, 8
TILING_AUTO, TILING_CTA, TILING_WARP = 0, 1, 2
SERVER_TIMING = 1
REGEX_SEARCH, REGEX_DOTALL, REGEX_NO_MINIMIZE = 1, 2, 4
RESULT_BYTES = 16

# every symbol include/sfa.h declares
EXPORTED = (
    "sfa_compile", "sfa_compile_sample", "sfa_destroy", "sfa_info", "sfa_export", "sfa_strerror",
    "sfa_match", "sfa_match_ex", "sfa_match_continue", "sfa_match_host", "sfa_match_map",
    "sfa_batch_create", "sfa_batch_launch", "sfa_batch_graph_launch", "sfa_batch_destroy",
    "sfa_match_batch", "sfa_kernel_launch_count", "sfa_match_noalloc",
    "sfa_batch_reserve", "sfa_batch_update", "sfa_batch_update_host",
    "sfa_server_create", "sfa_server_submit", "sfa_server_submit_many", "sfa_server_progress", "sfa_server_stats",
    "sfa_server_spans", "sfa_server_destroy",
    "sfa_arena_create", "sfa_arena_alloc", "sfa_arena_release", "sfa_arena_used", "sfa_arena_destroy",
    "sfa_regex_dfa", "sfa_regex_compile", "sfa_regex_nsfa_states",
)


class SfaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class CompileOpts(ctypes.Structure):
    _fields_ = [("cap_states", ctypes.c_uint32), ("force_mode", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("nq", ctypes.c_uint32), ("n_reachable", ctypes.c_uint32),
                ("n_accepting", ctypes.c_uint32), ("ncls", ctypes.c_uint32), ("on_device", ctypes.c_uint32),
                ("n_sfa_states", ctypes.c_uint64), ("n_nonconst", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64), ("compile_seconds", ctypes.c_double),
                ("n_stored", ctypes.c_uint64), ("id_bits", ctypes.c_uint32), ("placement", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LaunchOpts(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("chains", ctypes.c_uint32), ("max_ctas", ctypes.c_uint32),
                ("forced_chunks", ctypes.c_uint32), ("timeout_us", ctypes.c_uint32),
                ("debug_flags", ctypes.c_uint32), ("tiling", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("final_state", ctypes.c_uint32), ("accept_final", ctypes.c_uint8),
                ("status", ctypes.c_uint8), ("reserved", ctypes.c_uint16), ("count", ctypes.c_uint64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("chunk_bytes", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class BatchSpan(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int32), ("requests", ctypes.c_int32), ("bytes", ctypes.c_uint64),
                ("copy_start_ms", ctypes.c_float), ("copy_end_ms", ctypes.c_float),
                ("match_end_ms", ctypes.c_float), ("reserved", ctypes.c_float)]


class RegexInfo(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32), ("q0", ctypes.c_int32), ("positions", ctypes.c_int32),
                ("subset_states", ctypes.c_int32), ("ncls", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("result", Result)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_uint64), ("in_flight", ctypes.c_uint64),
                ("completed_waiting", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("requests", ctypes.c_uint64), ("arena_used", ctypes.c_uint64)]


_lib_handle = None


def lib():
    """The loaded libsfa.so.  Raises if it has not been built."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (the CUDA library is required)")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    L.sfa_compile.argtypes = [P, i32, i32, P, P, ctypes.POINTER(P)]
    L.sfa_compile_sample.argtypes = [P, i32, i32, P, P, P, u64, ctypes.POINTER(P)]
    L.sfa_destroy.argtypes = [P]
    L.sfa_destroy.restype = None
    L.sfa_info.argtypes = [P, ctypes.POINTER(Info)]
    L.sfa_export.argtypes = [P, i32, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.sfa_strerror.argtypes = [ctypes.c_int]
    L.sfa_strerror.restype = ctypes.c_char_p
    L.sfa_match.argtypes = [P, P, u64, P, P]
    L.sfa_match_ex.argtypes = [P, P, u64, P, P, ctypes.POINTER(LaunchOpts)]
    L.sfa_match_continue.argtypes = [P, P, u64, P, P, ctypes.POINTER(LaunchOpts)]
    L.sfa_match_host.argtypes = [P, P, u64, ctypes.POINTER(Result), P, ctypes.POINTER(LaunchOpts)]
    L.sfa_match_map.argtypes = [P, P, u64, P, P, P, ctypes.POINTER(LaunchOpts)]
    L.sfa_batch_create.argtypes = [P, P, P, i32, ctypes.POINTER(LaunchOpts), ctypes.POINTER(P)]
    L.sfa_batch_launch.argtypes = [P, P, P]
    L.sfa_batch_graph_launch.argtypes = [P, P, P]
    L.sfa_batch_destroy.argtypes = [P]
    L.sfa_batch_destroy.restype = None
    L.sfa_match_batch.argtypes = [P, P, P, i32, P, P]
    L.sfa_kernel_launch_count.argtypes = []
    L.sfa_kernel_launch_count.restype = u64
    L.sfa_match_noalloc.argtypes = [P, P, u64, P, P]
    L.sfa_batch_reserve.argtypes = [i32, u64, u32, ctypes.POINTER(LaunchOpts), ctypes.POINTER(P)]
    L.sfa_batch_update.argtypes = [P, P, P, P, i32, P]
    L.sfa_batch_update_host.argtypes = [P, P, P, P, P, i32, P]
    L.sfa_server_create.argtypes = [P, i32, ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
    L.sfa_server_submit.argtypes = [P, i32, P, u64, u64]
    L.sfa_server_submit_many.argtypes = [P, i32, P, P, P, P]
    L.sfa_server_progress.argtypes = [P, ctypes.POINTER(Completion), i32, ctypes.POINTER(i32)]
    L.sfa_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    L.sfa_server_spans.argtypes = [P, ctypes.POINTER(BatchSpan), i32, ctypes.POINTER(i32)]
    L.sfa_server_destroy.argtypes = [P]
    L.sfa_server_destroy.restype = None
    L.sfa_arena_create.argtypes = [u64]
    L.sfa_arena_create.restype = P
    L.sfa_arena_alloc.argtypes = [P, u64, ctypes.POINTER(u64)]
    L.sfa_arena_release.argtypes = [P, u64, u64]
    L.sfa_arena_used.argtypes = [P]
    L.sfa_arena_used.restype = u64
    L.sfa_arena_destroy.argtypes = [P]
    L.sfa_regex_dfa.argtypes = [ctypes.c_char_p, ctypes.c_size_t, u32, i32, P, P, ctypes.POINTER(RegexInfo),
                                ctypes.POINTER(ctypes.c_size_t)]
    L.sfa_regex_compile.argtypes = [ctypes.c_char_p, ctypes.c_size_t, u32, P, ctypes.POINTER(P)]
    L.sfa_regex_nsfa_states.argtypes = [ctypes.c_char_p, ctypes.c_size_t, u32, u64, ctypes.POINTER(u64)]
    L.sfa_arena_destroy.restype = None
    for name in EXPORTED:
        if name not in ("sfa_destroy", "sfa_batch_destroy", "sfa_strerror", "sfa_kernel_launch_count",
                        "sfa_server_destroy", "sfa_arena_create", "sfa_arena_used", "sfa_arena_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib_handle = L
    return L


def strerror(code: int) -> str:
    return lib().sfa_strerror(code).decode()


def _check(code: int, what: str):
    if code != OK:
        raise SfaError(code, what)


_NO_OPTS = None


def _launch_opts(chunk_bytes=0, block_threads=0, chains=0, max_ctas=0, forced_chunks=0, timeout_us=0,
                 debug_flags=0, tiling=0) -> Optional[LaunchOpts]:
    global _NO_OPTS
    if not (chunk_bytes or block_threads or chains or max_ctas or forced_chunks or timeout_us or debug_flags
            or tiling):
        # the automatic shape: one shared all-zero record (the library only reads it)
        if _NO_OPTS is None:
            _NO_OPTS = LaunchOpts(0, 0, 0, 0, 0, 0, 0, 0)
        return _NO_OPTS
    return LaunchOpts(chunk_bytes, block_threads, chains, max_ctas, forced_chunks, timeout_us, debug_flags, tiling)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dev_ptr(t, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def empty_results(k: int = 1, device=None):
    """Device buffer for k sfa_result records (16 bytes each)."""
    import torch
    return torch.empty(k * RESULT_BYTES, dtype=torch.uint8, device=device or "cuda")


def decode(out) -> list:
    """(final_state, accept_final, status, count) of each 16-byte record."""
    if hasattr(out, "detach"):
        out = out.detach().cpu().numpy()
    raw = np.ascontiguousarray(out, dtype=np.uint8).view(np.uint64).reshape(-1, 2)
    return [(int(w0 & 0xFFFFFFFF), int((w0 >> 32) & 0xFF), int((w0 >> 40) & 0xFF), int(c)) for w0, c in raw]


class Automaton:
    """A DFA compiled into a device-resident D-SFA (or simulation) handle."""

    def __init__(self, delta, q0: int, accept, cap_states: int = 0, mode: int = MODE_AUTO,
                 host_only: bool = False, bank_tune: bool = True, sample=None):
        """sample: host bytes (numpy uint8) like the texts to come, for the
        bank-conflict model of the state numbering (sfa_compile_sample)."""
        d = np.ascontiguousarray(delta, dtype=np.int32)
        a = np.ascontiguousarray(accept, dtype=np.uint8)
        if d.ndim != 2 or d.shape[1] != 256 or a.shape != (d.shape[0],):
            raise ValueError("delta must be int32 [nq, 256] and accept uint8 [nq]")
        flags = (COMPILE_HOST_ONLY if host_only else 0) | (0 if bank_tune else COMPILE_NO_BANK_TUNE)
        opts = CompileOpts(cap_states, mode, flags, 0)
        h = ctypes.c_void_p()
        if sample is None:
            _check(lib().sfa_compile(d.ctypes.data, d.shape[0], int(q0), a.ctypes.data, ctypes.byref(opts),
                                     ctypes.byref(h)), "sfa_compile")
        else:
            smp = np.ascontiguousarray(sample, dtype=np.uint8)
            _check(lib().sfa_compile_sample(d.ctypes.data, d.shape[0], int(q0), a.ctypes.data, ctypes.byref(opts),
                                            smp.ctypes.data if smp.size else None, smp.size, ctypes.byref(h)),
                   "sfa_compile_sample")
        self._h = h
        self.nq = d.shape[0]

    @classmethod
    def from_dfa(cls, dfa, **kw):
        return cls(dfa.delta, dfa.q0, dfa.accept, **kw)

    @classmethod
    def from_regex(cls, pattern: bytes, search: bool = False, dotall: bool = False, **kw):
        """The D-SFA of a regular expression's minimal DFA (sfa_regex_dfa)."""
        delta, q0, acc, _ = regex_dfa(pattern, search=search, dotall=dotall)
        return cls(delta, q0, acc, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sfa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = Info()
        _check(lib().sfa_info(self._h, ctypes.byref(i)), "sfa_info")
        return i.as_dict()

    def export(self, which: int) -> np.ndarray:
        size = ctypes.c_size_t()
        _check(lib().sfa_export(self._h, which, None, 0, ctypes.byref(size)), "sfa_export")
        dtype = {TABLE_CLASS: np.uint8, TABLE_DFA: np.uint8, TABLE_NC: np.uint32, TABLE_MAPS: np.uint8,
                 TABLE_ORIG: np.int32, TABLE_CDFA16: np.uint16, TABLE_MAPS16: np.uint16,
                 TABLE_SETS: np.uint32}[which]
        buf = np.zeros(size.value // np.dtype(dtype).itemsize, dtype=dtype)
        _check(lib().sfa_export(self._h, which, buf.ctypes.data, buf.nbytes, ctypes.byref(size)), "sfa_export")
        return buf

    def match(self, text, out=None, stream=None, **launch):
        """Enqueue sfa_match_ex on `stream` (default: torch's current stream).
        text: contiguous CUDA uint8 tensor.  Returns the 16-byte result tensor."""
        if out is None:
            out = empty_results(1, text.device)
        o = _launch_opts(**launch)
        n = text.numel()
        ptr = _dev_ptr(text, "text") if n else 0
        _check(lib().sfa_match_ex(self._h, ptr, n, _dev_ptr(out, "out"), _stream_ptr(stream), ctypes.byref(o)),
               "sfa_match_ex")
        return out

    def match_noalloc(self, text, out, stream=None):
        """sfa_match_noalloc: for callers that must not allocate device memory
        while matching; `out` must be a caller-owned 16-byte CUDA buffer.  Its
        scratch is the library's one fixed array: do not overlap calls."""
        n = text.numel()
        ptr = _dev_ptr(text, "text") if n else 0
        _check(lib().sfa_match_noalloc(self._h, ptr, n, _dev_ptr(out, "out"), _stream_ptr(stream)),
               "sfa_match_noalloc")
        return out

    def match_continue(self, text, inout, stream=None, **launch):
        """Lemma 1 streaming: `inout` holds the result of the text so far."""
        o = _launch_opts(**launch)
        n = text.numel()
        ptr = _dev_ptr(text, "text") if n else 0
        _check(lib().sfa_match_continue(self._h, ptr, n, _dev_ptr(inout, "inout"), _stream_ptr(stream),
                                        ctypes.byref(o)), "sfa_match_continue")
        return inout

    def match_map(self, text, out=None, map_out=None, stream=None, **launch):
        """sfa_match_map: the slice's mapping (int32 CUDA tensor of nq entries,
        caller ids, -1 for states not reachable from q0) and its result from
        q0.  Returns (out, map_out)."""
        if out is None:
            out = empty_results(1, text.device)
        if map_out is None:
            import torch
            map_out = torch.empty(self.nq, dtype=torch.int32, device=text.device)
        if map_out.numel() < self.nq:
            raise ValueError("map_out needs nq entries")
        o = _launch_opts(**launch)
        n = text.numel()
        ptr = _dev_ptr(text, "text") if n else 0
        _check(lib().sfa_match_map(self._h, ptr, n, _dev_ptr(out, "out"), _dev_ptr(map_out, "map_out"),
                                   _stream_ptr(stream), ctypes.byref(o)), "sfa_match_map")
        return out, map_out

    def match_host(self, text, stream=None, **launch):
        """End to end: host text (numpy uint8, or a pinned CPU tensor) in,
        (final_state, accept_final, status, count) out; synchronises."""
        if hasattr(text, "data_ptr"):
            ptr, n = text.data_ptr(), text.numel()
        else:
            arr = np.ascontiguousarray(text, dtype=np.uint8)
            ptr, n = arr.ctypes.data, arr.size
        r = Result()
        o = _launch_opts(**launch)
        _check(lib().sfa_match_host(self._h, ptr, n, ctypes.byref(r), _stream_ptr(stream), ctypes.byref(o)),
               "sfa_match_host")
        return (r.final_state, r.accept_final, r.status, r.count)


class Batch:
    """A planned persistent launch over many (automaton, text) pairs."""

    def __init__(self, automata: Sequence[Automaton], texts: Sequence, **launch):
        if len(automata) != len(texts):
            raise ValueError("one automaton per text")
        k = len(texts)
        self.k = k
        self._keep = list(texts)
        hs = (ctypes.c_void_p * max(k, 1))(*[a.handle.value for a in automata])
        ptrs = (ctypes.c_void_p * max(k, 1))(*[(_dev_ptr(t, "text") if t.numel() else 0) for t in texts])
        lens = (ctypes.c_uint64 * max(k, 1))(*[t.numel() for t in texts])
        self._automata = list(automata)
        o = _launch_opts(**launch)
        b = ctypes.c_void_p()
        _check(lib().sfa_batch_create(hs, ptrs, lens, k, ctypes.byref(o), ctypes.byref(b)), "sfa_batch_create")
        self._b = b

    def launch(self, out=None, stream=None, graph: bool = False):
        if out is None:
            out = empty_results(max(self.k, 1))
        fn = lib().sfa_batch_graph_launch if graph else lib().sfa_batch_launch
        _check(fn(self._b, _dev_ptr(out, "out"), _stream_ptr(stream)), "sfa_batch_launch")
        return out

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            lib().sfa_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match_batch(automata: Sequence[Automaton], texts: Sequence, out=None, stream=None):
    """sfa_match_batch: plan, launch, synchronise, free."""
    k = len(texts)
    if out is None:
        out = empty_results(max(k, 1))
    hs = (ctypes.c_void_p * max(k, 1))(*[a.handle.value for a in automata])
    ptrs = (ctypes.c_void_p * max(k, 1))(*[(_dev_ptr(t, "text") if t.numel() else 0) for t in texts])
    lens = (ctypes.c_uint64 * max(k, 1))(*[t.numel() for t in texts])
    _check(lib().sfa_match_batch(hs, ptrs, lens, k, _dev_ptr(out, "out"), _stream_ptr(stream)), "sfa_match_batch")
    return out


def regex_dfa(pattern: bytes, search: bool = False, dotall: bool = False, minimize: bool = True):
    """The DFA of a regular expression (sfa_regex_dfa): (delta int32 [nq, 256],
    q0, accept uint8 [nq], info dict)."""
    flags = (REGEX_SEARCH if search else 0) | (REGEX_DOTALL if dotall else 0) | (0 if minimize else REGEX_NO_MINIMIZE)
    pat = bytes(pattern)
    info, err = RegexInfo(), ctypes.c_size_t()
    rc = lib().sfa_regex_dfa(pat, len(pat), flags, 1, None, None, ctypes.byref(info), ctypes.byref(err))
    if rc == ERR_INVALID:
        raise SfaError(rc, f"sfa_regex_dfa: syntax error at byte {err.value} of {pat!r}")
    _check(rc, "sfa_regex_dfa")
    nq = info.nq
    delta = np.zeros((nq, 256), dtype=np.int32)
    acc = np.zeros(nq, dtype=np.uint8)
    _check(lib().sfa_regex_dfa(pat, len(pat), flags, nq, delta.ctypes.data, acc.ctypes.data, ctypes.byref(info),
                               ctypes.byref(err)), "sfa_regex_dfa")
    return delta, int(info.q0), acc, {f: getattr(info, f) for f, _ in RegexInfo._fields_ if f != "reserved"}


def regex_nsfa_states(pattern: bytes, search: bool = False, dotall: bool = False, cap: int = 1 << 20):
    """States of the N-SFA of the expression's position NFA, or None past cap."""
    flags = (REGEX_SEARCH if search else 0) | (REGEX_DOTALL if dotall else 0)
    pat = bytes(pattern)
    n = ctypes.c_uint64()
    rc = lib().sfa_regex_nsfa_states(pat, len(pat), flags, cap, ctypes.byref(n))
    if rc == ERR_UNSUPPORTED:
        return None
    _check(rc, "sfa_regex_nsfa_states")
    return int(n.value)


def kernel_launch_count() -> int:
    return int(lib().sfa_kernel_launch_count())
