"""Autotuner for the launch shape of a match and of a batch plan: block
size, chunks per thread and chunk length, timed with CUDA events on the
device, cached in a JSON file keyed by (device, automaton shape, text-size
bucket) for single texts and by (device, automaton mix, length histogram)
for batches.

    from paper_1405_0562_gb300 import autotune
    shape = autotune.tune(automaton, text_cuda_u8)       # dict of launch options
    out = automaton.match(text_cuda_u8, **shape)
    bshape = autotune.tune_batch(automata, texts)        # options of sfa_batch_create
    out = Batch(automata, texts, **bshape).launch(graph=True)

The cache file is ``$SFA_TUNE_CACHE`` or ``~/.cache/sfa_gb300_tune.json``.
Results never depend on the shape (Theorem 3: any division of the text gives
the same result); only the time does.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, List, Optional

from . import MODE_SIM, TILING_WARP, Batch, SfaError, empty_results

_LOCK = threading.Lock()

SFA_SHAPES = [(512, 1), (1024, 1), (256, 1), (512, 2), (256, 2), (128, 4)]
SIM_SHAPES = [(128, 1), (256, 1), (128, 2)]
SFA_CHUNKS = [512, 1024, 2048, 3072, 4096]
SIM_CHUNKS = [4096, 8192, 16384, 32768, 65536]


def cache_path() -> str:
    return os.environ.get("SFA_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sfa_gb300_tune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(cache: dict):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass   # a read-only home: tune again next time


def bucket(n: int) -> int:
    """Text-size bucket: the power of two at or above n (at least 1 MiB)."""
    return 1 << max(20, math.ceil(math.log2(max(n, 1))))


def key_for(info: dict, n: int, device_name: str) -> str:
    return (f"{device_name}|mode{info['mode']}|nr{info['n_reachable']}|cls{info['ncls']}|"
            f"nc{min(info['n_nonconst'], 1 << 20)}|n{bucket(n)}")


def candidates(info: dict, n: int) -> List[Dict[str, int]]:
    """The automatic shape first (one tile per resident CTA, two levels on
    long texts), then each CTA shape with the automatic chunk length and with
    fixed ones, then warp tiles."""
    sim = info["mode"] == MODE_SIM
    shapes = SIM_SHAPES if sim else SFA_SHAPES
    chunks = SIM_CHUNKS if sim else SFA_CHUNKS
    out = [{}]
    for th, ch in shapes:
        # the automatic chunk length (two levels on long texts) with this shape
        if (th, ch) != shapes[0] or sim:
            out.append({"block_threads": th, "chains": ch})
        for c in chunks:
            if c * th * ch > max(n, 1) * 2 and c > chunks[0]:
                continue   # a single tile would hold the text many times over
            out.append({"block_threads": th, "chains": ch, "chunk_bytes": c})
    for th in ((128, 256) if sim else (256, 512, 1024)):
        out.append({"block_threads": th, "chains": 1, "tiling": TILING_WARP})
    return out


def _time(torch, automaton, text, out, shape: dict, reps: int) -> float:
    for _ in range(2):
        automaton.match(text, out, **shape)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        automaton.match(text, out, **shape)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(automaton, text, reps: int = 5, force: bool = False, verbose: bool = False) -> Dict[str, int]:
    """Best launch options for this automaton on texts of this size bucket.
    `text` must be a CUDA uint8 tensor (its contents are used as a sample)."""
    import torch
    info = automaton.info()
    n = text.numel()
    dev = torch.cuda.get_device_name(text.device)
    key = key_for(info, n, dev)
    with _LOCK:
        cache = _load()
        if not force and key in cache:
            return dict(cache[key]["shape"])
    out = empty_results(1, text.device)
    best, best_ms, table = None, float("inf"), []
    ref = None
    for shape in candidates(info, n):
        try:
            ms = _time(torch, automaton, text, out, shape, reps)
        except SfaError:
            continue   # shape outside this automaton's shared-memory budget
        res = bytes(out.cpu().numpy())
        if ref is None:
            ref = res
        elif res != ref:
            raise RuntimeError(f"launch shape {shape} changed the result")
        table.append((ms, shape))
        if verbose:
            print(f"  {shape} {n / ms / 1e6:.1f} GB/s", flush=True)
        if ms < best_ms:
            best, best_ms = shape, ms
    if best is None:
        return {}
    with _LOCK:
        cache = _load()
        cache[key] = {"shape": best, "ms": best_ms, "GBps": n / best_ms / 1e6}
        _store(cache)
    return dict(best)


def cached(automaton, n: int, device_name: Optional[str] = None) -> Optional[Dict[str, int]]:
    """The cached shape for this automaton and text size, if any."""
    import torch
    dev = device_name or torch.cuda.get_device_name()
    ent = _load().get(key_for(automaton.info(), n, dev))
    return dict(ent["shape"]) if ent else None


# ---------------------------------------------------------------------------
# batch plans (one persistent launch over many texts)
# ---------------------------------------------------------------------------

BATCH_SHAPES = [(512, 1), (1024, 1), (256, 2), (256, 1)]
BATCH_CHUNKS = [0, 512, 1024, 2048, 4096]   # 0: the plan's automatic chunk length


def batch_key(infos: List[dict], lens: List[int], device_name: str) -> str:
    """The automaton mix (states and classes of each distinct automaton,
    sorted) and the length histogram (texts per power-of-4 length bucket, in
    eighths of the batch), with the total size's bucket."""
    mix = sorted({(i["mode"], i["n_reachable"], i["ncls"]) for i in infos})
    hist: Dict[int, int] = {}
    for n in lens:
        b = 0 if n <= 0 else (max(n, 1).bit_length() + 1) // 2
        hist[b] = hist.get(b, 0) + 1
    k = max(len(lens), 1)
    q = ",".join(f"{b}:{round(8 * c / k)}" for b, c in sorted(hist.items()) if round(8 * c / k))
    return f"batch|{device_name}|{mix}|h{q}|n{bucket(sum(lens))}"


def batch_candidates() -> List[Dict[str, int]]:
    out = [{}]
    for th, ch in BATCH_SHAPES:
        for c in BATCH_CHUNKS:
            if th == 512 and ch == 1 and c == 0:
                continue   # the default plan, already first
            out.append({"block_threads": th, "chains": ch, "chunk_bytes": c})
    return out


def tune_batch(automata, texts, reps: int = 3, force: bool = False, verbose: bool = False) -> Dict[str, int]:
    """Best sfa_batch_create options for this batch (automata[i] matches
    texts[i], CUDA uint8 tensors), timed as CUDA-graph launches; every
    candidate must give the same results."""
    import torch
    infos = [a.info() for a in automata]
    lens = [int(t.numel()) for t in texts]
    dev = torch.cuda.get_device_name()
    key = batch_key(infos, lens, dev)
    with _LOCK:
        cache = _load()
        if not force and key in cache:
            return dict(cache[key]["shape"])
    out = empty_results(max(len(texts), 1))
    best, best_ms, ref = None, float("inf"), None
    for shape in batch_candidates():
        try:
            b = Batch(automata, texts, **shape)
        except SfaError:
            continue   # shape outside the automata's shared-memory budget
        try:
            for _ in range(2):
                b.launch(out, graph=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.launch(out, graph=True)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        finally:
            b.close()
        res = bytes(out.cpu().numpy())
        if ref is None:
            ref = res
        elif res != ref:
            raise RuntimeError(f"batch shape {shape} changed the results")
        if verbose:
            print(f"  {shape} {sum(lens) / ms / 1e6:.1f} GB/s", flush=True)
        if ms < best_ms:
            best, best_ms = shape, ms
    if best is None:
        return {}
    with _LOCK:
        cache = _load()
        cache[key] = {"shape": best, "ms": best_ms, "GBps": sum(lens) / best_ms / 1e6}
        _store(cache)
    return dict(best)
