"""Autotuner for the launch shape of a match: block size, chunks per thread
and chunk length, timed with CUDA events on the device, cached in a JSON
file keyed by (device, automaton shape, text-size bucket).

    from paper_1405_0562_gb300 import autotune
    shape = autotune.tune(automaton, text_cuda_u8)       # dict of launch options
    out = automaton.match(text_cuda_u8, **shape)

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

from . import MODE_SIM, TILING_WARP, SfaError, empty_results

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
    long texts), then CTA shapes with fixed chunk lengths, then warp tiles."""
    sim = info["mode"] == MODE_SIM
    shapes = SIM_SHAPES if sim else SFA_SHAPES
    chunks = SIM_CHUNKS if sim else SFA_CHUNKS
    out = [{}]
    for th, ch in shapes:
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
