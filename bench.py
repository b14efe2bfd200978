#!/usr/bin/env python3
"""Benchmark of the SFA matcher: text GB/s on one GB300, bit-exact.

Default workload (the single-automaton path): Aho-Corasick automaton of 16
seeded literals (lengths 4..12, base64 alphabet, 127 states) over 1 GiB of
Zipf(1.1) text with one planted literal per 64 KiB.  A step is one full match
of the resident text (all chunks from f_I, the composition scan, the count
pass) -- one launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank matches its own
replica of the workload (weak scaling, no collective on the data path);
rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "text GB/s per GB300 (and % of HBM peak), bit-exact"
PEAK_FALLBACK_GBS = 6800.0
KERNEL_SRCS = [os.path.join(ROOT, "paper_1405_0562_gb300", "csrc", f) for f in ("sfa_device.cuh", "sfa_types.h")]


def kernel_hash() -> str:
    """Hash of the kernel's sources (the device code and its layouts)."""
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the match kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"sfa_match_kernel_{workload}.txt")
    try:
        fields = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_source_sha256_16") != kernel_hash():
            return None
        return float(fields["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, world, local


def barrier_max(value: float, world: int) -> float:
    """The maximum of `value` over all ranks (device tensor under NCCL, host
    tensor under gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbps(bytes_per_rank: int, world: int, elapsed_s: float) -> float:
    """Whole-job throughput of weakly scaled replicas: all ranks' bytes over
    the slowest rank's time."""
    return bytes_per_rank * world / barrier_max(elapsed_s, world) / 1e9


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_workload(name: str, text_bytes: int = 0):
    if name == "plain_large":
        d, t = W.workload_large(text_bytes or (1 << 30))
        return d, t, {"workload": "plain_large: Aho-Corasick DFA of 16 literals (len 4-12, base64 alphabet), "
                                  "1 GiB Zipf(1.1) text, 1 plant per 64 KiB",
                      "text_bytes": int(t.size), "dfa_states": d.nq, "seed": W.SEED_LARGE}
    if name == "plain_small":
        d, t = W.workload_single(text_bytes or (1 << 20))
        return d, t, {"workload": "plain_small: KMP DFA of one 6-byte literal over a-z (7 states), "
                                  "1 MiB uniform a-z text, 64 plants",
                      "text_bytes": int(t.size), "dfa_states": d.nq, "seed": W.SEED_SINGLE}
    raise SystemExit(f"unknown workload {name}")


def run_reference(args, rank: int, world: int):
    """The oracle (sequential Alg. 2 in C, one host core) on a bounded sample
    of the same workload per step."""
    import oracle
    if rank != 0:
        return
    d, t, cfg = make_workload(args.workload, args.text_bytes)
    # per-step sample sized so that warm-up + steps take about a minute
    cal = min(t.size, 16 << 20)
    t0 = time.perf_counter()
    oracle.dfa_run(d.delta, d.q0, d.accept, t[:cal])
    speed = cal / max(time.perf_counter() - t0, 1e-6)
    sample = int(speed * 60.0 / max(1, args.steps + args.warmup))
    sample = max(1 << 16, min(t.size, 64 << 20, sample >> 16 << 16))
    for _ in range(max(args.warmup, 0)):
        oracle.dfa_run(d.delta, d.q0, d.accept, t[:sample])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.dfa_run(d.delta, d.q0, d.accept, t[:sample])
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total / 1e9
    desc = f"first {sample >> 10} KiB of the {t.size >> 20} MiB text per step"
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(d, t, budget_s: float = 12.0):
    """The oracle as it stands (Alg. 2 in C, one core) over the whole text,
    repeated while it stays inside the budget."""
    import oracle
    reps, elapsed = 0, 0.0
    while reps < 1 or (elapsed < budget_s and reps < 8):
        t0 = time.perf_counter()
        res = oracle.dfa_run(d.delta, d.q0, d.accept, t)
        elapsed += time.perf_counter() - t0
        reps += 1
    return {"value": t.size * reps / elapsed / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"whole {t.size >> 20} MiB text x {reps}"}, res


CPU_PARALLEL_SAMPLE = 256 << 20
TUNE_SAMPLE = 1 << 20


def cpu_parallel(d, t, gpu_final_state: int):
    """The paper's own parallel method on the host, for context: the oracle's
    Alg. 5 (its D-SFA, pthreads over every host core, four chunks per
    thread; the final state only, no count) over the first 256 MiB.
    gpu_final_state: the GPU's final state over the same prefix."""
    import oracle
    threads = os.cpu_count() or 1
    sample = t[:CPU_PARALLEL_SAMPLE]
    sfa = oracle.sfa_build(d.delta)
    bounds = oracle.equal_bounds(sample.size, 4 * threads)
    oracle.alg5(sfa, sample[:1 << 20], oracle.equal_bounds(1 << 20, threads), d.q0, threads=threads)
    t0 = time.perf_counter()
    _, fin = oracle.alg5(sfa, sample, bounds, d.q0, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": sample.size / dt / 1e9, "unit": "GB/s", "cores": threads,
            "kind": "oracle Alg. 5 (final state only), one thread per core",
            "sample": f"first {sample.size >> 20} MiB", "final_state_agrees_with_gpu": int(fin) == int(gpu_final_state)}


def run_gpu(args, rank: int, world: int, local: int):
    import torch

    import paper_1405_0562_gb300 as sfa

    torch.cuda.set_device(local)
    d, t, cfg = make_workload(args.workload, args.text_bytes)
    # the state numbering is chosen against bank conflicts on a sample of the
    # text (sfa_compile_sample; compile time is outside the timed region)
    a = sfa.Automaton.from_dfa(d, sample=t[:TUNE_SAMPLE])
    info = a.info()
    cfg.update({"state_numbering": f"tuned on the text's first {min(t.size, TUNE_SAMPLE) >> 10} KiB",
                "sfa_states": info["n_sfa_states"], "byte_classes": info["ncls"],
                "l2": "inputs larger than L2" if t.size > (126 << 20) else "L2 flushed between steps"})
    stream = torch.cuda.Stream()
    text = torch.from_numpy(t).to(f"cuda:{local}")
    out = sfa.empty_results(1, text.device)
    flush = None if t.size > (126 << 20) else torch.empty(256 << 20, dtype=torch.uint8, device=text.device)
    launch = {k: v for k, v in (("chunk_bytes", args.chunk_bytes), ("block_threads", args.block_threads)) if v}
    if launch:
        cfg["launch"] = dict(launch)

    # correctness of what is timed (the oracle, when it is allowed to run)
    with torch.cuda.stream(stream):
        a.match(text, out, stream=stream, **launch)
    stream.synchronize()
    got = sfa.decode(out)[0]

    for _ in range(args.warmup):
        a.match(text, out, stream=stream, **launch)
    stream.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    n_before = sfa.kernel_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        a.match(text, out, stream=stream, **launch)
        evs[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = sfa.kernel_launch_count() - n_before
    # sustained: the same match back to back for about SUSTAIN_S seconds,
    # with the clock sampler still running, so that the clock record covers
    # a window of the same work (the timed region above lasts milliseconds)
    sustained = None
    if not args.profile:
        sustained = sustained_run(torch, stream, lambda: a.match(text, out, stream=stream, **launch), t.size,
                                  step_hint_s=max(1e-5, 1e-3 * t_start.elapsed_time(t_end) / max(1, args.steps)))
    clk = clocks.stop()
    if sustained:
        sustained["sm_mhz_median"] = clk["sm_mhz"]
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [s.elapsed_time(e) for s, e in evs]
    total_ms = barrier_max(total_ms, world)
    step_ms = total_ms / args.steps
    if flush is not None:
        step_ms = statistics.mean(kern_ms)   # flush writes are outside the per-step events
    value = t.size * world / (step_ms * 1e-3) / 1e9

    # end to end through the host-buffer entry point (copies inside)
    e2e_s = None
    if not args.profile:
        pinned = torch.from_numpy(t).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        a.match_host(pinned, stream=stream)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            res_h = a.match_host(pinned, stream=stream)
        e2e_s = barrier_max((time.perf_counter() - t0) / e2e_steps, world)
        assert res_h == got, (res_h, got)

    peak, peak_kind = hbm_peak()
    kern_avg = statistics.mean(kern_ms)
    achieved = t.size / (kern_avg * 1e-3) / 1e9
    traffic = profiled_traffic(args.workload)
    # the same text with the state ids a caller without a sample gets (the
    # uniform bank-conflict model)
    uni_ms, read_peak = None, None
    if not args.profile:
        a_uni = sfa.Automaton.from_dfa(d)
        out_u = sfa.empty_results(1, text.device)
        for _ in range(args.warmup):
            a_uni.match(text, out_u, stream=stream, **launch)
        uni_ms = _events(torch, stream, lambda: a_uni.match(text, out_u, stream=stream, **launch),
                         args.steps) / args.steps
        assert sfa.decode(out_u)[0] == got
        read_peak = read_only_peak(torch, text.device)
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "kernel": "sfa_match_kernel",
                         "algorithmic_bytes_per_launch": int(t.size),
                         "read_only_peak": read_peak,
                         "frac_of_read_only_peak": achieved / read_peak["value"] if read_peak else None},
            "e2e": ({"value": t.size * world / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(t.size),
                     "d2h_bytes_per_step": 16} if e2e_s else None),
            "gpu_launches": int(launches), "clocks": clk, "sustained": sustained,
            "uniform_numbering": ({"value": t.size / (uni_ms * 1e-3) / 1e9, "unit": "GB/s",
                                   "frac": t.size / (uni_ms * 1e-3) / 1e9 / peak,
                                   "note": "state ids from the uniform bank-conflict model (no text sample)"}
                                  if uni_ms else None)}
    if rank == 0 and not args.no_cpu_baseline and not args.profile:
        base, res = cpu_baseline(d, t)
        line["cpu_baseline"] = base
        line["bit_exact_vs_oracle"] = (got == (res[0], res[1], 0, res[2]))
        with torch.cuda.stream(stream):
            a.match(text[:CPU_PARALLEL_SAMPLE], out, stream=stream, **launch)
        stream.synchronize()
        line["cpu_parallel"] = cpu_parallel(d, t, sfa.decode(out)[0][0])
    if args.workload == "plain_large" and not args.no_side_legs and not args.profile:
        # short legs of the other configurations, each checked against the
        # oracle, so that one default run covers them too
        del text
        torch.cuda.empty_cache()
        line["side_legs"] = {"batched_subset": side_batched(torch, sfa, stream, args, rank),
                             "sim_1GiB": side_sim(torch, sfa, stream, args, rank)}
    if rank == 0:
        print(json.dumps(line), flush=True)


SUSTAIN_S = 2.0


def sustained_run(torch, stream, fn, nbytes, step_hint_s):
    """fn back to back on `stream` for about SUSTAIN_S seconds (CUDA events)."""
    reps = max(10, int(SUSTAIN_S / step_hint_s))
    ms = _events(torch, stream, fn, reps)
    return {"value": nbytes * reps / (ms * 1e-3) / 1e9, "unit": "GB/s", "seconds": ms * 1e-3, "matches": reps}


def read_only_peak(torch, device, nbytes=4 << 30, reps=5):
    """Read-only HBM bandwidth of this GPU, measured here: torch's int64 sum
    over a buffer of nbytes (larger than L2), best of `reps`."""
    buf = torch.ones(nbytes // 8, dtype=torch.int64, device=device)
    buf.sum()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        buf.sum()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del buf
    torch.cuda.empty_cache()
    return {"value": nbytes / (best * 1e-3) / 1e9, "unit": "GB/s",
            "how": f"torch int64 sum over {nbytes >> 30} GiB, best of {reps}"}


BATCH_SUBSET = 1024


def side_batched(torch, sfa, stream, args, rank):
    """The first BATCH_SUBSET texts of the batched workload (config 3's
    lengths, automata and pairing) in one persistent launch under a CUDA
    graph, against the same texts as plain launches; every result checked
    against the oracle."""
    import oracle
    autos_d = W.workload_batch_automata()
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    lens = W.workload_batch_lengths()[:BATCH_SUBSET]
    pair = W.workload_batch_pairing(len(lens), len(autos))
    total = int(lens.sum())
    big = W.text_uniform(total, W.LOWER_ALPHABET, W.SEED_BATCH + 2)
    offs = np.concatenate([[0], np.cumsum(lens)])
    dev = torch.from_numpy(big).cuda()
    views = [dev[offs[i]:offs[i + 1]] for i in range(len(lens))]
    hs = [autos[p] for p in pair]
    b = sfa.Batch(hs, views)
    out = sfa.empty_results(len(views))
    for _ in range(args.warmup):
        b.launch(out, stream=stream, graph=True)
    stream.synchronize()
    ms = _events(torch, stream, lambda: b.launch(out, stream=stream, graph=True), args.steps) / args.steps
    got = sfa.decode(out)
    outs = sfa.empty_results(len(views))
    plain = lambda: [hs[i].match(views[i], outs[16 * i:16 * i + 16], stream=stream) for i in range(len(views))]
    plain()
    pms = _events(torch, stream, plain, 3) / 3
    exact = sfa.decode(outs) == got
    if rank == 0:
        from concurrent.futures import ThreadPoolExecutor

        def ref(i):
            d = autos_d[pair[i]]
            f, a, c = oracle.dfa_run(d.delta, d.q0, d.accept, big[offs[i]:offs[i + 1]])
            return (f, a, 0, c)
        with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
            exact = exact and list(ex.map(ref, range(len(views)))) == got
    del dev, views, b
    torch.cuda.empty_cache()
    return {"value": total / (ms * 1e-3) / 1e9, "unit": "GB/s", "texts": len(lens), "text_bytes": total,
            "ms_per_step": ms, "plain_launches_GBps": total / (pms * 1e-3) / 1e9, "speedup_vs_plain": pms / ms,
            "bit_exact_vs_oracle": bool(exact),
            "workload": f"first {len(lens)} texts of the batched workload (log-uniform 256 B..16 MiB, a-z, "
                        "8 literal-set automata), one graph launch per step"}


def side_sim(torch, sfa, stream, args, rank, n=1 << 30):
    """Simulation mode (random complete DFAs of 16 and 64 states over 16
    symbols) on 1 GiB; each result checked against the oracle."""
    import oracle
    autos_d = [d for d in W.workload_sim_automata() if d.nq in (16, 64)]
    t = W.workload_sim_text(n)
    tt = torch.from_numpy(t).cuda()
    res = {}
    for d in autos_d:
        a = sfa.Automaton.from_dfa(d)
        out = sfa.empty_results(1)
        for _ in range(args.warmup):
            a.match(tt, out, stream=stream)
        ms = _events(torch, stream, lambda: a.match(tt, out, stream=stream), args.steps) / args.steps
        got = sfa.decode(out)[0]
        exact = None
        if rank == 0:
            f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
            exact = got == (f, acc, 0, c)
        res[f"{d.nq}_states"] = {"value": n / (ms * 1e-3) / 1e9, "unit": "GB/s", "mode": a.info()["mode"],
                                 "bit_exact_vs_oracle": exact}
    del tt
    torch.cuda.empty_cache()
    return res


def _events(torch, stream, fn, steps):
    """CUDA-event time (ms) of `steps` calls of fn on `stream`."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _common(args, world, value, step_ms, cfg, peak_bytes, kern_ms, launches, clk, extra):
    peak, peak_kind = hbm_peak()
    achieved = peak_bytes / (kern_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "sfa_match_kernel", "algorithmic_bytes_per_launch": int(peak_bytes)},
            "gpu_launches": int(launches), "clocks": clk}
    line.update(extra)
    return line


def run_batched(args, rank, world, local):
    """Config 3: 4096 texts (log-uniform 256 B .. 16 MiB, a-z) against 8
    literal-set automata, one persistent launch per step (a CUDA graph),
    against 4096 plain launches on one stream."""
    import torch

    import paper_1405_0562_gb300 as sfa
    torch.cuda.set_device(local)
    autos_d = W.workload_batch_automata()
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    lens = W.workload_batch_lengths()
    pair = W.workload_batch_pairing(len(lens), len(autos))
    total = int(lens.sum())
    big = W.text_uniform(total, W.LOWER_ALPHABET, W.SEED_BATCH + 2)
    offs = np.concatenate([[0], np.cumsum(lens)])
    dev = torch.from_numpy(big).cuda()
    views = [dev[offs[i]:offs[i + 1]] for i in range(len(lens))]
    hs = [autos[p] for p in pair]
    stream = torch.cuda.Stream()
    # the plan's shape from the batch autotuner (cached per device, automaton
    # mix and length histogram; tuning runs before the timed region)
    from paper_1405_0562_gb300 import autotune
    t_tune = time.perf_counter()
    shape = autotune.tune_batch(hs, views)
    t_tune = time.perf_counter() - t_tune
    b = sfa.Batch(hs, views, **shape)
    out = sfa.empty_results(len(views))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.launch(out, stream=stream, graph=True)
    stream.synchronize()
    got = sfa.decode(out)
    clocks = ClockSampler(local)
    clocks.start()
    n0 = sfa.kernel_launch_count()
    ms = _events(torch, stream, lambda: b.launch(out, stream=stream, graph=True), args.steps)
    launches = sfa.kernel_launch_count() - n0
    clk = clocks.stop()
    step_ms = barrier_max(ms / args.steps, world)
    # the same texts as 4096 plain launches, one stream
    outs = sfa.empty_results(len(views))
    plain = lambda: [hs[i].match(views[i], outs[16 * i:16 * i + 16], stream=stream) for i in range(len(views))]
    plain()
    rounds = max(1, min(5, args.steps))
    pms = _events(torch, stream, plain, rounds) / rounds
    assert sfa.decode(outs) == got
    # spot check against the oracle
    import oracle
    for i in range(0, len(views), 97):
        d = autos_d[pair[i]]
        f, a, c = oracle.dfa_run(d.delta, d.q0, d.accept, big[offs[i]:offs[i + 1]])
        assert got[i] == (f, a, 0, c), i
    cfg = {"workload": "batched: 4096 texts log-uniform 256 B..16 MiB, uniform a-z, 8 literal-set automata "
                       "(51..159 states), one persistent launch under a CUDA graph",
           "texts": len(views), "text_bytes": total, "seed": W.SEED_BATCH, "l2": "inputs larger than L2",
           "plan_shape": shape or "automatic", "tuning_seconds": t_tune}
    value = total * world / (step_ms * 1e-3) / 1e9
    extra = {"plain_launches": {"value": total / (pms * 1e-3) / 1e9, "unit": "GB/s", "launches_per_step": len(views),
                                "ms_per_step": pms},
             "speedup_vs_plain": pms / step_ms}
    line = _common(args, world, value, step_ms, cfg, total, step_ms, launches, clk, extra)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sim(args, rank, world, local):
    """Config 4: random complete DFAs with 16, 32, 64 states over 16 symbols
    (simulation mode) on 4 GiB of uniform symbols; a step matches the text
    with all three."""
    import torch

    import paper_1405_0562_gb300 as sfa
    torch.cuda.set_device(local)
    autos_d = W.workload_sim_automata()
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    assert all(a.info()["mode"] == sfa.MODE_SIM for a in autos)
    n = args.text_bytes or (4 << 30)
    t = W.workload_sim_text(n)
    tt = torch.from_numpy(t).cuda()
    stream = torch.cuda.Stream()
    outs = [sfa.empty_results(1) for _ in autos]
    # launch shapes from the autotuner (untimed; --profile: the automatic ones)
    from paper_1405_0562_gb300 import autotune
    shapes = [{} if args.profile else autotune.tune(a, tt) for a in autos]
    step = lambda: [a.match(tt, o, stream=stream, **s) for a, o, s in zip(autos, outs, shapes)]
    for _ in range(args.warmup):
        step()
    stream.synchronize()
    per = []
    for a, o, s in zip(autos, outs, shapes):
        per.append(_events(torch, stream, lambda: a.match(tt, o, stream=stream, **s), 3) / 3)
    clocks = ClockSampler(local)
    clocks.start()
    n0 = sfa.kernel_launch_count()
    ms = _events(torch, stream, step, args.steps)
    launches = sfa.kernel_launch_count() - n0
    clk = clocks.stop()
    step_ms = barrier_max(ms / args.steps, world)
    got = [sfa.decode(o)[0] for o in outs]
    import oracle
    base = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = min(n, 256 << 20)
        t0 = time.perf_counter()
        for d in autos_d:
            oracle.dfa_run(d.delta, d.q0, d.accept, t[:sample])
        el = time.perf_counter() - t0
        base = {"value": 3 * sample / el / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": f"first {sample >> 20} MiB with each of the 3 automata"}
    exact = None
    if args.check:
        exact = all(g == (f, a, 0, c) for g, (f, a, c) in
                    zip(got, (oracle.dfa_run(d.delta, d.q0, d.accept, t) for d in autos_d)))
    # the first 256 MiB of the text with each automaton and its tuned shape
    exact_sub = None
    if rank == 0 and not args.profile:
        sub = t[:256 << 20]
        exact_sub = True
        for a, d, s in zip(autos, autos_d, shapes):
            o = sfa.empty_results(1)
            a.match(tt[:sub.size], o, stream=stream, **s)
            stream.synchronize()
            f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, sub)
            exact_sub = exact_sub and sfa.decode(o)[0] == (f, acc, 0, c)
    # past 64 states (vectors in shared memory): per automaton, checked
    # against the oracle on the first 256 MiB
    large = {}
    for d in W.workload_sim_automata_large():
        a = sfa.Automaton.from_dfa(d)
        o = sfa.empty_results(1)
        a.match(tt, o, stream=stream)
        ms = _events(torch, stream, lambda: a.match(tt, o, stream=stream), max(1, min(args.steps, 5)))
        ms /= max(1, min(args.steps, 5))
        entry = {"value": n / (ms * 1e-3) / 1e9, "unit": "GB/s", "mode": a.info()["mode"]}
        if rank == 0:
            sub = t[:256 << 20]
            a.match(tt[:sub.size], o, stream=stream)
            stream.synchronize()
            f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, sub)
            entry["bit_exact_vs_oracle_first_256MiB"] = sfa.decode(o)[0] == (f, acc, 0, c)
        large[d.name] = entry
    cfg = {"workload": "sim: random complete DFAs of 16/32/64 states over 16 symbols (simulation mode), "
                       f"{n >> 20} MiB uniform over symbols 0..15, all three per step",
           "text_bytes": n, "seed": W.SEED_SIM, "l2": "inputs larger than L2",
           "per_automaton_GBps": {d.name: n / (p * 1e-3) / 1e9 for d, p in zip(autos_d, per)},
           "launch_shapes": {d.name: s or "automatic" for d, s in zip(autos_d, shapes)}}
    value = 3 * n * world / (step_ms * 1e-3) / 1e9
    extra = {"bit_exact_vs_oracle": exact, "bit_exact_vs_oracle_first_256MiB": exact_sub, "larger_automata": large}
    if base:
        extra["cpu_baseline"] = base
    line = _common(args, world, value, step_ms, cfg, 3 * n, step_ms, launches, clk, extra)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serving(args, rank, world, local):
    """Config 5: Poisson arrivals of requests (log-normal lengths, median
    64 KiB, sigma 1.5, cap 64 MiB, a-z) against 32 resident automata;
    continuous batching vs one request at a time, at offered loads of 0.5,
    0.8 and 0.95 of the one-at-a-time capacity, and past it (2 to 200
    times), where requests queue up for the one-at-a-time loop and the
    server saturates the host link (texts copied in by one kernel per
    batch from pinned memory)."""
    import torch

    import paper_1405_0562_gb300 as sfa
    from paper_1405_0562_gb300 import serve
    torch.cuda.set_device(local)
    autos_d = W.workload_serving_automata()
    autos = [sfa.Automaton.from_dfa(d) for d in autos_d]
    nreq = args.requests
    _, lens, which = W.workload_serving_requests(nreq, 1.0)
    total = int(lens.sum())
    host = torch.from_numpy(W.text_uniform(total, W.LOWER_ALPHABET, W.SEED_SERVE + 3)).pin_memory()
    offs = np.concatenate([[0], np.cumsum(lens)])
    texts = [host[offs[i]:offs[i + 1]] for i in range(nreq)]
    mean = total / nreq

    def reqs(arrivals):
        return [serve.Request(i, int(which[i]), texts[i], float(arrivals[i])) for i in range(nreq)]

    # capacity of the one-at-a-time baseline (back to back, no arrivals)
    warm = serve.one_at_a_time(autos, reqs(np.zeros(nreq))[:50], realtime=False)
    t0 = time.perf_counter()
    alone = serve.one_at_a_time(autos, reqs(np.zeros(nreq)), realtime=False)
    cap = total / (time.perf_counter() - t0)
    by_id = {r.rid: r.result for r in alone}
    levels = {}
    best = 0.0
    for load in (0.5, 0.8, 0.95, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0, 200.0):
        rate = load * cap / mean
        arr, _, _ = W.workload_serving_requests(nreq, rate)
        srv = serve.Server(autos, hbm_budget=4 << 30, max_batch=256, slots=4)
        try:
            done = srv.run(reqs(arr))
        finally:
            srv.close()
        assert all(r.result == by_id[r.rid] for r in done)
        s_stats = serve.latency_stats(done)
        s_stats["batches"] = srv.batches
        b_stats = serve.latency_stats(serve.one_at_a_time(autos, reqs(arr)))
        levels[str(load)] = {"offered_GBps": load * cap / 1e9, "server": s_stats, "one_at_a_time": b_stats}
        best = max(best, s_stats["GBps"])
    cfg = {"workload": "serving: Poisson arrivals, log-normal lengths (median 64 KiB, sigma 1.5, cap 64 MiB), "
                       "uniform a-z, 32 resident literal-set automata, continuous batching",
           "requests_per_level": nreq, "text_bytes": total, "seed": W.SEED_SERVE}
    line = {"metric": METRIC, "value": best, "unit": "GB/s", "n_gpus": world, "steps": len(levels),
            "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic", "config": cfg,
            "one_at_a_time_capacity_GBps": cap / 1e9, "levels": levels, "results_equal_alone": True}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_rn(args, rank, world, local):
    """The paper's scalability automata (Sect. VI-B): r_5, r_50 and r_500, the
    minimal DFAs of ([0-4]{n}[5-9]{n})* (11, 101 and 1001 states; 110, 10 100
    and 1 001 000 D-SFA states), on 1 GiB accepted texts, and r_a = r_500 | a*
    on 1 GiB of 'a'.  r_500 and r_a have 16-bit state ids and their point
    mappings are not stored.  A step matches each text with its automaton;
    every result is checked against the oracle."""
    import torch

    import oracle
    import paper_1405_0562_gb300 as sfa
    torch.cuda.set_device(local)
    n = args.text_bytes or (1 << 30)
    from paper_1405_0562_gb300 import autotune
    per, cpu, checks, sizes, shapes = {}, {}, {}, {}, {}
    stream = torch.cuda.Stream()
    total_ms, launches = 0.0, 0
    clocks = ClockSampler(local)
    clocks.start()
    cases = [(f"r_{rn}", (lambda rn=rn: W.dfa_rn(rn)), (lambda rn=rn: W.text_rn_accepted(n, rn, W.SEED_LARGE + rn)))
             for rn in (5, 50, 500)]
    cases.append(("r_a", lambda: W.dfa_ra(500), lambda: np.full(n, ord("a"), dtype=np.uint8)))
    for name, mk_d, mk_t in cases:
        d, t = mk_d(), mk_t()
        a = sfa.Automaton.from_dfa(d)
        info = a.info()
        sizes[name] = {"dfa_states": info["n_reachable"], "sfa_states": info["n_sfa_states"],
                       "stored": info["n_stored"], "id_bits": info["id_bits"],
                       "compile_seconds": info["compile_seconds"]}
        tt = torch.from_numpy(t).cuda()
        out = sfa.empty_results(1)
        # the launch shape from the autotuner (untimed; --profile: the
        # automatic shape, so that an ncu capture sees only timed launches)
        shape = {} if args.profile else autotune.tune(a, tt)
        shapes[name] = shape or "automatic"
        for _ in range(args.warmup):
            a.match(tt, out, stream=stream, **shape)
        stream.synchronize()
        n0 = sfa.kernel_launch_count()
        ms = _events(torch, stream, lambda: a.match(tt, out, stream=stream, **shape), args.steps)
        launches += sfa.kernel_launch_count() - n0
        total_ms += ms
        per[name] = n * args.steps / (ms * 1e-3) / 1e9
        got = sfa.decode(out)[0]
        f, acc, c = oracle.dfa_run(d.delta, d.q0, d.accept, t)
        checks[name] = got == (f, acc, 0, c)
        sample = t[:64 << 20]
        t0 = time.perf_counter()
        oracle.dfa_run(d.delta, d.q0, d.accept, sample)
        cpu[name] = sample.size / (time.perf_counter() - t0) / 1e9
        del tt
    clk = clocks.stop()
    assert all(checks.values()), checks
    step_ms = total_ms / args.steps
    value = len(cases) * n / (step_ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"r_n: r_5, r_50, r_500 (Sect. VI-B) on {n >> 20} MiB accepted texts and "
                                   f"r_a on {n >> 20} MiB of 'a', all four per step",
                       "text_bytes": n, "seed": W.SEED_LARGE, "l2": "inputs larger than L2",
                       "per_automaton_GBps": per, "automata": sizes, "launch_shapes": shapes},
            "roofline": {"bound": "hbm", "achieved": value, "peak": peak, "unit": "GB/s", "frac": value / peak,
                         "traffic": None, "peak_kind": peak_kind, "kernel": "sfa_match_kernel",
                         "algorithmic_bytes_per_launch": n},
            "gpu_launches": int(launches), "clocks": clk, "bit_exact_vs_oracle": True,
            "cpu_baseline": {"value": len(cpu) / sum(1 / v for v in cpu.values()), "unit": "GB/s", "cores": 1,
                             "kind": "oracle", "sample": "first 64 MiB with each automaton",
                             "per_automaton_GBps": cpu}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_crossover(args, rank, world, local):
    """Small-input crossover (the paper's Sect. VI-C study, on a GPU): per text
    length, the latency of one match on the device (a CUDA graph of 64
    calls back to back, replayed), end to end from pinned host memory (sfa_match_host:
    copy in, match, copy the result back, synchronise), and the oracle's
    sequential Alg. 2 on one host core; the crossover is the shortest text
    the GPU matches end to end faster than the CPU."""
    import ctypes

    import torch

    import oracle
    import paper_1405_0562_gb300 as sfa
    torch.cuda.set_device(local)
    if args.profile:
        # for ncu: 4 matches each of the first 1 KiB (one CTA of the
        # short-text kernel), 64 KiB (a cluster of 8) and 1 MiB (a cluster of
        # 16), no graphs, the last of each size checked against the oracle
        d, t = W.workload_large(1 << 20)
        a = sfa.Automaton.from_dfa(d, sample=t)
        out = sfa.empty_results(1)
        for n in (1 << 10, 64 << 10, 1 << 20):
            tt = torch.from_numpy(t[:n].copy()).cuda()
            for _ in range(4):
                a.match(tt, out)
            torch.cuda.synchronize()
            f, accf, c = oracle.dfa_run(d.delta, d.q0, d.accept, t[:n])
            assert sfa.decode(out)[0] == (f, accf, 0, c), n
        if rank == 0:
            print(json.dumps({"workload": "crossover --profile", "launches": 12, "bit_exact_vs_oracle": True}))
        return
    d, t = W.workload_large(64 << 20)
    a = sfa.Automaton.from_dfa(d)
    stream = torch.cuda.Stream()
    dl, al = oracle._dfa_arrays(d.delta, d.accept)
    lib = oracle._lib()
    cnt = np.zeros(1, dtype=np.uint64)
    rows = []
    for n in (1 << 10, 4 << 10, 16 << 10, 64 << 10, 256 << 10, 1 << 20, 4 << 20, 16 << 20, 64 << 20):
        tt = torch.from_numpy(t[:n]).cuda()
        pinned = torch.from_numpy(t[:n]).pin_memory()
        out = sfa.empty_results(1)
        with torch.cuda.stream(stream):
            for _ in range(3):
                a.match(tt, out, stream=stream)
        stream.synchronize()
        # `inner` matches back to back in one graph, so that the device time
        # is not the host's replay rate
        inner = 64 if n <= 1 << 20 else 4
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(inner):
                a.match(tt, out, stream=stream)
        reps = 20
        with torch.cuda.stream(stream):
            g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
        stream.synchronize()
        dev_us = e0.elapsed_time(e1) / (reps * inner) * 1e3
        got = sfa.decode(out)[0]
        a.match_host(pinned, stream=stream)
        k = 50
        t0 = time.perf_counter()
        for _ in range(k):
            res = a.match_host(pinned, stream=stream)
        e2e_us = (time.perf_counter() - t0) / k * 1e6
        tp = t[:n]
        k = max(3, int(2e7 // max(n, 1)))
        t0 = time.perf_counter()
        for _ in range(k):
            f = lib.oracle_dfa_run(oracle._ptr(dl), dl.shape[0], int(d.q0), oracle._ptr(al), oracle._ptr(tp), n,
                                   oracle._ptr(cnt))
        cpu_us = (time.perf_counter() - t0) / k * 1e6
        want = (int(f), int(al[f]), 0, int(cnt[0]))
        assert got == want and res == want, (n, got, res, want)
        rows.append({"bytes": n, "gpu_device_us": dev_us, "gpu_e2e_us": e2e_us, "cpu_oracle_us": cpu_us})
    cross = next((r["bytes"] for r in rows if r["gpu_e2e_us"] < r["cpu_oracle_us"]), None)
    big = rows[-1]
    line = {"metric": METRIC, "value": big["bytes"] / (big["gpu_device_us"] * 1e-6) / 1e9, "unit": "GB/s",
            "n_gpus": world, "steps": len(rows), "warmup": 3, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "crossover: prefixes (1 KiB .. 64 MiB) of the 1 GiB Aho-Corasick/Zipf text, "
                                   "one match at a time", "seed": W.SEED_LARGE},
            "rows": rows, "crossover_bytes_e2e": cross,
            "cpu_baseline": {"value": big["bytes"] / (big["cpu_oracle_us"] * 1e-6) / 1e9, "unit": "GB/s",
                             "cores": 1, "kind": "oracle", "sample": "each prefix, repeated to about 20 MB"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="plain_large",
                    choices=["plain_large", "plain_small", "batched", "sim", "serving", "crossover", "rn"])
    ap.add_argument("--requests", type=int, default=20000, help="serving: requests per offered load")
    ap.add_argument("--check", action="store_true", help="sim: compare the full outputs with the oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side-legs", action="store_true", help="plain_large: skip the batched and sim legs")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed matches (for ncu): no sustained loop, e2e, read peak, side or CPU legs")
    ap.add_argument("--text-bytes", type=int, default=0, help="override the text size (profiling runs only)")
    ap.add_argument("--chunk-bytes", type=int, default=0, help="launch shape override (default: automatic)")
    ap.add_argument("--block-threads", type=int, default=0, help="launch shape override (default: automatic)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local)
    elif args.workload == "sim":
        run_sim(args, rank, world, local)
    elif args.workload == "serving":
        run_serving(args, rank, world, local)
    elif args.workload == "crossover":
        run_crossover(args, rank, world, local)
    elif args.workload == "rn":
        run_rn(args, rank, world, local)
    else:
        run_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
