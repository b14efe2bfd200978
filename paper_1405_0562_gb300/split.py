"""One text split over several processes, one GPU each (Lemma 1, Theorem 3).

The text is cut into contiguous slices, one per rank.  The only exchange is
one all-gather of the slices' mappings (nq int32 each):

1. every rank matches its slice in map mode (``sfa_match_map``): the slice's
   mapping delta^(., w_r) over the states reachable from q0, and its result
   from q0;
2. all-gather of the mappings;
3. rank r's entering state is the mappings of ranks 0..r-1 applied in order
   to q0 (the reverse composition of Lemma 1); rank 0 enters in q0 and keeps
   its map-mode result, every other rank matches its slice again from its
   entering state (``sfa_match_continue`` from a record {s, count 0});
4. one all-reduce sums the counts; the last rank's final state is the text's.

By Theorem 3 the result equals the whole text's, wherever it was cut.  The
arithmetic of step 3 is host-side and on nq integers; every pass over text
runs in the library's kernels.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

RESULT_BYTES = 16


def entering_states(maps: Sequence[np.ndarray], q0: int) -> list:
    """The entering state of every slice: s_0 = q0, s_{r+1} = maps[r][s_r].
    maps[r][q] is the state after slice r entered in q (-1: q unreachable,
    which an entering state never is)."""
    s = [int(q0)]
    for m in maps[:-1]:
        nxt = int(m[s[-1]])
        if nxt < 0:
            raise ValueError("a slice mapping sends a reachable state to an unreachable one")
        s.append(nxt)
    return s


def result_record(final_state: int, count: int = 0) -> np.ndarray:
    """The 16 bytes of an sfa_result {final_state, accept 0, status 0, count}
    (the accept bit of a carried record is not read)."""
    rec = np.zeros(RESULT_BYTES, dtype=np.uint8)
    rec[:4] = np.frombuffer(np.uint32(final_state).tobytes(), dtype=np.uint8)
    rec[8:] = np.frombuffer(np.uint64(count).tobytes(), dtype=np.uint8)
    return rec


def match_split(automaton, text, q0: int, group=None, stream=None):
    """Match this rank's slice `text` of a text split over the ranks of
    `group` (in rank order) and return the whole text's
    (final_state, accept_final, status, count) on every rank.

    automaton: a ``paper_1405_0562_gb300.Automaton`` (or an object with the
    same match_map / match_continue methods); q0 its initial state."""
    import torch
    import torch.distributed as dist

    from . import decode

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    out, m = automaton.match_map(text, stream=stream)
    on_device = dist.get_backend(group) == "nccl"
    if stream is not None and hasattr(stream, "synchronize"):
        stream.synchronize()
    local = m if on_device else m.cpu()
    gathered = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(gathered, local, group=group)
    maps = [g.cpu().numpy() for g in gathered]
    s = entering_states(maps, q0)[rank]
    if rank > 0:
        rec = torch.from_numpy(result_record(s)).to(out.device)
        out = automaton.match_continue(text, rec, stream=stream)
    if stream is not None and hasattr(stream, "synchronize"):
        stream.synchronize()
    final, acc, status, count = decode(out)[0]
    # the count is summed; the status is the worst; final state and accept
    # bit come from the last slice
    dev = out.device if on_device else "cpu"
    total = torch.tensor([count], dtype=torch.int64, device=dev)
    worst = torch.tensor([status], dtype=torch.int64, device=dev)
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(worst, op=dist.ReduceOp.MAX, group=group)
    last = torch.tensor([final, acc], dtype=torch.int64, device=dev)
    src = world - 1 if group is None else dist.get_global_rank(group, world - 1)
    dist.broadcast(last, src=src, group=group)
    last = last.cpu()
    return int(last[0]), int(last[1]), int(worst.item()), int(total.item())
