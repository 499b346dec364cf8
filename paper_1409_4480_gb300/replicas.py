"""Data-parallel replicas: one process per GPU, packets split by id.

Packets are independent and every random number is keyed by the packet id, so
a solve split into disjoint id ranges over R processes gives, after summing the
tallies, the result of the unsplit solve: integer tallies (escape spectrum,
outcome counters) exactly, FP64 peel-off tallies up to summation order.  The
only exchange is that sum, done here with torch.distributed on host tensors
(gloo or nccl process groups); no collective runs inside the transport.
"""
from __future__ import annotations

import numpy as np

INT_KEYS = ("spec", "n_emitted", "n_escaped", "n_absorbed", "n_capped", "n_scat", "n_scat_hi", "spec_under",
            "spec_over")
FLOAT_KEYS = ("cam_spec", "cam_spec2", "cam_image")


def packet_range(n_packets: int, rank: int, world: int):
    """(first packet id, count) of replica `rank` out of `world` for a solve of
    n_packets packets: contiguous ranges, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(int(n_packets), world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def allreduce_tallies(result: dict, group=None) -> dict:
    """Sum one replica's tallies over the process group (every rank gets the
    total).  Keys missing from `result` are skipped."""
    import torch
    import torch.distributed as dist

    out = dict(result)
    for keys, dt in ((INT_KEYS, torch.int64), (FLOAT_KEYS, torch.float64)):
        for k in keys:
            if k not in result or result[k] is None:
                continue
            a = np.asarray(result[k])
            t = torch.from_numpy(np.ascontiguousarray(a).astype(np.int64 if dt == torch.int64 else np.float64))
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            v = t.numpy()
            out[k] = v if a.ndim else v.item()
    return out
