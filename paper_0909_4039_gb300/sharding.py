"""Independent instances of a batch spread over ranks (one GPU each).

The instances of a batch share nothing on the data path, so a multi-GPU run
needs no collective while it steps: every rank advances its own share of the
instances with one teuk_batch per GPU.  The only exchange is at the end, a
host gather of the per-instance waveforms.  This is the data-parallel
decomposition over independent problems (Sec. 4 of the paper, there over
grid points of one problem).

partition() is a deterministic longest-processing-time greedy on the
instances' grid points, so every rank computes the same assignment without
communicating.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def partition(weights: Sequence[float], nranks: int) -> List[List[int]]:
    """Instance indices per rank.  Instances are taken in decreasing weight
    (ties by index) and each goes to the rank with the least load so far
    (ties by rank), so the largest rank load exceeds the mean by at most the
    largest single weight."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(weights)), key=lambda k: (-float(weights[k]), k))
    load = [0.0] * nranks
    out: List[List[int]] = [[] for _ in range(nranks)]
    for k in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += float(weights[k])
    return [sorted(x) for x in out]


def local_instances(weights: Sequence[float], rank: int, nranks: int) -> List[int]:
    """This rank's instance indices."""
    if not 0 <= rank < nranks:
        raise ValueError("rank out of range")
    return partition(weights, nranks)[rank]


def gather_waveforms(local: Dict[int, object], group=None) -> Dict[int, object]:
    """Merge every rank's {instance index: waveform} on every rank
    (torch.distributed object all-gather; works on gloo and NCCL).  An
    instance reported by two ranks is an error."""
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return dict(local)
    parts: list = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, dict(local), group=group)
    merged: Dict[int, object] = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"instance {k} was stepped on two ranks")
            merged[k] = v
    return merged
