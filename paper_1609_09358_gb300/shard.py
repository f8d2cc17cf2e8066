"""Replica sharding of a decoding job over ranks.

Frames are independent (inter-frame parallelism of Sec. II-B) and the method has no exchange
step, so a multi-GPU job is N replicas: rank r decodes its own contiguous range of frame indices
of the counter-based generator (weak scaling: the frames per rank are fixed).  The only
cross-rank operations are host-side measurement reductions -- the slowest rank's time and sums
of error counters -- never on the decoding path.
"""
from __future__ import annotations


def frame_range(rank: int, world: int, frames_per_rank: int) -> tuple[int, int]:
    """(first frame index, count) of `rank`: ranks own consecutive, disjoint ranges."""
    if not 0 <= rank < world or frames_per_rank < 0:
        raise ValueError("rank %d of %d, %d frames" % (rank, world, frames_per_rank))
    return rank * frames_per_rank, frames_per_rank


def _reduce(values, op, dist, device):
    import torch
    t = torch.tensor(values, dtype=torch.float64 if op == "max" else torch.int64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.tolist()


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The job's time: the largest of the ranks' values (device: CUDA for NCCL, CPU for gloo)."""
    return float(_reduce([value], "max", dist, device)[0])


def sum_over_ranks(counts: dict, dist=None, device="cpu") -> dict:
    """Integer counters (frames, frame errors, bit errors, fallbacks) summed over the ranks."""
    keys = sorted(counts)
    out = _reduce([int(counts[k]) for k in keys], "sum", dist, device)
    return dict(zip(keys, (int(v) for v in out)))
