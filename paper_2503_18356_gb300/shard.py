"""Multi-rank plumbing of the ensemble path (host logic only, no RACIPE
arithmetic).

Every (parameter set, IC) solve is independent and the dedupe is per set, so
ranks take contiguous ranges of parameter sets and exchange nothing on the
data path; the counter-based sampler draws set s identically on every rank
(`sample_params(..., set0=...)`).  What crosses ranks: the max of the timed
region over ranks, and optionally a final gather of per-set results.  The
functions work with any torch.distributed backend (NCCL on GPUs, gloo on
CPU); `device` is where the small exchange tensors live.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def rank_sets(per_rank: int, rank: int) -> tuple[int, int]:
    """Weak scaling: rank r integrates sets [r * per_rank, (r+1) * per_rank)."""
    return rank * per_rank, per_rank


def split_sets(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Strong scaling: n_total sets in contiguous ranges, the first
    n_total % world ranks one set more.  Returns (first set, count)."""
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _ready() -> bool:
    return dist.is_available() and dist.is_initialized()


def barrier(device=None) -> None:
    if _ready():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the value itself on one rank)."""
    if not _ready():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(a: np.ndarray, device=None) -> np.ndarray:
    """Concatenates every rank's array along axis 0 in rank order (the arrays
    may have different lengths); every rank gets the result."""
    if not _ready():
        return a
    world = dist.get_world_size()
    n = torch.tensor([a.shape[0]], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    flat = np.zeros((m,) + a.shape[1:], dtype=a.dtype)
    flat[: a.shape[0]] = a
    t = torch.from_numpy(flat.view(np.uint8).reshape(m, -1)).to(device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out = [p.cpu().numpy().reshape(-1).view(a.dtype).reshape((m,) + a.shape[1:])[:c]
           for p, c in zip(parts, counts)]
    return np.concatenate(out, axis=0)
