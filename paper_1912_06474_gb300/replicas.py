"""Replicated rendering over several processes (one per GPU).

The path shards without any exchange: renders, pixels and samples are
independent units (Sec. 5, the classical split by pixels), so N processes each
take a disjoint subset of the renders, run them through their own context, and
the host gathers the images. Nothing here sits on a kernel's data path; the
only collective is the host-side gather of finished images.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def render_cost(spec) -> int:
    """Work estimate of one render: paths x maximum depth."""
    return int(spec.width) * int(spec.height) * int(spec.spp) * max(1, int(spec.max_depth))


def shard_renders(costs: Sequence[int], world: int) -> List[List[int]]:
    """Assign render indices to ``world`` ranks: longest job first onto the
    least-loaded rank (ties to the lower rank), so the slowest rank's load is
    at most 4/3 of the optimum. Every index lands on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-int(costs[i]), i))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(costs[i])
    return [sorted(p) for p in parts]


def my_renders(specs, rank: int, world: int) -> List[int]:
    """The render indices this rank takes."""
    return shard_renders([render_cost(s) for s in specs], world)[rank]


def gather_images(local: Dict[int, "object"], n_renders: int, dst: int = 0):
    """Collect {render index: image (host array)} from every rank on ``dst``.
    Returns the list of all ``n_renders`` images on ``dst`` and None elsewhere.
    Uses torch.distributed's object gather (gloo or NCCL process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [local[i] for i in range(n_renders)]
    world = dist.get_world_size()
    rank = dist.get_rank()
    box = [None] * world if rank == dst else None
    dist.gather_object(local, box, dst=dst)
    if rank != dst:
        return None
    out = [None] * n_renders
    for part in box:
        for i, img in part.items():
            if out[i] is not None:
                raise RuntimeError(f"render {i} returned by two ranks")
            out[i] = img
    missing = [i for i, img in enumerate(out) if img is None]
    if missing:
        raise RuntimeError(f"renders {missing} returned by no rank")
    return out
