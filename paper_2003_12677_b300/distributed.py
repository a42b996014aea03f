"""Slice distribution over processes (one GPU each), following Sec. 3.1.

Slices are independent, so ranks need no exchange while they iterate.  The
paper's rule: a process handles at most `chunk` slices per loop; when the
stack holds more slices than all processes can take at once, every process
loops over similar-size chunks, and only the last loop chunk is split
unequally, with the last ranks receiving one slice less than the first ones.

`slice_plan` gives each rank's slice ranges; `gather_slices` collects the
per-rank results on rank 0 through torch.distributed (NCCL for CUDA tensors,
gloo for CPU tensors).  Each rank builds its own copy of the projector: the
build is deterministic, so every replica is bit-identical.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import torch
import torch.distributed as dist


def slice_plan(n_z: int, world: int, chunk: Optional[int] = None) -> List[List[Tuple[int, int]]]:
    """Per-rank lists of [begin, end) slice ranges, one range per loop.

    chunk: at most this many slices per rank per loop (None: one loop)."""
    if n_z < 0 or world < 1:
        raise ValueError("n_z >= 0 and world >= 1 required")
    per = max(1, -(-n_z // world)) if chunk is None else int(chunk)
    if per < 1:
        raise ValueError("chunk must be >= 1")
    plan: List[List[Tuple[int, int]]] = [[] for _ in range(world)]
    start = 0
    while start < n_z:
        rem = n_z - start
        if rem >= per * world:
            sizes = [per] * world
        else:
            # last loop: split the remainder as evenly as possible, the first
            # ranks taking one slice more than the last ones
            q, r = divmod(rem, world)
            sizes = [q + (1 if k < r else 0) for k in range(world)]
        for k, sz in enumerate(sizes):
            if sz > 0:
                plan[k].append((start, start + sz))
            start += sz
    return plan


def rank_slices(n_z: int, world: int, rank: int, chunk: Optional[int] = None) -> List[int]:
    """Flat list of the slice indices one rank owns."""
    return [s for b, e in slice_plan(n_z, world, chunk)[rank] for s in range(b, e)]


def world_rank() -> Tuple[int, int]:
    """(world size, rank) of the default process group; (1, 0) when there is
    none (a single process)."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def gather_slices(local: torch.Tensor, n_z: int, chunk: Optional[int] = None, dst: int = 0) -> Optional[torch.Tensor]:
    """Assemble (n_z, ...) on rank `dst` from each rank's (n_local, ...) results
    (ordered like rank_slices).  Other ranks return None.  A single process
    (no process group) owns every slice in order: `local` is the stack."""
    world, rank = world_rank()
    if world == 1:
        return local
    owned = [rank_slices(n_z, world, k, chunk) for k in range(world)]
    tail = tuple(local.shape[1:])
    maxn = max(len(o) for o in owned)
    pad = torch.zeros((maxn,) + tail, dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)] if rank == dst else None
    dist.gather(pad, bufs, dst=dst)
    if rank != dst:
        return None
    out = torch.empty((n_z,) + tail, dtype=local.dtype, device=local.device)
    for k in range(world):
        for i, s in enumerate(owned[k]):
            out[s] = bufs[k][i]
    return out


def solve_sharded(solve: Callable[[torch.Tensor], torch.Tensor], sino: torch.Tensor, chunk: Optional[int] = None,
                  dst: int = 0, out_shape: Optional[Tuple[int, ...]] = None) -> Optional[torch.Tensor]:
    """One slice stack solved by all ranks (Sec. 3.1): every rank takes its own
    slices of `sino` (n_z, ...) by slice_plan -- loops of at most `chunk`
    slices, the last loop split unevenly -- and runs `solve` on each loop's
    consecutive slices (a callable mapping sinograms (k, ...) to tomograms
    (k, ...), e.g. a CGLS solve with the library's kernels on this rank's GPU);
    rank `dst` gathers the tomograms in stack order and returns them, the other
    ranks return None.  No data moves between ranks while they iterate; the
    gather at the end is the only collective.  out_shape: the shape of one
    tomogram, needed only by a rank that owns no slice (else it solves one
    slice to learn it)."""
    world, rank = world_rank()
    n_z = sino.shape[0]
    outs = [solve(sino[b:e].contiguous()) for b, e in slice_plan(n_z, world, chunk)[rank]]
    if outs:
        local = torch.cat(outs)
    elif out_shape is not None:  # more ranks than slices: this rank contributes nothing
        local = torch.empty((0,) + tuple(out_shape), dtype=sino.dtype, device=sino.device)
    else:
        probe = solve(sino[:1].contiguous()) if n_z else None
        tail = tuple(probe.shape[1:]) if probe is not None else ()
        local = torch.empty((0,) + tail, dtype=probe.dtype if probe is not None else sino.dtype, device=sino.device)
    return gather_slices(local, n_z, chunk, dst)
