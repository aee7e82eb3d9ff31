"""Host-side helpers of the multi-GPU path: one process per GPU, independent work per rank.

A single tree does not shard: the one-site TDVP sweep is a sequential traversal, so N GPUs
run N replicas.  A batch of independent trees (different Hamiltonian parameters) shards by
tree with no data-path collective.  The only cross-rank operations are the barrier around
the timed region, the maximum of the per-rank times, and an optional gather of per-tree
results on rank 0.  The helpers take the process group that torch.distributed was
initialised with (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import Any, Dict, List, Optional, Sequence, Tuple


def shard_range(n_items: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block [lo, hi) of n_items for this rank; block sizes differ by at most one
    (the first n_items % world ranks take one more)."""
    if world < 1 or not (0 <= rank < world) or n_items < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _device_for_backend():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank float over all ranks (the job's wall time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for_backend())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def gather_to_rank0(obj: Any) -> Optional[List[Any]]:
    """Every rank's object on rank 0 (in rank order), None elsewhere."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out


def merge_shards(parts: Sequence[Dict[int, Any]], n_items: int) -> List[Any]:
    """Per-item results from the ranks' {item index: result} dictionaries, in item order;
    every item must come from exactly one rank."""
    merged: Dict[int, Any] = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise ValueError(f"item {k} computed by two ranks")
            merged[k] = v
    missing = [k for k in range(n_items) if k not in merged]
    if missing:
        raise ValueError(f"items {missing} computed by no rank")
    return [merged[k] for k in range(n_items)]


def aggregate_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * float(units_per_rank) / max_seconds if max_seconds > 0 else 0.0
