"""Host logic of the multi-GPU benchmark path: one independent lattice per
rank ("replicas only": the single-lattice path does not shard on one B300,
and replicas need no data exchange), timed together.

The only collectives are the timing barrier and a max over ranks of the
measured times; the result is whole-job throughput under weak scaling
(each rank keeps its own lattice, so total work grows with the rank count).
"""
from typing import Sequence, Tuple


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's lattice: base + r (independent Philox keys)."""
    return (base_seed + rank) & (2**64 - 1)


def max_over_ranks(values: Sequence[float], device=None) -> Tuple[float, ...]:
    """Element-wise maximum of per-rank timings (all ranks get the result).
    Works with any initialised torch.distributed backend (gloo on CPU,
    NCCL with `device` on GPUs); without one it returns the input."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return tuple(float(v) for v in values)
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return tuple(float(v) for v in t.tolist())


def weak_scaling_value(world: int, sites_per_rank: float, steps: int, max_ms: float) -> float:
    """Whole-job spin-flip attempts per ns: all ranks' sites times steps,
    divided by the slowest rank's time."""
    return world * sites_per_rank * steps / (max_ms * 1e6)
