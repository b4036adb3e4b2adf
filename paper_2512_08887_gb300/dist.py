"""Multi-GPU host logic: independent replicas, one process per GPU (torch.distributed).

Blocks of a stream, requests and whole arrays are independent (Sec. III-A streaming remark,
Sec. VI on parallel execution), so N GPUs each run their own plan on their own blocks and no data
crosses GPUs. The only collectives are for measurement: a barrier around the timed region and a
maximum of the per-rank times.
"""
from __future__ import annotations


def rank_blocks(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [begin, end) of `total` blocks for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad partition arguments")
    return total * rank // world, total * (rank + 1) // world


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units of all ranks divided by the slowest rank's time (weak scaling)."""
    return units_per_rank * world / max_seconds
