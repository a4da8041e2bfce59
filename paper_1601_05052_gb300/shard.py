"""Host-side logic for dedispersing beams on several GPUs, one process each.

Beams are independent (the paper, Sections II and III-A), so the forward
needs no exchange: rank r dedisperses its own contiguous share of the beams.
Only two reductions exist: the slowest rank's time defines a step, and a
weight gradient summed over beams that live on different ranks is an
all-reduce of n_chan floats.
"""
import torch
import torch.distributed as dist


def beams_for_rank(n_beams: int, rank: int, world: int) -> range:
    """Contiguous share of beams for `rank`; shares differ by at most one beam."""
    if not (0 <= rank < world) or n_beams < 0:
        raise ValueError("bad rank/world/beam count")
    base, extra = divmod(n_beams, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (a step lasts as long as its slowest rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_grad_w(gw: torch.Tensor) -> torch.Tensor:
    """Sums per-rank weight gradients in place (weights are shared by all beams)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(gw, op=dist.ReduceOp.SUM)
    return gw
