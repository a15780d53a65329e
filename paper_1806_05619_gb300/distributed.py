"""Several GPUs: the R randomly shifted rules are independent replicas of the
estimator (Sec. 3.2: one shift, one randomised lattice rule), so ranks take
disjoint ranges of shifts, run their samples with no communication, and one
sum of the (L+1) x R x 2 reuse sums per round (eq. Upsilon-reuse) joins them;
the estimator then follows from the joined sums (eqs. MGMLQMC,
var_of_mgmlqmc). Host logic only: the collective is torch.distributed's
(NCCL between GPUs, gloo between CPU processes)."""
from __future__ import annotations

from typing import List, Sequence, Tuple

Work = Tuple[int, int, int, int, int]  # (level, n_begin, n_end, r_begin, r_end)


def shift_range(R: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous block of shifts [r0, r1) of `rank` among `world` ranks."""
    if not (0 <= rank < world) or R < 1:
        raise ValueError("need 0 <= rank < world and R >= 1")
    return rank * R // world, (rank + 1) * R // world


def shard_work(work: Sequence[Work], R: int, rank: int, world: int) -> List[Work]:
    """The part of a work list whose shifts fall in this rank's range."""
    r0, r1 = shift_range(R, rank, world)
    out = []
    for (lv, nb, ne, rb, re_) in work:
        a, b = max(rb, r0), min(re_, r1)
        if a < b and nb < ne:
            out.append((lv, nb, ne, a, b))
    return out


def allreduce_sums(sums, group=None):
    """Sum the reuse sums over all ranks in place (each (level, shift) entry
    comes from the one rank that owns the shift, so the result is exact)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums
