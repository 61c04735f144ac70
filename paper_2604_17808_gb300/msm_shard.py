"""Window-sharded MSM across ranks (one process per GPU).

Algorithm 2 (LS-PPG) distributes its windows over devices: the windows are
independent until the window merge, so each rank takes a contiguous range of
windows, computes the part sum_{k in its range} 2^(k c) W_k on its GPU
(``msm_execute_windows``), and the ranks all-gather the parts (one point
each, a few hundred bytes) and add them with an MSM whose scalars are all 1.
Every rank ends with the same result.

The arithmetic runs in the CUDA library; this module only assigns ranges and
moves the parts (``torch.distributed``: NCCL for GPU tensors).
"""

from __future__ import annotations


def window_range(num_windows: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced share [begin, end) of rank ``rank`` of ``world``
    ranks; the shares of all ranks partition [0, num_windows)."""
    if world < 1 or not 0 <= rank < world or num_windows < 0:
        raise ValueError("bad rank or world size")
    base, extra = divmod(num_windows, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def sum_points(points, curve: str):
    """Sum of the points of a [m, words] device tensor (affine, standard form):
    an MSM with all-one scalars on the GPU."""
    import torch

    from . import MsmPlan

    m = points.shape[0]
    ones = torch.zeros((max(m, 1), 4), dtype=torch.int64, device=points.device)
    ones[:, 0] = 1
    with MsmPlan(max(m, 1), curve=curve) as plan:
        out = plan.execute(ones, points.contiguous(), count=m)
        return out.clone()


def sharded_msm(plan, scalars, points, count: int | None = None, group=None, partial_fn=None, sum_fn=None):
    """MSM of ``scalars`` and ``points`` with this rank's share of the windows
    on its GPU, the parts gathered from every rank of ``group`` and added.

    ``plan`` is an ``MsmPlan`` (the same window size on every rank).  Without
    an initialised process group the call is the whole MSM on one GPU.
    ``partial_fn(begin, end)`` and ``sum_fn(stacked_parts)`` replace the GPU
    calls (used by the CPU tests of the host logic)."""
    import torch
    import torch.distributed as dist

    distributed = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if distributed else 1
    rank = dist.get_rank(group) if distributed else 0
    n = scalars.shape[0] if count is None else int(count)
    begin, end = window_range(plan.info()["num_windows"], rank, world)
    if partial_fn is not None:
        part = partial_fn(begin, end)
    else:
        part = plan.execute_windows(scalars, points, begin, end, count=n)
    if world == 1:
        return part
    parts = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(parts, part.contiguous(), group=group)
    stacked = torch.stack(parts)
    if sum_fn is not None:
        return sum_fn(stacked)
    return sum_points(stacked, plan.curve)
