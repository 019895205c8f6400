"""Data-parallel helpers for running the convolution with one process per GPU.

The paper trains ResNet-50 data-parallel with Horovod (Sec. 6.C): every rank
holds a shard of the batch and the same filters. For a convolution that means:

* forward and data gradient: each rank convolves its own images; there is
  nothing to exchange (the sample index n only ever appears on one side of
  the sum defining y and dx);
* weight and bias gradients: dw[k,r,s,c] and db[k] are sums over n, p, q, so
  a rank's result over its shard is a partial sum, and one all-reduce (sum)
  over the ranks gives the gradient of the whole batch.

These helpers hold only that host-side logic (which images a rank owns, the
one exchange, and the timing reduction the benchmark uses); every arithmetic
step on the data runs in the library's kernels. They work with any
torch.distributed backend: NCCL with CUDA tensors on GPUs, gloo with CPU
tensors for the multi-process tests.
"""
from __future__ import annotations

from typing import Iterable, Tuple


def shard(n_total: int, rank: int, world: int) -> Tuple[int, int]:
    """Images [start, stop) of `n_total` owned by `rank` of `world`.

    Contiguous, in rank order, sizes differing by at most one (the first
    n_total % world ranks take one extra image). Raises ValueError on a bad
    rank or world size.
    """
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError(f"bad shard request: n_total={n_total}, rank={rank}, world={world}")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        raise RuntimeError("torch.distributed is not initialised")
    return dist


def all_reduce_sum_(tensors: Iterable, group=None) -> None:
    """Adds each tensor across the ranks of `group`, in place (the one
    exchange of data-parallel training: the weight and bias gradients).

    Every rank must pass tensors of the same shapes and dtypes, in the same
    order, on the device its backend uses. With a single rank it is a no-op.
    """
    dist = _dist()
    if dist.get_world_size(group) == 1:
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest `value` over the ranks (a step time: the job is as slow as
    its slowest rank). Returns `value` unchanged when torch.distributed is not
    initialised. `device`: where the one-element tensor lives (the backend's
    device: "cuda" for NCCL, "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def weak_scaling_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of a weak-scaling run: every rank processes
    `units_per_rank`, the job takes `seconds` (the maximum over ranks)."""
    if seconds <= 0 or world < 1:
        raise ValueError("seconds must be positive and world at least 1")
    return units_per_rank * world / seconds
