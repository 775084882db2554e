"""Sharding of the mocks across ranks (one process per GPU).

Mocks are independent: every rank counts its own contiguous range of mocks
with no collective (weak scaling); the only exchange is gathering the
per-mock correlation-function rows before the covariance, which needs all
mocks (Eqs. bruteforce, R1R2, LCdef).  The functions here are backend-agnostic
(NCCL on GPUs, gloo on CPU) and hold no arithmetic of the method.
"""
from __future__ import annotations

import torch


def mock_range(rank: int, per_rank: int) -> range:
    """Global mock indices owned by `rank` when every rank holds `per_rank` mocks."""
    return range(rank * per_rank, (rank + 1) * per_rank)


def gather_rows(local: torch.Tensor, world: int) -> torch.Tensor:
    """Concatenate every rank's [n, ...] rows in rank order (all_gather along dim 0)."""
    if world == 1:
        return local
    import torch.distributed as dist
    out = torch.empty((world * local.shape[0],) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(out, local.contiguous())
    return out
