"""One APD split across ranks by slabs of the grid's last axis.

The per-cell sums of eq. (2.7) (count, sum of u, sum of u u^T per cell) are the
only data that couple pixels, and they add up over disjoint sets of pixels.  So
each rank (one process, one GPU) scores the contiguous slab
``apd_shard_range(res, rank, world)`` of every grid the solve uses, and one
int64 sum-allreduce of the n x K moment words per evaluation gives every rank
the full moments; the dual, its gradient and L-BFGS then run identically on all
ranks.  Integer sums make the result bit-for-bit independent of the split.

This module only marshals: it turns the library's device pointers into torch
tensors without copying and hands them to ``torch.distributed.all_reduce``.
"""
from __future__ import annotations

from . import capi


class _CudaArray:
    """A device buffer described by the CUDA array interface (no copy)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, count: int, dtype: str = "int64"):
    """A torch CUDA tensor aliasing ``count`` values at device address ``ptr``."""
    import torch
    typestr = {"int64": "<i8", "float64": "<f8"}[dtype]
    return torch.as_tensor(_CudaArray(ptr, count, typestr), device="cuda")


def _stream_of(ptr: int):
    import torch
    return torch.cuda.ExternalStream(ptr) if ptr else torch.cuda.default_stream()


def allreduce_hook(group=None):
    """A reduction hook (capi.REDUCE_FN) that sums the moments over the ranks of
    ``group`` with torch.distributed (NCCL for CUDA tensors), ordered on the
    library's stream."""
    import torch.distributed as dist

    def hook(ctx, mom_ptr, words, seeds, stream_ptr):
        try:
            import torch
            t = device_view(mom_ptr, words, "int64")
            with torch.cuda.stream(_stream_of(stream_ptr)):
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return 0
        except Exception:  # noqa: BLE001 - reported to the library as a failed reduction
            return 1

    return capi.REDUCE_FN(hook)


def slab_range(res: int, rank: int, world: int):
    """(k_begin, k_count) of rank's slab (the library's rule)."""
    return capi.apd_shard_range(res, rank, world)


def shard_workspace(ws: "capi.Workspace", rank: int, world: int, group=None):
    """Make ``ws`` score rank's slab and sum the moments over the ranks."""
    ws.set_shard(rank, world, allreduce_hook(group) if world > 1 else None)
    return ws


__all__ = ["device_view", "allreduce_hook", "slab_range", "shard_workspace"]
