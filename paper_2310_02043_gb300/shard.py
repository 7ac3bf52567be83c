"""Photon sharding across ranks (one process per GPU).

Photons are independent and their random numbers are keyed by the global
photon index, so splitting one photon budget into contiguous per-rank ranges
changes no path: every rank traces its range of the common budget with the
same seed, the integer texel sums of all ranks add up (exactly) to the
single-GPU sums, and so do the per-light gradients.
"""
from __future__ import annotations


def photon_range(rank: int, world: int, photons_per_rank: int):
    """(n_photons, begin, end): the common budget and this rank's range."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    total = photons_per_rank * world
    begin = rank * photons_per_rank
    return total, begin, begin + photons_per_rank


def device_view(ptr: int, n: int, typestr: str = "<i8"):
    """A torch tensor viewing `n` elements of device memory at `ptr` (no copy),
    e.g. the library's texel accumulator for an in-place all-reduce."""
    import torch

    class _Iface:
        __cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}

    return torch.as_tensor(_Iface(), device="cuda")


def allreduce_sum(tensor, group=None):
    """In-place sum over ranks (integer texel sums add exactly)."""
    import torch.distributed as dist
    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
