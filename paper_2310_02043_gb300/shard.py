"""Photon sharding across ranks (one process per GPU).

Photons are independent and their random numbers are keyed by the global
photon index, so splitting one photon budget into contiguous per-rank ranges
changes no path: every rank traces its range of the common budget with the
same seed, the integer texel sums of all ranks add up (exactly) to the
single-GPU sums, and so do the per-light gradients.

``ShardedPass`` is the per-rank hot path of one optimisation step: forward
over the rank's range, an in-place all-reduce of the int64 texel sums (the
one exchange of the method), the objective and adjoint weights from the
summed irradiance (the same on every rank), the adjoint over the rank's range
and a reduction of the per-light gradient: either an all-reduce of the
doubles (asynchronous, on the device) or, with ``exact=True``, an all-gather
of every rank's exact 128-bit gradient sums added as integers on the host,
which gives every rank the gradient of a single pass over the whole budget
bit for bit.
"""
from __future__ import annotations

import numpy as np


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


class ShardedPass:
    """One rank's part of a photon-sharded forward + objective + adjoint.

    tracer       an object with the Tracer methods trace_forward, loss and
                 trace_adjoint (lighttrace.Tracer, or a stand-in in tests)
    accumulator  a torch tensor aliasing the tracer's int64 texel sums
                 (``device_view`` of lt_texel_accumulator for the library);
                 summed in place over the ranks after every forward pass
    exact        reduce the gradient through the tracer's exact sums
                 (gradient_fixed) instead of summing doubles; this
                 synchronises the host once per adjoint pass
    With world == 1 nothing is exchanged and no process group is needed."""

    def __init__(self, tracer, rank: int, world: int, photons_per_rank: int, hits: int, accumulator=None,
                 group=None, exact: bool = False):
        self.tracer, self.rank, self.world, self.hits, self.group = tracer, rank, world, hits, group
        self.exact = exact
        self.n_total, self.begin, self.end = photon_range(rank, world, photons_per_rank)
        if world > 1 and accumulator is None:
            raise ValueError("several ranks need the texel accumulator to sum")
        self.q = accumulator

    def forward(self, seed: int):
        """Alg. 1 over this rank's photons, then the texel sums of all ranks."""
        self.tracer.trace_forward(seed, self.n_total, self.hits, self.begin, self.end)
        if self.world > 1:
            allreduce_sum(self.q, self.group)

    def loss(self, out=None):
        """Eq. 6 on the summed texels (every rank forms the same weights)."""
        return self.tracer.loss(out=out) if out is not None else self.tracer.loss()

    def adjoint(self, seed: int, out=None):
        """Alg. 2 over this rank's photons; returns dO/dp summed over ranks
        (into `out` when given: a float64 tensor or numpy array)."""
        g = self.tracer.trace_adjoint(seed, self.n_total, self.hits, self.begin, self.end, out=out)
        if self.world > 1 and self.exact:
            total = self._exact_sum()
            if isinstance(g, np.ndarray):
                g[...] = total
            else:
                import torch
                g.copy_(torch.from_numpy(total))
        elif self.world > 1:
            if isinstance(g, np.ndarray):
                import torch
                import torch.distributed as dist
                t = torch.from_numpy(g)             # aliases g
                if dist.get_backend(self.group) == "nccl":
                    d = t.cuda()
                    allreduce_sum(d, self.group)
                    t.copy_(d.cpu())
                else:
                    allreduce_sum(t, self.group)
            else:
                allreduce_sum(g, self.group)
        return g

    def _exact_sum(self):
        """Every rank's exact gradient sums, gathered and added as integers,
        converted once (all ranks share the weights and lights, so the scale)."""
        import torch
        import torch.distributed as dist
        from .lighttrace import fixed_to_ints, gradient_from_fixed
        sums, scale = self.tracer.gradient_fixed()
        t = torch.from_numpy(np.ascontiguousarray(sums, np.int64))
        if dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        parts = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(parts, t, group=self.group)
        total = None
        for part in parts:
            ints = fixed_to_ints(part.cpu().numpy())
            total = ints if total is None else total + ints
        return gradient_from_fixed(total, scale)

    def step(self, seed_fwd: int, seed_adj: int, grad_out=None, loss_out=None):
        """Forward, objective and adjoint: returns (objective, gradient)."""
        self.forward(seed_fwd)
        O = self.loss(loss_out)
        g = self.adjoint(seed_adj, grad_out)
        return O, g
