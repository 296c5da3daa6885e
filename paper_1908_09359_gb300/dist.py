"""The one exchange of a multi-GPU job (Algorithm 1, the gradient step of Sec. II B).

Markov chains are independent, so a job shards them over ranks (one GPU each, tensors
replicated, each rank's chains numbered from its ``chain_offset`` so the Philox draws do
not depend on the sharding).  Before every sign-SGD step the float64 sums behind the
gradient (sum E, sum E^2, the sample count, sum G E_loc and sum G per tensor entry) are
added over the ranks; every rank then recomputes the identical gradient and applies the
identical update.  This module only moves those sums: the gradient and the update are
computed by the library (pepsvmc_set_sums / pepsvmc_finalize_sums, pepsvmc_update).
"""
from __future__ import annotations

import numpy as np


class _DeviceArray:
    """A float64 device array of the library exposed to torch without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3,
                                         "strides": None}


def device_sums(ctx):
    """torch views (scalars[3], sumGE[P], sumG[P]) of a context's device sums."""
    import torch
    sc, ge, g = ctx.sums_device()
    P = ctx.n_params
    return (torch.as_tensor(_DeviceArray(sc, 3), device="cuda"), torch.as_tensor(_DeviceArray(ge, P), device="cuda"),
            torch.as_tensor(_DeviceArray(g, P), device="cuda"))


def allreduce_device(ctx, group=None):
    """Sum the context's device sums over the ranks in place (NCCL on the current
    stream) and recompute the gradient from the totals."""
    import torch.distributed as dist
    for t in device_sums(ctx):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    ctx.finalize_sums()


def allreduce_host(scalars, sumGE, sumG, group=None):
    """Sum host float64 sums over the ranks (any backend; gloo on CPU) and return the
    totals as numpy arrays."""
    import torch
    import torch.distributed as dist
    out = []
    for a in (scalars, sumGE, sumG):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.append(t.numpy())
    return tuple(out)
