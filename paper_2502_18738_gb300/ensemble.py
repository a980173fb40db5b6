"""Shared-parameter ensembles over several processes (one GPU each): every rank runs its
own fires or realisations through pf_forward / pf_backward, and the gradients of the
shared parameters (p_h, c1, c2, a) are summed over the ranks with one FP64 all-reduce of
32 bytes. The fires themselves exchange nothing; this is the only collective of the path.
Uses torch.distributed (NCCL between GPUs, gloo on CPU)."""
from __future__ import annotations

import torch


def allreduce_param_grads(grad_params, group=None, device=None):
    """Sum the four parameter gradients of this rank (a sequence of 4 floats, as
    pf_backward returns them) over every rank of `group` in FP64; returns the sums as a
    list of 4 floats on every rank. `device`: where the 32-byte buffer lives (the rank's
    CUDA device for NCCL, the CPU for gloo; default: CUDA when available)."""
    import torch.distributed as dist
    if device is None:
        device = "cuda" if torch.cuda.is_available() and dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in grad_params], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.cpu()]
