"""Sharded residual across processes (the multi-GPU split of the paper's
Sec. III): each rank's context evaluates one shard of the residual
(thc_config.shard_index / shard_count) and the partial sigma^WX, Omega1 and
energy are summed over the ranks with one all-reduce.

Argument marshalling and the collective only; every step of the residual
runs in the CUDA library.  With the nccl backend the sum runs on the device
tensors, with gloo on host copies.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n: int, index: int, count: int):
    """[lo, hi) of the contiguous block of n items owned by shard `index` of
    `count` (the split the library uses for Cholesky vectors and rows X)."""
    return n * index // count, n * (index + 1) // count


def allreduce_parts(sig, sig1, energy, group=None):
    """Sum (sigma, Omega1, energy) over the ranks of `group`.  sig and sig1
    are numpy arrays or torch tensors (device tensors need the nccl
    backend); returns the summed triple in the same kinds."""
    import torch
    import torch.distributed as dist
    torch_in = hasattr(sig, "data_ptr")
    if torch_in:
        dev = sig.device
        flat = torch.cat([sig.reshape(-1), sig1.reshape(-1),
                          torch.tensor([float(energy)], dtype=sig.dtype, device=dev)])
    else:
        flat = torch.from_numpy(np.concatenate([np.ravel(sig), np.ravel(sig1),
                                                [float(energy)]]).astype(np.float64))
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    n0, n1 = sig.numel() if torch_in else sig.size, sig1.numel() if torch_in else sig1.size
    s = flat[:n0].reshape(sig.shape)
    s1 = flat[n0:n0 + n1].reshape(sig1.shape)
    e = float(flat[n0 + n1])
    if not torch_in:
        s, s1 = s.numpy(), s1.numpy()
    return s, s1, e


def sharded_residual(ctx, Zc, t1, group=None):
    """This rank's shard of the residual at (Zc, t1), summed over `group`:
    the whole projected residual and energy on every rank."""
    sig, sig1, e = ctx.residual(Zc, t1)
    return allreduce_parts(sig, sig1, e, group)
