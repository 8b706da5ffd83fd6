"""Data-parallel training over the ray batch: one process per GPU.

Each rank holds a full replica of the octree, the feature table and the
network parameters, and trains on its own shard of the batch's rays. The
method's one exchange step sits between the backward and Adam:

1. each rank evaluates the loss of its shard divided by the WHOLE batch's ray
   count (svlf_loss with n_total, i.e. the C call svlf_loss_shard), so the
   shards' losses and gradients sum exactly to the batch's mean loss and
   its gradient;
2. the feature and network gradients live in one contiguous float32 buffer
   (GradientBuffer), and one all-reduce (sum) over it gives every rank the
   batch's gradient (NCCL between GPUs; gloo on CPU);
3. every rank then runs the same Adam step on identical inputs, so the
   replicas stay identical without exchanging parameters.

Rendering needs no exchange (rays are independent): ranks render their own
rays. The paper trains on one GPU (Sec. 4.5); this is the scale-out form of
its training step, not a different method.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import torch


class GradientBuffer:
    """One contiguous float32 buffer holding the gradients of every trained
    table, in the given order, with a view per table (what the backward
    kernels accumulate into)."""

    def __init__(self, shapes: Sequence[Tuple[int, ...]], device=None, dtype=torch.float32):
        sizes = [int(torch.Size(s).numel()) for s in shapes]
        # keep every float32 view 16-byte aligned for the kernels' vector reductions
        offs, off = [], 0
        for n in sizes:
            offs.append(off)
            off += (n + 3) // 4 * 4
        self.flat = torch.zeros(off, dtype=dtype, device=device)
        self.views = [self.flat[o:o + n].view(s) for o, n, s in zip(offs, sizes, shapes)]

    def zero_(self):
        self.flat.zero_()
        return self


def shard(n_total: int, rank: int, world: int) -> slice:
    """Rank `rank`'s contiguous share of n_total rays (sizes differ by at
    most one)."""
    base, extra = divmod(int(n_total), int(world))
    begin = rank * base + min(rank, extra)
    return slice(begin, begin + base + (1 if rank < extra else 0))


def allreduce_gradients(buf: GradientBuffer, group: Optional[object] = None) -> GradientBuffer:
    """Sums the ranks' gradient buffers in place (one collective over the
    contiguous buffer). Each rank's buffer must hold the gradient of its
    shard's loss divided by the batch's total ray count."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(buf.flat, op=dist.ReduceOp.SUM, group=group)
    return buf
