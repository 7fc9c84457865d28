"""Aux-sharded Fock build across processes, one GPU each.

J = sum_P w_P B_P and K = sum_P X_P X_P^T are sums over the auxiliary index,
so the three-index tensor partitions by aux rows (the per-GPU partition of
the CD-ERIs, paper Sec. 2.2.2; near-linear multi-GPU scaling, Sec. 3.2): each
process builds a DF handle holding its rows [P0, P1) (bqc_df_build with an
aux range), bqc_jk returns the partial J and K of those rows, and one
all-reduce per Fock build sums the partials.  This module holds only the
host-side plumbing: the row ranges and the all-reduce (torch.distributed;
NCCL between GPUs, gloo on the CPU).
"""
from __future__ import annotations

from typing import List, Tuple


def aux_ranges(naux: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous aux row ranges [P0, P1), as equal as possible, covering
    [0, naux) once (the per-build work of a shard is proportional to its
    rows)."""
    if world < 1 or naux < world:
        raise ValueError("need 1 <= world <= naux")
    base, extra = divmod(naux, world)
    out, p = [], 0
    for r in range(world):
        q = p + base + (1 if r < extra else 0)
        out.append((p, q))
        p = q
    return out


def allreduce_jk(J, K, group=None):
    """Sums the partial J and K of every rank in place with one all-reduce
    over a packed buffer (2 N^2 values)."""
    import torch
    import torch.distributed as dist
    n2 = J.numel()
    buf = torch.cat([J.reshape(-1), K.reshape(-1)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    # copy back through shaped views: J and K may have any strides
    J.copy_(buf[:n2].view(J.shape))
    K.copy_(buf[n2:].view(K.shape))
    return J, K


def sharded_jk(df, Cocc, prec, group=None):
    """J and K of the whole tensor from this rank's shard handle: the local
    partials (bqc_jk) followed by allreduce_jk."""
    J, K = df.jk(Cocc, prec)
    return allreduce_jk(J, K, group)
