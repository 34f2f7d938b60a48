"""Host-side logic for running the discretization on several GPUs (one process per GPU).

Intervals and instances are independent (Sec. VI: multiple shooting makes the
transcription parallel across grid intervals), so the work shards without a
collective on the data path:

* independent batches: every rank linearizes its own instances
  (``instance_range`` gives each rank a contiguous share balanced by cost when
  one batch is split; the benchmark instead gives every rank a full batch,
  i.e. weak scaling);
* one long horizon split across ranks: rank r takes the contiguous intervals
  ``interval_ranges(N, world)[r]``.  The forward linearization needs no
  exchange.  The VJP needs one: the node shared by ranks r and r+1 gets
  gradient contributions from both sides (dL/dx~ gets -w of the left interval,
  dL/dU in node layout gets the u_R part of the left interval and the u_L part
  of the right one), summed by ``merge_cut_rows``; L is a plain sum.

Works with any torch.distributed backend (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


def interval_ranges(N: int, world: int):
    """Contiguous interval ranges [k0, k1) per rank, sizes differing by at most one."""
    if N < world:
        raise ValueError(f"cannot split {N} intervals over {world} ranks")
    base, extra = divmod(N, world)
    out, k0 = [], 0
    for r in range(world):
        k1 = k0 + base + (1 if r < extra else 0)
        out.append((k0, k1))
        k0 = k1
    return out


def instance_range(costs, rank: int, world: int):
    """[start, stop) of the instances rank `rank` takes: contiguous, split where the
    cumulative cost crosses rank/world of the total (costs e.g. N_i * n_sub_i * n_links_i)."""
    c = np.cumsum(np.asarray(costs, dtype=np.float64))
    total = c[-1] if len(c) else 0.0
    bounds = [0] + [int(np.searchsorted(c, total * r / world, side="left")) for r in range(1, world)] + [len(c)]
    return bounds[rank], max(bounds[rank], bounds[rank + 1])


def merge_cut_rows(gX, gU, L=None, group=None):
    """Combine a rank's VJP of its interval range with its neighbours'.

    gX [n_r + 1, n_x~] and gU [n_r + 1, n_u] (node layout) are this rank's
    gradients for its nodes k0..k1.  Rank r sends its last row (node k1, which
    rank r+1 owns) to rank r+1, which adds it to its first row.  Returns
    (gX_owned, gU_owned, L_total): the rows of the nodes this rank owns
    (k0..k1-1, and node N on the last rank) and, if L is given, the sum of L
    over all ranks.  Tensors may live on CPU (gloo) or GPU (NCCL)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    reqs = []
    if rank + 1 < world:
        sx, su = gX[-1].contiguous(), gU[-1].contiguous()
        reqs.append(dist.isend(sx, dst=rank + 1, group=group))
        reqs.append(dist.isend(su, dst=rank + 1, group=group))
    if rank > 0:
        rx = torch.empty_like(gX[0])
        ru = torch.empty_like(gU[0])
        dist.recv(rx, src=rank - 1, group=group)
        dist.recv(ru, src=rank - 1, group=group)
        gX = gX.clone()
        gU = gU.clone()
        gX[0] += rx
        gU[0] += ru
    for r in reqs:
        r.wait()
    if rank + 1 < world:
        gX, gU = gX[:-1], gU[:-1]
    Lt = None
    if L is not None:
        Lt = L.clone().reshape(1)
        dist.all_reduce(Lt, op=dist.ReduceOp.SUM, group=group)
        Lt = Lt[0]
    return gX, gU, Lt


def max_over_ranks(values, device=None, group=None):
    """Element-wise maximum of a list of floats over all ranks (timing: max rank time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.tolist()
