"""One BC job split over several GPUs, one process (rank) per GPU.

Sources are independent units of the computation (the paper's computeBC loops
over its source set, Appendix A), so the job shards with no exchange until the
end: every rank holds the whole graph, runs its share of the job's batches
through bc_compute_ex, and the ranks' partial BC vectors are summed once, in
rank order, by bc_reduce_ranks.  The only collectives are a small status
exchange and one all-gather of n doubles per rank (torch.distributed: NCCL
between GPUs).  Everything here is marshalling and plumbing; the arithmetic
runs in libbc's kernels.

Split: the job's batch order comes from bc_source_batches (the order and width
a single-GPU call would use); batch b goes to rank b mod world.  Each rank's
columns therefore hold exactly the sources, in the same batches, that the
single-GPU call would traverse, so every per-source dependency is the same;
only the order in which they add into BC differs (rank partials first, then
the rank-order sum), which rounds within the parity tolerance.
"""
from __future__ import annotations

import numpy as np

from . import BC_E_CUDA, BC_OK, BCError, reduce_ranks, status_string


def shard_of(order: np.ndarray, K: int, rank: int, world: int) -> np.ndarray:
    """The sources of rank `rank`: batches b = rank, rank + world, ... of `order` (K per batch), in order."""
    order = np.asarray(order, dtype=np.int32)
    nb = (len(order) + K - 1) // K
    parts = [order[b * K:(b + 1) * K] for b in range(rank, nb, world)]
    return np.concatenate(parts).astype(np.int32) if parts else np.empty(0, np.int32)


def worst_status(statuses) -> int:
    """One status for the job: the first rank's error if any rank failed, else the largest warning."""
    statuses = [int(x) for x in statuses]
    errors = [x for x in statuses if x < 0]
    return errors[0] if errors else max(statuses + [BC_OK])


def exchange_statuses(status: int, group=None, device="cpu") -> int:
    """Every rank learns every rank's status before any rank touches the partials."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.tensor([int(status)], dtype=torch.int32, device=device)
    allst = [torch.zeros(1, dtype=torch.int32, device=device) for _ in range(world)]
    dist.all_gather(allst, mine, group=group)
    return worst_status(int(t.item()) for t in allst)


def gather_partials(part, group=None):
    """[world][n] tensor of every rank's partial BC, row r = rank r's (same device as `part`)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rows = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(rows, part.contiguous(), group=group)
    return torch.stack(rows)


def compute(graph, sources, out=None, group=None, stream=None, **opts):
    """BC over `sources` on `graph` (a Graph resident on this rank's GPU), split
    over the ranks of `group`.  Every rank passes the same source list and gets
    the whole result in `out`.  Returns (out, status)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    order, K = graph.source_batches(sources, stream=stream, batch_width=opts.get("batch_width", 0),
                                    source_order=opts.get("source_order", 0))
    mine = shard_of(order, K, rank, world)
    run = dict(opts, batch_width=K, source_order=1)
    status, local_error = BC_OK, None
    try:
        part = torch.zeros(graph.n, dtype=torch.float64, device="cuda")
        if len(mine):
            _, status = graph.compute(mine, out=part, stream=stream, **run)
    except BCError as err:
        status, local_error = err.status, err
    except Exception as err:  # anything else still reaches the other ranks as a failed status
        status, local_error = BC_E_CUDA, err
    job = exchange_statuses(status, group, device="cuda")
    if job < 0:
        if local_error is not None:
            raise local_error
        raise BCError(job, f"another rank failed: {status_string(job)}")
    parts = gather_partials(part, group)
    out = reduce_ranks(parts, out=out, stream=stream)
    return out, job
